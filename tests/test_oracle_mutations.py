"""Mutation check of the oracle pins.

Each case plants one plausible mistake in an oracle (a wrong sign, a dropped term or factor, a
transposed operand, an off-by-one, the wrong end of an interval) by replacing one function of the
oracle module for the duration of the case, on the CPU.  It then runs that oracle's own pin tests and
asserts that at least one of them fails.  A case that no pin catches would mean the pins leave that
part of the oracle unchecked.  The oracle files themselves are never modified.
"""
import importlib
import inspect
import itertools

import numpy as np
import pytest

from oracle import cn_oracle as C
from oracle import gp_oracle as G
from oracle import ism_oracle as O
from oracle import mc_oracle as M


# ------------------------------------------------------------------------ running the pin tests
def _cases(fn):
    """Expand the parametrize marks of a test function into keyword-argument dicts."""
    marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
    per_mark = []
    for m in marks:
        names, values = m.args[0], m.args[1]
        names = [s.strip() for s in names.split(",")] if isinstance(names, str) else list(names)
        rows = []
        for v in values:
            v = getattr(v, "values", v)                    # pytest.param(...)
            if len(names) == 1 and not (isinstance(v, tuple) and len(v) == 1):
                v = (v,)
            rows.append(dict(zip(names, v)))
        per_mark.append(rows)
    out = []
    for combo in itertools.product(*per_mark):
        kw = {}
        for part in combo:
            kw.update(part)
        out.append(kw)
    return out or [{}]


def _pins(module_name):
    """(id, function, kwargs) for every test function of a pin module, in definition order."""
    mod = importlib.import_module(module_name)
    pins = []
    for name, fn in vars(mod).items():
        if not (name.startswith("test_") and callable(fn)):
            continue
        params = set(inspect.signature(fn).parameters)
        for kw in _cases(fn):
            if params - set(kw) - {"monkeypatch"}:
                continue                                   # needs a fixture this runner lacks
            pins.append((f"{name}{sorted(kw.items()) if kw else ''}", fn, kw))
    return pins


def _first_failing_pin(pins):
    """Run the pins in order; return the id of the first one that fails (None if all pass)."""
    for pid, fn, kw in pins:
        try:
            with pytest.MonkeyPatch.context() as mp:
                args = dict(kw)
                if "monkeypatch" in inspect.signature(fn).parameters:
                    args["monkeypatch"] = mp
                with np.errstate(all="ignore"):
                    fn(**args)
        except pytest.skip.Exception:
            continue
        except (Exception, pytest.fail.Exception):       # an assertion, or any error of the mutant
            return pid
    return None


PIN_MODULES = {O: "test_oracle_pins", C: "test_oracle_cn_pins", G: "test_oracle_gp_pins",
               M: "test_oracle_mc_pins"}


# ------------------------------------------------------------------ mutants of oracle/ism_oracle.py
_iw, _su, _pa, _ta, _pen, _obj = (O.interval_weights, O.step_unitaries, O.propagate_adjoint,
                                   O.terminal_adjoint, O.penalty, O.objective)
_phi, _asm, _sub, _gg, _eg = (O.intermediate_states, O.assembled_intermediate_states, O.subinterval,
                              O.global_gradient, O.exact_gradient)


def _o_ab_swapped(mp):
    def iw(T, Nt, N):
        j, t, a, b, beta = _iw(T, Nt, N)
        return j, t, b, a, beta
    mp.setattr(O, "interval_weights", iw)


def _o_beta_equal_lengths(mp):
    def iw(T, Nt, N):
        j, t, a, b, beta = _iw(T, Nt, N)
        return j, t, a, b, np.full(N, float(N))            # T / (T/N) whatever the partition
    mp.setattr(O, "interval_weights", iw)


def _o_partition_end_off_by_one(mp):
    def part(Nt, N):
        if not (1 <= N <= Nt):
            raise ValueError("need 1 <= N <= Nt")
        return np.array([(n * (Nt - 1)) // N for n in range(N + 1)], dtype=np.int64)
    mp.setattr(O, "partition", part)


def _o_exponent_sign(mp):
    mp.setattr(O, "step_unitaries", lambda w, u, j0, j1: np.conj(_su(w, u, j0, j1)))


def _o_tau_over_nt_minus_one(mp):
    def su(w, u, j0, j1):
        tau = w.T / (w.Nt - 1)
        H = w.H0[None] + np.asarray(u[j0:j1], dtype=np.float64)[:, None, None] * w.H1[None]
        lam, V = np.linalg.eigh(H)
        return (V * np.exp(-1j * tau * lam)[:, None, :]) @ np.conj(np.swapaxes(V, 1, 2))
    mp.setattr(O, "step_unitaries", su)


def _o_adjoint_not_daggered(mp):
    def pa(w, u, chi_end, j0, j1):
        out = np.empty((j1 - j0 + 1, w.d), dtype=np.complex128)
        out[-1] = chi_end
        U = _su(w, u, j0, j1)
        for k in reversed(range(j1 - j0)):
            out[k] = U[k] @ out[k + 1]
        return out
    mp.setattr(O, "propagate_adjoint", pa)
    mp.setattr(O, "DENSE_MAX", 10 ** 9)


def _o_observable_drops_O(mp):
    mp.setattr(O, "terminal_adjoint", lambda w, psi_T: np.asarray(w.psi_f, dtype=np.complex128)
               if w.objective == "overlap" else np.asarray(psi_T, dtype=np.complex128))


def _o_weight_one(mp):
    mp.setattr(O, "weight", lambda w: 1.0)


def _o_penalty_without_half(mp):
    mp.setattr(O, "penalty", lambda w, u: 2.0 * _pen(w, u))


def _o_gradient_penalty_sign(mp):
    tau = lambda w: w.T / w.Nt   # noqa: E731
    mp.setattr(O, "global_gradient", lambda w, u: _gg(w, u) + 2.0 * tau(w) * O._alpha(w) * np.asarray(u))


def _o_gradient_real_part(mp):
    def gg(w, u):
        tau = w.T / w.Nt
        psi = O.forward_trajectory(w, u)
        chi = O.backward_trajectory(w, u, O.terminal_adjoint(w, psi[-1]))
        re = np.real(np.einsum("jk,jk->j", chi.conj(), psi @ w.H1.T))
        return O.weight(w) * 0.5 * tau * (re[1:] + re[:-1]) - tau * O._alpha(w) * np.asarray(u)
    mp.setattr(O, "global_gradient", gg)


def _o_gradient_one_end(mp):
    def gg(w, u):
        tau = w.T / w.Nt
        psi = O.forward_trajectory(w, u)
        chi = O.backward_trajectory(w, u, O.terminal_adjoint(w, psi[-1]))
        im = np.imag(np.einsum("jk,jk->j", chi.conj(), psi @ w.H1.T))
        return O.weight(w) * tau * im[1:] - tau * O._alpha(w) * np.asarray(u)
    mp.setattr(O, "global_gradient", gg)


def _o_phi_renormalised(mp):
    def phi(w, u):
        p = _phi(w, u)
        return p / np.linalg.norm(p, axis=1, keepdims=True)
    mp.setattr(O, "intermediate_states", phi)


def _o_assembly_order_reversed(mp):
    def asm(w, u):
        j, t, a, b, _ = O.interval_weights(w.T, w.Nt, w.N)
        M_ = []
        for n in range(w.N):
            U = O.step_unitaries(w, u, int(j[n]), int(j[n + 1]))
            Mn = np.eye(w.d, dtype=np.complex128)
            for k in range(U.shape[0]):
                Mn = Mn @ U[k]                             # earlier steps on the left
            M_.append(Mn)
        psi = [np.asarray(w.psi_i, dtype=np.complex128)]
        for n in range(w.N):
            psi.append(M_[n] @ psi[n])
        chi = [None] * (w.N + 1)
        chi[w.N] = O.terminal_adjoint(w, psi[w.N])
        for n in reversed(range(w.N)):
            chi[n] = M_[n].conj().T @ chi[n + 1]
        return np.array([a[n] * psi[n] + b[n] * chi[n] for n in range(w.N + 1)])
    mp.setattr(O, "assembled_intermediate_states", asm)


def _o_subproblem_adjoint_from_phi_n(mp):
    def sub(w, phi, u, n):
        shifted = np.array(phi, copy=True)
        shifted[n + 1] = phi[n]
        g, _ = _sub(w, shifted, u, n)
        _, Jn = _sub(w, phi, u, n)
        return g, Jn
    mp.setattr(O, "subinterval", sub)


def _o_subproblem_penalty_unscaled(mp):
    def sub(w, phi, u, n):
        j, _, _, _, beta = O.interval_weights(w.T, w.Nt, w.N)
        g, Jn = _sub(w, phi, u, n)
        tau = w.T / w.Nt
        j0, j1 = int(j[n]), int(j[n + 1])
        al, uu = O._alpha(w)[j0:j1], np.asarray(u[j0:j1], dtype=np.float64)
        return (g - tau * al * uu * (1.0 - 1.0 / beta[n]),
                Jn - 0.5 * tau * float(np.sum(al * uu ** 2)) * (1.0 - 1.0 / beta[n]))
    mp.setattr(O, "subinterval", sub)


def _o_subproblem_value_unweighted(mp):
    def sub(w, phi, u, n):
        g, Jn = _sub(w, phi, u, n)
        j, _, _, _, beta = O.interval_weights(w.T, w.Nt, w.N)
        j0, j1 = int(j[n]), int(j[n + 1])
        tau = w.T / w.Nt
        pen = 0.5 * tau * float(np.sum(O._alpha(w)[j0:j1] / beta[n] * np.asarray(u[j0:j1]) ** 2))
        return g, (Jn + pen) / O.weight(w) - pen
    mp.setattr(O, "subinterval", sub)


def _o_update(sign, with_beta):
    def mutate(mp):
        def it(w, u, rho, L=1):
            j, t, a, b, beta = O.interval_weights(w.T, w.Nt, w.N)
            tau = w.T / w.Nt
            phi = O.intermediate_states(w, u)
            u_next = np.array(u, dtype=np.float64, copy=True)
            err, Jn0 = 0.0, np.empty(w.N)
            for n in range(w.N):
                j0, j1 = int(j[n]), int(j[n + 1])
                local = np.array(u, dtype=np.float64, copy=True)
                for ell in range(L):
                    g, Jn = O.subinterval(w, phi, local, n)
                    if ell == 0:
                        err += float(np.sum(np.abs(g)))
                        Jn0[n] = Jn
                    local[j0:j1] += sign * rho * (beta[n] if with_beta else 1.0) * g / tau
                u_next[j0:j1] = local[j0:j1]
            return u_next, err, Jn0
        mp.setattr(O, "ism_iteration", it)
    return mutate


def _o_err_from_last_local_step(mp):
    def it(w, u, rho, L=1):
        j, t, a, b, beta = O.interval_weights(w.T, w.Nt, w.N)
        tau = w.T / w.Nt
        phi = O.intermediate_states(w, u)
        u_next = np.array(u, dtype=np.float64, copy=True)
        err, Jn0 = 0.0, np.empty(w.N)
        for n in range(w.N):
            j0, j1 = int(j[n]), int(j[n + 1])
            local = np.array(u, dtype=np.float64, copy=True)
            for ell in range(L):
                g, Jn = O.subinterval(w, phi, local, n)
                if ell == 0:
                    Jn0[n] = Jn
                if ell == L - 1:
                    err += float(np.sum(np.abs(g)))
                local[j0:j1] += rho * beta[n] * g / tau
            u_next[j0:j1] = local[j0:j1]
        return u_next, err, Jn0
    mp.setattr(O, "ism_iteration", it)


def _o_exact_gradient_wrong_block(mp):
    def eg(w, u):
        from scipy.linalg import expm
        tau, d = w.T / w.Nt, w.d
        psi = O.forward_trajectory(w, u)
        chi = O.backward_trajectory(w, u, O.terminal_adjoint(w, psi[-1]))
        g = np.empty(w.Nt)
        for j in range(w.Nt):
            A = -1j * tau * (w.H0 + u[j] * w.H1)
            B = expm(np.block([[A, -1j * tau * w.H1], [np.zeros((d, d)), A]]))
            g[j] = O.weight(w) * float(np.vdot(chi[j + 1], B[:d, :d] @ psi[j]).real)   # U, not dU/du
        return g - tau * O._alpha(w) * np.asarray(u)
    mp.setattr(O, "exact_gradient", eg)


def _o_propagator_transposed_h(mp):
    # exp(-i tau H^T): the same for real symmetric H; for complex Hermitian H it is exp(-i tau conj(H))
    def su(w, u, j0, j1):
        return _su(w.with_(H0=w.H0.T, H1=w.H1.T), u, j0, j1)
    mp.setattr(O, "step_unitaries", su)


def _o_gradient_h1_transposed(mp):
    def gg(w, u):
        tau = w.T / w.Nt
        psi = O.forward_trajectory(w, u)
        chi = O.backward_trajectory(w, u, O.terminal_adjoint(w, psi[-1]))
        im = np.imag(np.einsum("jk,jk->j", chi.conj(), psi @ w.H1))   # H1^T psi
        return O.weight(w) * 0.5 * tau * (im[1:] + im[:-1]) - tau * O._alpha(w) * np.asarray(u)
    mp.setattr(O, "global_gradient", gg)


def _o_subproblem_h1_conjugated(mp):
    mp.setattr(O, "subinterval", lambda w, phi, u, n: _sub(w.with_(H1=np.conj(w.H1)), phi, u, n))


def _o_fidelity_not_squared(mp):
    def obj(w, u, psi=None):
        J, F = _obj(w, u, psi)
        return J, (float(np.sqrt(F)) if w.objective == "overlap" else F)
    mp.setattr(O, "objective", obj)


# ------------------------------------------------------------------- mutants of oracle/cn_oracle.py
_c_sm, _c_pa, _c_gt, _c_sub = C.step_matrices, C.propagate_adjoint, C._grad_terms, C.subinterval


def _c_a_b_swapped(mp):
    def sm(w, u_j):
        A, B = _c_sm(w, u_j)
        return B, A
    mp.setattr(C, "step_matrices", sm)


def _c_full_tau_in_cayley(mp):
    def sm(w, u_j):
        tau = w.T / w.Nt
        H = w.H0 + float(u_j) * w.H1
        Id = np.eye(w.d)
        return Id + 1j * tau * H, Id - 1j * tau * H
    mp.setattr(C, "step_matrices", sm)


def _c_xi_solved_with_A(mp):
    def pa(w, u, lam_end, j0, j1):
        lam = np.empty((j1 - j0 + 1, w.d), dtype=np.complex128)
        xi = np.empty((j1 - j0, w.d), dtype=np.complex128)
        lam[-1] = lam_end
        for k in reversed(range(j1 - j0)):
            A, B = C.step_matrices(w, u[j0 + k])
            xi[k] = np.linalg.solve(A, lam[k + 1])
            lam[k] = A @ np.linalg.solve(B, lam[k + 1])
        return lam, xi
    mp.setattr(C, "propagate_adjoint", pa)


def _c_grad_terms_left_state_only(mp):
    mp.setattr(C, "_grad_terms", lambda w, psi, xi: np.imag(np.einsum("jk,jk->j", xi.conj(), (2.0 * psi[:-1]) @ w.H1.T)))


def _c_subproblem_adjoint_from_phi_n(mp):
    def sub(w, phi, u, n):
        shifted = np.array(phi, copy=True)
        shifted[n + 1] = phi[n]
        g, _ = _c_sub(w, shifted, u, n)
        return g, _c_sub(w, phi, u, n)[1]
    mp.setattr(C, "subinterval", sub)


def _c_update_without_beta(mp):
    def it(w, u, rho, L=1):
        j = C.partition(w.Nt, w.N)
        tau = w.T / w.Nt
        phi = C.intermediate_states(w, u)
        u_next = np.array(u, dtype=np.float64, copy=True)
        err = 0.0
        for n in range(w.N):
            j0, j1 = int(j[n]), int(j[n + 1])
            local = np.array(u, dtype=np.float64, copy=True)
            for ell in range(L):
                g, _ = C.subinterval(w, phi, local, n)
                if ell == 0:
                    err += float(np.sum(np.abs(g)))
                local[j0:j1] += rho * g / tau
            u_next[j0:j1] = local[j0:j1]
        return u_next, err
    mp.setattr(C, "ism_iteration", it)


# ------------------------------------------------------------------- mutants of oracle/gp_oracle.py
_g_hk, _g_pdu, _g_pot, _g_sub = G._half_kinetic, G.potential_du, G.potential, G.subinterval


def _g_kinetic_sign(mp):
    mp.setattr(G, "_half_kinetic", lambda w: np.conj(_g_hk(w)))


def _g_full_kinetic_each_side(mp):
    mp.setattr(G, "_half_kinetic", lambda w: _g_hk(w) ** 2)


def _g_adjoint_drops_nonlinear_term(mp):
    def adj(w, lam_next, psi_j, u_j):
        a = G._K(w, psi_j)
        mu = np.exp(1j * w.tau * G._theta(w, a, u_j)) * G._KH(w, lam_next)
        g = w.tau * np.sum(G.potential_du(w, w.x, u_j) * np.imag(np.conj(mu) * a)) * w.dx
        return G._KH(w, mu), float(g)
    mp.setattr(G, "_adjoint_step", adj)


def _g_potential_derivative_sign(mp):
    mp.setattr(G, "potential_du", lambda w, x, u_j: -_g_pdu(w, x, u_j))


def _g_nonlinear_phase_on_unkicked_state(mp):
    def step(w, psi, u_j):
        a = G._K(w, psi)
        return G._K(w, np.exp(-1j * w.tau * (G.potential(w, w.x, u_j) + w.g * np.abs(psi) ** 2)) * a)
    mp.setattr(G, "strang_step", step)


def _g_subproblem_target_chi_n(mp):
    def sub_all(w, psi_t, chi_t, u):
        g = np.empty(w.Nt)
        Jn = np.empty(w.N)
        j = G.partition(w.Nt, w.N)
        for n in range(w.N):
            g[j[n]:j[n + 1]], Jn[n] = G.subinterval(w, psi_t[n], chi_t[n], u, n)
        return g, Jn
    mp.setattr(G, "subinterval_all", sub_all)


def _g_double_well_inner_branch_sign(mp):
    def pot(w, x, u_j):
        if getattr(w, "potential", "harmonic") == "harmonic":
            return _g_pot(w, x, u_j)
        d, ax = w.dw, np.abs(np.asarray(x, dtype=np.float64))
        return np.where(ax > u_j * d / 4.0, 0.5 * (ax - u_j * d / 2.0) ** 2, 0.5 * ((u_j * d) ** 2 / 8.0 + ax ** 2))
    mp.setattr(G, "potential", pot)


def _g_descent(mp):
    def it(w, u, rho, L=1):
        j = G.partition(w.Nt, w.N)
        psi_t, chi_t = G.intermediate_pairs(w, u)
        u_next = np.array(u, dtype=np.float64, copy=True)
        err = 0.0
        for n in range(w.N):
            j0, j1 = int(j[n]), int(j[n + 1])
            local = np.array(u, dtype=np.float64, copy=True)
            for ell in range(L):
                g, _ = G.subinterval(w, psi_t[n], chi_t[n + 1], local, n)
                if ell == 0:
                    err += float(np.sum(np.abs(g)))
                local[j0:j1] -= rho * g / w.tau
            u_next[j0:j1] = local[j0:j1]
        return u_next, err
    mp.setattr(G, "ism_iteration", it)


# ------------------------------------------------------------------- mutants of oracle/mc_oracle.py
_m_p1, _m_pa, _m_it = M.pauli_1q, M.propagate_adjoint, M._im_terms


def _m_y_conjugated(mp):
    mp.setattr(M, "pauli_1q", lambda q, b, a: _m_p1(q, b, a).conj() if a == "Y" else _m_p1(q, b, a))


def _m_bit_order_reversed(mp):
    mp.setattr(M, "pauli_1q", lambda q, b, a: _m_p1(q, q - 1 - b, a))


def _m_adjoint_not_daggered(mp):
    def pa(w, u, chi_end, j0, j1):
        out = np.empty((j1 - j0 + 1, w.d), dtype=np.complex128)
        out[-1] = chi_end
        for k in reversed(range(j1 - j0)):
            out[k] = M._step(w, u[j0 + k], out[k + 1], +1)
        return out
    mp.setattr(M, "propagate_adjoint", pa)


def _m_gradient_one_end(mp):
    def gg(w, u):
        psi = M.propagate(w, u, w.psi_i, 0, w.Nt)
        chi = M.propagate_adjoint(w, u, w.psi_f, 0, w.Nt)
        return w.tau * M._im_terms(w, chi, psi)[1:]
    mp.setattr(M, "global_gradient", gg)


def _m_controls_swapped(mp):
    def im_terms(w, chi, psi):
        out = _m_it(w, chi, psi)
        return out[:, ::-1].copy()                         # gradient of control c reported as m-1-c
    mp.setattr(M, "_im_terms", im_terms)


MUTANTS = [
    (O, "propagator built from H^T (conj(H) for complex Hermitian H)", _o_propagator_transposed_h),
    (O, "gradient applies H1^T", _o_gradient_h1_transposed),
    (O, "sub-problems with conj(H1)", _o_subproblem_h1_conjugated),
    (O, "a_n and b_n swapped in Eq. (cible)", _o_ab_swapped),
    (O, "beta_n taken as N on an uneven partition", _o_beta_equal_lengths),
    (O, "partition ends one step short", _o_partition_end_off_by_one),
    (O, "step exponent exp(+i tau H)", _o_exponent_sign),
    (O, "tau = T/(Nt - 1)", _o_tau_over_nt_minus_one),
    (O, "adjoint propagated with U_j instead of U_j^H", _o_adjoint_not_daggered),
    (O, "observable objective: chi(T) = psi(T) without O", _o_observable_drops_O),
    (O, "weight 1 on the observable's Im-terms", _o_weight_one),
    (O, "control cost without its factor 1/2", _o_penalty_without_half),
    (O, "penalty gradient with the wrong sign", _o_gradient_penalty_sign),
    (O, "gradient from Re instead of Im", _o_gradient_real_part),
    (O, "gradient from one end of each step (no trapezoid)", _o_gradient_one_end),
    (O, "intermediate states renormalised", _o_phi_renormalised),
    (O, "propagator assembly multiplies in the wrong order", _o_assembly_order_reversed),
    (O, "sub-problem adjoint started from phi_n", _o_subproblem_adjoint_from_phi_n),
    (O, "sub-problem penalty alpha not divided by beta_n", _o_subproblem_penalty_unscaled),
    (O, "sub-problem value without the weight w", _o_subproblem_value_unweighted),
    (O, "update without beta_n", _o_update(+1.0, False)),
    (O, "descent instead of ascent", _o_update(-1.0, True)),
    (O, "Err from the last local step", _o_err_from_last_local_step),
    (O, "exact gradient from the wrong block of the Van Loan exponential", _o_exact_gradient_wrong_block),
    (O, "fidelity |<psi(T)|psi_f>| not squared", _o_fidelity_not_squared),
    (C, "Crank-Nicolson matrices A and B swapped", _c_a_b_swapped),
    (C, "Crank-Nicolson with tau H instead of tau H/2", _c_full_tau_in_cayley),
    (C, "adjoint xi_j solved with A_j instead of B_j", _c_xi_solved_with_A),
    (C, "gradient pairs xi_j with 2 psi_j instead of psi_j + psi_{j+1}", _c_grad_terms_left_state_only),
    (C, "sub-problem adjoint started from phi_n", _c_subproblem_adjoint_from_phi_n),
    (C, "update without beta_n", _c_update_without_beta),
    (G, "kinetic half step exp(+i tau k^2/4)", _g_kinetic_sign),
    (G, "full kinetic step on each side of the Strang step", _g_full_kinetic_each_side),
    (G, "adjoint drops the nonlinear term", _g_adjoint_drops_nonlinear_term),
    (G, "potential derivative with the wrong sign", _g_potential_derivative_sign),
    (G, "nonlinear phase from the density before the kinetic half step", _g_nonlinear_phase_on_unkicked_state),
    (G, "sub-problem target chi(t_n) instead of chi(t_{n+1})", _g_subproblem_target_chi_n),
    (G, "double-well inner branch +x^2", _g_double_well_inner_branch_sign),
    (G, "descent instead of ascent", _g_descent),
    (M, "Y conjugated in the Liouville-space operators", _m_y_conjugated),
    (M, "control bits in reversed order", _m_bit_order_reversed),
    (M, "adjoint propagated forward", _m_adjoint_not_daggered),
    (M, "gradient from one end of each step", _m_gradient_one_end),
    (M, "gradients of the controls reported in reversed order", _m_controls_swapped),
]


@pytest.mark.parametrize("module,what,mutate", MUTANTS, ids=[f"{m.__name__.split('.')[-1]}: {w}" for m, w, _ in MUTANTS])
def test_pins_catch_planted_mistake(module, what, mutate):
    pins = _pins(PIN_MODULES[module])
    assert pins
    with pytest.MonkeyPatch.context() as mp:
        mutate(mp)
        caught = _first_failing_pin(pins)
    assert caught is not None, f"no pin of {PIN_MODULES[module]} fails when the oracle has: {what}"


@pytest.mark.parametrize("module", list(PIN_MODULES), ids=[m.__name__.split(".")[-1] for m in PIN_MODULES])
def test_runner_passes_the_unmutated_oracle(module):
    """The runner itself: every pin of the unmodified oracle passes through it."""
    assert _first_failing_pin(_pins(PIN_MODULES[module])) is None
