"""Pins of the several-control oracle (the five-spin example of Sec. 4): the Liouville-space state form
against the density-matrix form built from the paper's operator definitions, a sigma_y closed form,
reduction to the single-control bit-flip oracle, the trapezoid gradient against finite differences,
and the ISM identities (Theorems 1-2, N-independence).  CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import ism_oracle as O
from oracle import mc_oracle as M


def test_liouville_form_equals_density_matrix_form():
    """The 1024-dimensional state form of the five spins (diagonal generator, X/Y flips on row and
    column bits) reproduces the density-matrix propagation rho -> U rho U^H, J and the gradient."""
    w = W.spin5_liouville(Nt=24, N=3, seed=11, u_amp=300.0)
    psi = M.propagate(w, w.u0, w.psi_i, 0, w.Nt)
    rho = M.dm_forward(w, w.u0)
    for j in (0, 7, 24):
        v = rho[j].T.reshape(-1)   # v[s + 32 s'] = rho[s, s']
        assert np.max(np.abs(psi[j] - v)) < 1e-12
    assert abs(M.objective(w, w.u0)[0] - M.dm_objective(w, w.u0)) < 1e-12
    g = M.global_gradient(w, w.u0)
    g_dm = M.dm_gradient(w, w.u0)
    assert np.max(np.abs(g - g_dm)) < 1e-12 * max(1.0, np.abs(g_dm).max())
    assert np.abs(g_dm).max() > 1e-6   # a non-trivial comparison


def test_density_matrix_form_conserves_trace_and_purity():
    w = W.spin5_liouville(Nt=20, N=2, seed=12, u_amp=300.0)
    rho = M.dm_forward(w, w.u0)
    r0 = rho[0]
    for r in rho[[5, 20]]:
        assert abs(np.trace(r) - np.trace(r0)) < 1e-12
        assert abs(np.trace(r @ r) - np.trace(r0 @ r0)) < 1e-12
        assert np.max(np.abs(r - r.conj().T)) < 1e-12


def _sigma_y(Nt=30, N=5, seed=3):
    rng = np.random.default_rng(seed)
    return W.MCWorkload(name="sy", q=1, H0d=np.zeros(2), ax=np.zeros((1, 1)), ay=np.ones((1, 1)),
                        psi_i=np.array([1.0, 0.0], dtype=np.complex128),
                        psi_f=np.array([0.0, 1.0], dtype=np.complex128), T=1.5, Nt=Nt, N=N,
                        u0=rng.uniform(-1, 1, (Nt, 1)))


def test_sigma_y_closed_form():
    """H = u sigma_y: U_j = [[cos, -sin], [sin, cos]](tau u_j), psi(T) = cos S |0> + sin S |1>,
    S = tau sum u, so J = sin S and dJ/du_j = tau cos S (all U_j commute: the trapezoid is exact),
    also through the sub-problems (beta_n g_n, Theorem 2)."""
    w = _sigma_y()
    S = w.tau * w.u0.sum()
    assert abs(M.objective(w, w.u0)[0] - np.sin(S)) < 1e-14
    assert np.allclose(M.global_gradient(w, w.u0)[:, 0], w.tau * np.cos(S), atol=1e-14)
    phi = M.intermediate_states(w, w.u0)
    g, _ = M.subinterval_all(w, phi, w.u0)
    beta = np.repeat(O.interval_weights(w.T, w.Nt, w.N)[4], np.diff(O.partition(w.Nt, w.N)))
    assert np.allclose(beta * g[:, 0], w.tau * np.cos(S), atol=1e-14)


def test_single_x_control_equals_the_bitflip_oracle():
    """One control with X weights only is the single-control bit-flip problem of the base oracle."""
    rng = np.random.default_rng(8)
    q, Nt, N = 3, 60, 4
    h = rng.uniform(0.5, 1.5, q)
    H0d = rng.uniform(-2, 2, 1 << q)
    u = rng.uniform(-1, 1, Nt)
    psi_i = np.zeros(1 << q, dtype=np.complex128)
    psi_i[0] = 1.0
    f = rng.standard_normal(1 << q) + 1j * rng.standard_normal(1 << q)
    psi_f = f / np.linalg.norm(f)
    mc = W.MCWorkload(name="x", q=q, H0d=H0d, ax=h[None, :], ay=np.zeros((1, q)), psi_i=psi_i, psi_f=psi_f,
                      T=2.0, Nt=Nt, N=N, u0=u[:, None])
    s = np.arange(1 << q)
    H1 = np.zeros((1 << q, 1 << q))
    for b in range(q):
        H1[s, s ^ (1 << b)] += h[b]
    single = W.Workload(name="x1", kind="bitflip", H0=np.diag(H0d), H1=H1, psi_i=psi_i, objective="overlap",
                        psi_f=psi_f, O=None, T=2.0, Nt=Nt, N=N, u0=u)
    assert abs(M.objective(mc, mc.u0)[0] - O.objective(single, u)[0]) < 1e-13
    assert np.max(np.abs(M.global_gradient(mc, mc.u0)[:, 0] - O.global_gradient(single, u))) < 1e-13
    um, Jm, _, _ = M.ism_solve(mc, mc.u0, 3, 0.4)
    us, Js, _, _ = O.ism_solve(single, u, 3, 0.4)
    assert np.max(np.abs(um[:, 0] - us)) < 1e-12 and np.max(np.abs(Jm - Js)) < 1e-12


def test_trapezoid_gradient_is_second_order_against_finite_differences():
    """Every control's trapezoid gradient differs from central differences of the discrete J by
    O(tau^2): the gap falls by ~4 when the same piecewise-constant control is taken on twice the steps."""
    base = W.random_pauli(3, 3, 21, T=1.0, Nt=16, N=2, u_amp=1.0)

    def gap(w):
        g = M.global_gradient(w, w.u0)
        fd = np.empty_like(g)
        h = 1e-5
        for j in range(w.Nt):
            for c in range(w.m):
                vals = []
                for k in (-2, -1, 1, 2):
                    u = w.u0.copy()
                    u[j, c] += k * h
                    vals.append(M.objective(w, u)[0])
                fd[j, c] = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
        return np.linalg.norm(g / w.tau - fd / w.tau) / np.linalg.norm(fd / w.tau)

    e1 = gap(base)
    e2 = gap(base.with_(Nt=32, u0=np.repeat(base.u0, 2, axis=0)))
    assert e1 < 0.05 and 3.0 < e1 / e2 < 5.0, (e1, e2)


def test_theorem1_value_identity():
    w = W.random_pauli(3, 2, 22, T=1.5, Nt=40, N=5)
    phi = M.intermediate_states(w, w.u0)
    _, Jn = M.subinterval_all(w, phi, w.u0)
    beta = O.interval_weights(w.T, w.Nt, w.N)[4]
    assert abs(np.sum(beta * Jn) + 1.0 - M.objective(w, w.u0)[0]) < 1e-12


def test_theorem2_gradient_decomposition():
    w = W.random_pauli(3, 3, 23, T=1.5, Nt=41, N=6)
    phi = M.intermediate_states(w, w.u0)
    g, _ = M.subinterval_all(w, phi, w.u0)
    beta = np.repeat(O.interval_weights(w.T, w.Nt, w.N)[4], np.diff(O.partition(w.Nt, w.N)))
    assert np.max(np.abs(beta[:, None] * g - M.global_gradient(w, w.u0))) < 1e-12


def test_n_independence_and_gradient_method():
    w = W.random_pauli(3, 2, 24, T=1.5, Nt=30, N=1)
    u_ref, J_ref = M.gradient_method(w, w.u0, 3, 0.3)
    for N in (1, 5, 30):
        u, J, _, _ = M.ism_solve(w.with_(N=N), w.u0, 3, 0.3)
        assert np.max(np.abs(u - u_ref)) < 1e-12 and np.max(np.abs(J - J_ref)) < 1e-12


def test_spin5_rho_increases_J():
    """The step size of the five-spin problem (rho = 100 with u += rho g / tau) increases J
    monotonically over 5 gradient iterations (density-matrix form, Nt = 1024 at the same T)."""
    w = W.spin5_liouville(Nt=1024, N=8)
    u = w.u0.copy()
    J = [M.dm_objective(w, u)]
    for _ in range(5):
        u = u + 100.0 * M.dm_gradient(w, u) / w.tau
        J.append(M.dm_objective(w, u))
    assert np.all(np.diff(J) > 0), J
