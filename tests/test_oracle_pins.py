"""Pins of the FP64 oracle against facts that do not come from the oracle itself: textbook closed
forms, a different library routine, finite differences, and the two theorems of Sec. 2 stated as
identities between independently computed quantities.  CPU only."""
import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle import ism_oracle as O


# ----------------------------------------------------------------------------- partition (Sec. 2)
@pytest.mark.parametrize("Nt,N", [(1000, 4), (20000, 64), (20000, 128), (10000, 64), (50000, 256), (7, 7), (5, 1)])
def test_partition_covers_interval(Nt, N):
    j = O.partition(Nt, N)
    assert j[0] == 0 and j[-1] == Nt and len(j) == N + 1
    steps = np.diff(j)
    assert steps.min() >= 1
    assert steps.max() - steps.min() <= 1          # uneven splits differ by one step at most
    _, t, a, b, beta = O.interval_weights(2.5, Nt, N)
    assert np.allclose(a + b, 1.0)
    assert a[0] == 1.0 and b[-1] == 1.0
    assert np.isclose(np.sum(1.0 / beta), 1.0)      # sum (t_{n+1}-t_n)/T = 1


def test_partition_rejects_bad_sizes():
    with pytest.raises(ValueError):
        O.partition(3, 4)
    with pytest.raises(ValueError):
        O.partition(3, 0)


# ------------------------------------------------------------------------- propagator pins
def _rabi_populations(delta, u, t):
    Om = np.sqrt(delta ** 2 + u ** 2)
    return (u ** 2 / Om ** 2) * np.sin(Om * t / 2.0) ** 2


@pytest.mark.parametrize("delta,u", [(1.3, 0.7), (0.0, 2.0), (2.0, -0.4)])
def test_rabi_closed_form(delta, u):
    """H = (delta/2) sz + (u/2) sx, constant u: P_1(t) = (u/Omega)^2 sin^2(Omega t/2)."""
    w = W.rabi(delta, u, T=5.0, Nt=50)
    psi = O.forward_trajectory(w, w.u0)
    t = np.arange(w.Nt + 1) * w.tau
    assert np.allclose(np.abs(psi[:, 1]) ** 2, _rabi_populations(delta, u, t), atol=1e-13)
    if delta == 0.0:   # psi(t) = cos(ut/2)|0> - i sin(ut/2)|1>
        assert np.allclose(psi[:, 0], np.cos(u * t / 2), atol=1e-13)
        assert np.allclose(psi[:, 1], -1j * np.sin(u * t / 2), atol=1e-13)


def test_unitarity_and_norm():
    w = W.random_dense(16, 7, T=3.0, Nt=40, N=4)
    U = O.step_unitaries(w, w.u0, 0, w.Nt)
    eye = np.eye(w.d)
    for k in range(U.shape[0]):
        assert np.allclose(U[k].conj().T @ U[k], eye, atol=1e-13)
    psi = O.forward_trajectory(w, w.u0)
    assert np.allclose(np.linalg.norm(psi, axis=1), 1.0, atol=1e-13)


@pytest.mark.parametrize("d", [2, 5, 16, 41, 64])
def test_step_unitary_matches_pade_expm(d):
    """numpy eigh-based exponential vs scipy's scaling-and-squaring Pade expm."""
    w = W.random_dense(d, 11 + d, T=1.0, Nt=8, N=1, u_amp=3.0)
    U = O.step_unitaries(w, w.u0, 0, w.Nt)
    for k in range(w.Nt):
        ref = expm(-1j * w.tau * (w.H0 + w.u0[k] * w.H1))
        assert np.allclose(U[k], ref, atol=1e-12)


# ------------------------------------------------------------------------- gradient pins
def _sigma_x_problem(Nt=25, N=5, seed=3):
    """H0 = 0, H1 = sx, psi_i = |0>, psi_f = -i|1>: all U_j commute, J = sin(tau sum u) and
    dJ/du_j = tau cos(tau sum u) exactly."""
    rng = np.random.default_rng(seed)
    w = W.rabi(0.0, 0.0, T=2.0, Nt=Nt, N=N)
    w = w.with_(H1=np.array([[0.0, 1.0], [1.0, 0.0]]), psi_f=np.array([0.0, -1j]),
                u0=rng.uniform(-1, 1, Nt))
    return w


def test_sigma_x_closed_form_objective_and_gradient():
    w = _sigma_x_problem()
    th = w.tau * np.sum(w.u0)
    J, F = O.objective(w, w.u0)
    assert np.isclose(J, np.sin(th), atol=1e-14)
    assert np.isclose(F, np.sin(th) ** 2, atol=1e-14)
    g_ref = np.full(w.Nt, w.tau * np.cos(th))
    assert np.allclose(O.global_gradient(w, w.u0), g_ref, atol=1e-14)
    assert np.allclose(O.exact_gradient(w, w.u0), g_ref, atol=1e-14)
    # sub-interval route (Theorem 2): beta_n g_{n,j} is the same number
    phi = O.intermediate_states(w, w.u0)
    g, _ = O.subinterval_all(w, phi, w.u0)
    beta = np.repeat(O.interval_weights(w.T, w.Nt, w.N)[4], np.diff(O.partition(w.Nt, w.N)))
    assert np.allclose(beta * g, g_ref, atol=1e-14)


@pytest.mark.parametrize("objective", ["overlap", "observable"])
def test_exact_gradient_matches_central_differences(objective):
    w = W.random_dense(4, 5, T=2.0, Nt=30, N=3, objective=objective)
    w = w.with_(alpha=np.linspace(0.01, 0.05, w.Nt))
    g = O.exact_gradient(w, w.u0)
    h = 1e-4
    fd = np.empty(w.Nt)

    def J_at(j, s):
        v = w.u0.copy()
        v[j] += s
        return O.objective(w, v)[0]

    for j in range(w.Nt):   # fourth-order central difference
        fd[j] = (8 * (J_at(j, h) - J_at(j, -h)) - (J_at(j, 2 * h) - J_at(j, -2 * h))) / (12 * h)
    assert np.linalg.norm(g - fd) <= 1e-9 * np.linalg.norm(fd)


def test_trapezoid_gradient_is_second_order():
    """(trapezoid - exact) shrinks ~4x when tau halves for a smooth control sampled at midpoints."""
    errs = []
    for Nt in (20, 40, 80):
        w = W.random_dense(4, 9, T=2.0, Nt=Nt, N=1)
        tm = (np.arange(Nt) + 0.5) * w.tau
        u = 0.8 * np.sin(1.7 * tm) + 0.3
        w = w.with_(u0=u)
        # compare L2 gradients (per unit time) so refinement is comparable
        errs.append(np.linalg.norm(O.global_gradient(w, u) - O.exact_gradient(w, u)) / w.tau * np.sqrt(w.tau))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5


# ------------------------------------------------------------------ intermediate states (Eq. cible)
@pytest.mark.parametrize("objective", ["overlap", "observable"])
def test_phi_endpoints_and_assembly(objective):
    w = W.random_dense(6, 21, T=3.0, Nt=47, N=5, objective=objective)
    phi = O.intermediate_states(w, w.u0)
    psi = O.forward_trajectory(w, w.u0)
    assert np.allclose(phi[0], w.psi_i, atol=1e-15)
    assert np.allclose(phi[-1], O.terminal_adjoint(w, psi[-1]), atol=1e-13)
    phiM = O.assembled_intermediate_states(w, w.u0)
    assert np.allclose(phiM, phi, atol=1e-13)


def test_phi_is_not_normalised():
    """||phi_n||^2 = a^2 + b^2 + 2ab Re<psi(t_n)|chi(t_n)>: intermediate states are not unit vectors."""
    w = W.random_dense(6, 22, T=3.0, Nt=40, N=4)
    phi = O.intermediate_states(w, w.u0)
    j, t, a, b, _ = O.interval_weights(w.T, w.Nt, w.N)
    psi = O.forward_trajectory(w, w.u0)
    ov = np.vdot(psi[-1], w.psi_f).real                   # Re<psi(t)|chi(t)> is constant in t
    assert np.allclose(np.linalg.norm(phi, axis=1) ** 2, a ** 2 + b ** 2 + 2 * a * b * ov, atol=1e-13)


# ------------------------------------------------------------------------ Theorems 1 and 2
@pytest.mark.parametrize("N", [1, 3, 8])
def test_theorem1_value_identity_overlap(N):
    """sum_n beta_n J_n[u, phi^u] = J[u] - 1 for unit psi_i, psi_f (the paper's '=' is up to this
    additive constant; the penalty parts sum exactly)."""
    w = W.random_dense(5, 31, T=2.0, Nt=48, N=N)
    w = w.with_(alpha=np.linspace(0.02, 0.2, w.Nt))
    phi = O.intermediate_states(w, w.u0)
    J, _ = O.objective(w, w.u0)
    assert np.isclose(O.j_parallel(w, phi, w.u0), J - 1.0, atol=1e-12)


def test_theorem1_value_identity_observable():
    """Observable objective with weight w=2: sum beta_n J_n = w Re<psi(T)|chi(T)> - (w/2)(||psi_i||^2 +
    ||chi(T)||^2) - penalty, with chi(T) = O psi(T)."""
    w = W.random_dense(5, 32, T=2.0, Nt=48, N=6, objective="observable")
    w = w.with_(alpha=np.linspace(0.02, 0.2, w.Nt))
    phi = O.intermediate_states(w, w.u0)
    psi = O.forward_trajectory(w, w.u0)
    chiT = w.O @ psi[-1]
    expect = 2 * np.vdot(psi[-1], chiT).real - (1.0 + np.linalg.norm(chiT) ** 2) - O.penalty(w, w.u0)
    assert np.isclose(O.j_parallel(w, phi, w.u0), expect, atol=1e-12)


def test_theorem1_argmax():
    """phi^u maximises J_par over interior intermediate states (endpoints fixed)."""
    w = W.random_dense(4, 33, T=2.0, Nt=24, N=4)
    phi = O.intermediate_states(w, w.u0)
    best = O.j_parallel(w, phi, w.u0)
    rng = np.random.default_rng(0)
    for _ in range(10):
        pert = phi.copy()
        pert[1:-1] += 1e-2 * (rng.standard_normal(pert[1:-1].shape) + 1j * rng.standard_normal(pert[1:-1].shape))
        assert O.j_parallel(w, pert, w.u0) < best


@pytest.mark.parametrize("objective,N", [("overlap", 1), ("overlap", 4), ("overlap", 7), ("observable", 5)])
def test_theorem2_gradient_decomposition(objective, N):
    """beta_n * (sub-interval gradient at phi^u) = full-interval gradient on that sub-interval; the two
    sides are computed from different trajectories (p, c from phi vs psi, chi from psi_i, chi(T))."""
    w = W.random_dense(6, 41, T=2.5, Nt=53, N=N, objective=objective)
    w = w.with_(alpha=np.linspace(0.01, 0.1, w.Nt))
    phi = O.intermediate_states(w, w.u0)
    g, _ = O.subinterval_all(w, phi, w.u0)
    beta = np.repeat(O.interval_weights(w.T, w.Nt, w.N)[4], np.diff(O.partition(w.Nt, w.N)))
    G = O.global_gradient(w, w.u0)
    assert np.allclose(beta * g, G, atol=1e-13 * max(1.0, np.abs(G).max()))


def test_n_independence_of_iterates():
    """With one local step (L = 1) the iterates do not depend on N (Sec. 4, first example)."""
    w = W.random_dense(4, 51, T=2.0, Nt=36, N=1)
    res = [O.ism_solve(w.with_(N=N), w.u0, 4, 0.3)[0] for N in (1, 2, 3, 6, 36)]
    for u in res[1:]:
        assert np.allclose(u, res[0], atol=1e-12)


def test_n1_is_the_sequential_gradient_method():
    w = W.random_dense(4, 52, T=2.0, Nt=30, N=1, objective="observable")
    u_ism, J_ism, _, _ = O.ism_solve(w, w.u0, 5, 0.2)
    u_gm, J_gm = O.gradient_method(w, w.u0, 5, 0.2)
    assert np.allclose(u_ism, u_gm, atol=1e-13)
    assert np.allclose(J_ism, J_gm, atol=1e-13)


def test_local_iterations_differ_from_global_step():
    """L > 1 runs several steps on each J_n with phi frozen: iterates then depend on N (no Theorem 2
    equivalence), and the first local step still equals the global one."""
    w = W.random_dense(4, 53, T=2.0, Nt=30, N=3)
    u1, _, _ = O.ism_iteration(w, w.u0, 0.2, L=1)
    u3, _, _ = O.ism_iteration(w, w.u0, 0.2, L=3)
    uN1, _, _ = O.ism_iteration(w.with_(N=1), w.u0, 0.2, L=3)
    assert not np.allclose(u3, u1)
    assert not np.allclose(u3, uN1)


def test_err_is_l1_of_subgradients():
    w = W.random_dense(4, 54, T=2.0, Nt=30, N=3)
    phi = O.intermediate_states(w, w.u0)
    g, _ = O.subinterval_all(w, phi, w.u0)
    _, err, _ = O.ism_iteration(w, w.u0, 0.2)
    assert np.isclose(err, np.abs(g).sum(), rtol=1e-14)


@pytest.mark.parametrize("L", [1, 3])
def test_err_is_taken_at_the_first_local_step(L):
    """Err (Algorithm 1 (e), read as the sub-gradients at u^(k)) does not depend on the number of
    local steps, and by Theorem 2 equals sum_j |g_j| / beta_n(j) with g the full-interval gradient
    (an uneven partition, so that the beta_n differ)."""
    w = W.random_dense(4, 55, T=2.0, Nt=31, N=4)
    j, _, _, _, beta = O.interval_weights(w.T, w.Nt, w.N)
    g_full = O.global_gradient(w, w.u0)
    expected = sum(np.abs(g_full[j[n]:j[n + 1]]).sum() / beta[n] for n in range(w.N))
    _, err, _ = O.ism_iteration(w, w.u0, 0.2, L=L)
    assert np.isclose(err, expected, rtol=1e-11)


# --------------------------------------------------------------------- benchmark configurations
def test_spin16_step_size_is_monotone():
    w = W.config("spin16", iters=6)
    _, J, _, _ = O.ism_solve(w, w.u0, w.iters, w.rho)
    assert np.all(np.diff(J) > 0)


def test_rotor_reduced_step_size_is_monotone():
    w = W.config("rotor41", Nt=800, N=16)
    _, J, _, _ = O.ism_solve(w, w.u0, 4, w.rho)
    assert np.all(np.diff(J) > 0)


# --------------------------------------------------------------------- large-d propagation route
def test_large_d_route_matches_eigh(monkeypatch):
    """For d > 64 the oracle applies each step with scipy's expm_multiply on the sparse H(u_j); on a
    d = 64 problem both routes must agree, forward and adjoint."""
    w = W.spin_chain(6, 5, T=2.0, Nt=40, N=4, u_amp=1.0)
    p1 = O.forward_trajectory(w, w.u0)
    c1 = O.backward_trajectory(w, w.u0, p1[-1])
    monkeypatch.setattr(O, "DENSE_MAX", 32)
    p2 = O.forward_trajectory(w, w.u0)
    c2 = O.backward_trajectory(w, w.u0, p1[-1])
    assert np.abs(p1 - p2).max() < 1e-12 and np.abs(c1 - c2).max() < 1e-12


def test_ising1024_norm_and_reversibility():
    w = W.config("ising1024", Nt=60, N=4)
    p = O.forward_trajectory(w, w.u0)
    assert np.allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-12)
    back = O.backward_trajectory(w, w.u0, p[-1])
    assert np.abs(back[0] - w.psi_i).max() < 1e-12


# ------------------------------------------------- complex Hermitian H (Sec. 2: any Hermitian H0, H1)
SY = np.array([[0.0, -1j], [1j, 0.0]])


def _sigma_y_problem(Nt=25, N=5, seed=4):
    """H0 = 0, H1 = sy (complex), psi_i = |0>, psi_f = |1>: exp(-i th sy)|0> = cos th |0> + sin th |1>,
    so J = sin(tau sum u) and dJ/du_j = tau cos(tau sum u) exactly."""
    rng = np.random.default_rng(seed)
    w = W.rabi(0.0, 0.0, T=2.0, Nt=Nt, N=N)
    return w.with_(H0=np.zeros((2, 2), dtype=np.complex128), H1=SY.copy(), psi_f=np.array([0.0, 1.0 + 0j]),
                   u0=rng.uniform(-1, 1, Nt))


@pytest.mark.parametrize("delta,u", [(1.3, 0.7), (0.0, 2.0)])
def test_sigma_y_rabi_closed_form(delta, u):
    """H = (delta/2) sz + (u/2) sy: the same populations as the sx drive, P_1 = (u/Omega)^2 sin^2(Omega t/2);
    at delta = 0, psi(t) = cos(ut/2)|0> + sin(ut/2)|1> (a real rotation, where sx gives -i sin)."""
    w = W.rabi(delta, u, T=5.0, Nt=50).with_(H1=0.5 * SY)
    psi = O.forward_trajectory(w, w.u0)
    t = np.arange(w.Nt + 1) * w.tau
    assert np.allclose(np.abs(psi[:, 1]) ** 2, _rabi_populations(delta, u, t), atol=1e-13)
    if delta == 0.0:
        assert np.allclose(psi[:, 0], np.cos(u * t / 2), atol=1e-13)
        assert np.allclose(psi[:, 1], np.sin(u * t / 2), atol=1e-13)


def test_sigma_y_closed_form_objective_and_gradient():
    w = _sigma_y_problem()
    th = w.tau * np.sum(w.u0)
    J, F = O.objective(w, w.u0)
    assert np.isclose(J, np.sin(th), atol=1e-14)
    g_ref = np.full(w.Nt, w.tau * np.cos(th))
    assert np.allclose(O.global_gradient(w, w.u0), g_ref, atol=1e-14)
    assert np.allclose(O.exact_gradient(w, w.u0), g_ref, atol=1e-14)
    phi = O.intermediate_states(w, w.u0)
    g, _ = O.subinterval_all(w, phi, w.u0)
    beta = np.repeat(O.interval_weights(w.T, w.Nt, w.N)[4], np.diff(O.partition(w.Nt, w.N)))
    assert np.allclose(beta * g, g_ref, atol=1e-14)


def test_hermitian_step_unitary_matches_pade_expm():
    w = W.random_hermitian(6, 71, T=1.0, Nt=6, N=1, u_amp=3.0)
    U = O.step_unitaries(w, w.u0, 0, w.Nt)
    for k in range(w.Nt):
        assert np.allclose(U[k], expm(-1j * w.tau * (w.H0 + w.u0[k] * w.H1)), atol=1e-12)


def test_gauge_invariance_of_algorithm1():
    """The basis change D = diag(exp(i theta)) turns a real symmetric problem into a complex Hermitian
    one (H -> D H D^H, psi -> D psi) with the same objective, gradients, sub-problem values and
    iterates, and intermediate states rotated by D."""
    w = W.random_dense(5, 72, T=2.0, Nt=36, N=4).with_(alpha=np.linspace(0.01, 0.05, 36))
    theta = np.random.default_rng(73).uniform(0, 2 * np.pi, w.d)
    wc = W.gauge(w, theta)
    assert np.abs(wc.H1.imag).max() > 0.1                 # genuinely complex
    J, F = O.objective(w, w.u0)
    Jc, Fc = O.objective(wc, w.u0)
    assert abs(J - Jc) <= 1e-13 and abs(F - Fc) <= 1e-13
    assert np.allclose(O.global_gradient(wc, w.u0), O.global_gradient(w, w.u0), atol=1e-14)
    assert np.allclose(O.exact_gradient(wc, w.u0), O.exact_gradient(w, w.u0), atol=1e-14)
    phi, phic = O.intermediate_states(w, w.u0), O.intermediate_states(wc, w.u0)
    assert np.allclose(phic, np.exp(1j * theta)[None, :] * phi, atol=1e-13)
    g, Jn = O.subinterval_all(w, phi, w.u0)
    gc, Jnc = O.subinterval_all(wc, phic, w.u0)
    assert np.allclose(gc, g, atol=1e-14) and np.allclose(Jnc, Jn, atol=1e-13)
    u, Jh, _, E = O.ism_solve(w, w.u0, 2, 0.5)
    uc, Jhc, _, Ec = O.ism_solve(wc, w.u0, 2, 0.5)
    assert np.allclose(uc, u, atol=1e-12) and np.allclose(Jhc, Jh, atol=1e-13) and np.allclose(Ec, E, atol=1e-12)


@pytest.mark.parametrize("objective", ["overlap", "observable"])
def test_hermitian_exact_gradient_matches_central_differences(objective):
    w = W.random_hermitian(4, 74, T=2.0, Nt=20, N=2, objective=objective)
    w = w.with_(alpha=np.linspace(0.01, 0.05, w.Nt))
    g = O.exact_gradient(w, w.u0)
    h = 1e-4
    fd = np.empty(w.Nt)

    def J_at(j, s):
        v = w.u0.copy()
        v[j] += s
        return O.objective(w, v)[0]

    for j in range(w.Nt):
        fd[j] = (8 * (J_at(j, h) - J_at(j, -h)) - (J_at(j, 2 * h) - J_at(j, -2 * h))) / (12 * h)
    assert np.linalg.norm(g - fd) <= 1e-9 * np.linalg.norm(fd)


@pytest.mark.parametrize("objective,N", [("overlap", 5), ("observable", 3)])
def test_hermitian_theorem2_and_theorem1(objective, N):
    """Theorem 2 (beta_n g_n at phi^u = the global gradient) and, for the overlap, Theorem 1's value
    identity, with complex Hermitian H."""
    w = W.random_hermitian(5, 75, T=2.5, Nt=41, N=N, objective=objective)
    w = w.with_(alpha=np.linspace(0.01, 0.1, w.Nt))
    phi = O.intermediate_states(w, w.u0)
    g, _ = O.subinterval_all(w, phi, w.u0)
    beta = np.repeat(O.interval_weights(w.T, w.Nt, w.N)[4], np.diff(O.partition(w.Nt, w.N)))
    G = O.global_gradient(w, w.u0)
    assert np.allclose(beta * g, G, atol=1e-13 * max(1.0, np.abs(G).max()))
    if objective == "overlap":
        J, _ = O.objective(w, w.u0)
        assert np.isclose(O.j_parallel(w, phi, w.u0), J - 1.0, atol=1e-12)
