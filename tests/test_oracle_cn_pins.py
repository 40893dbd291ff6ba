"""Pins of the Crank-Nicolson oracle (Sec. 3 scheme) against what the mathematics fixes: the Cayley
transform is exactly unitary and second order; for H = u sigma_x it is exp(-i 2 arctan(tau u/2)
sigma_x), which gives J and its exact gradient in closed form; the adjoint gradient equals central
differences of the discrete J; and the ISM identities (Theorems 1 and 2, N-independence) hold."""
import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle import cn_oracle as C
from oracle import ism_oracle as O


def _sigma_x_problem(Nt=25, N=5, seed=3):
    rng = np.random.default_rng(seed)
    w = W.rabi(0.0, 0.0, T=2.0, Nt=Nt, N=N)
    return w.with_(H1=np.array([[0.0, 1.0], [1.0, 0.0]]), psi_f=np.array([0.0, -1j]), u0=rng.uniform(-3, 3, Nt))


def test_cayley_step_is_unitary():
    w = W.random_dense(6, 11, T=40.0, Nt=20, N=2, u_amp=3.0)   # tau ||H|| ~ 4: far from small
    p = C.forward_trajectory(w, w.u0)
    assert np.allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-13)
    lam, _ = C.backward_trajectory(w, w.u0, w.psi_f)
    assert np.allclose(np.linalg.norm(lam, axis=1), 1.0, atol=1e-13)


def test_second_order_in_tau():
    """Constant control: the error against exp(-i T H) psi falls by ~4 when tau halves."""
    w = W.random_dense(5, 12, T=1.0, Nt=40, N=1)
    H = w.H0 + 0.3 * w.H1
    exact = expm(-1j * w.T * H) @ w.psi_i
    errs = []
    for Nt in (40, 80, 160):
        ww = w.with_(Nt=Nt, u0=np.full(Nt, 0.3))
        errs.append(np.linalg.norm(C.forward_trajectory(ww, ww.u0)[-1] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.9 < r2 < 4.1, (r1, r2)


def test_sigma_x_closed_form():
    """U_j = exp(-i theta_j sigma_x), theta_j = 2 arctan(tau u_j / 2): J = sin(S), S = sum theta_j,
    and dJ/du_j = tau cos(S) / (1 + (tau u_j / 2)^2), on the full interval and through the
    sub-problems (beta_n g_n, Theorem 2)."""
    w = _sigma_x_problem()
    tau = w.T / w.Nt
    S = np.sum(2.0 * np.arctan(0.5 * tau * w.u0))
    J, F = C.objective(w, w.u0)
    assert np.isclose(J, np.sin(S), atol=1e-14)
    assert np.isclose(F, np.sin(S) ** 2, atol=1e-14)
    g_ref = tau * np.cos(S) / (1.0 + (0.5 * tau * w.u0) ** 2)
    assert np.allclose(C.global_gradient(w, w.u0), g_ref, atol=1e-14)
    phi = C.intermediate_states(w, w.u0)
    g, _ = C.subinterval_all(w, phi, w.u0)
    beta = np.repeat(O.interval_weights(w.T, w.Nt, w.N)[4], np.diff(O.partition(w.Nt, w.N)))
    assert np.allclose(beta * g, g_ref, atol=1e-14)


@pytest.mark.parametrize("objective", ["overlap", "observable"])
def test_gradient_matches_central_differences(objective):
    w = W.random_dense(4, 5, T=2.0, Nt=30, N=3, objective=objective)
    w = w.with_(alpha=np.linspace(0.1, 0.3, w.Nt))
    g = C.global_gradient(w, w.u0)
    h = 1e-3
    fd = np.empty(w.Nt)
    for j in range(w.Nt):   # fourth-order central difference
        vals = []
        for k in (-2, -1, 1, 2):
            u = w.u0.copy()
            u[j] += k * h
            vals.append(C.objective(w, u)[0])
        fd[j] = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
    assert np.max(np.abs(g - fd)) <= 1e-9 * np.max(np.abs(fd))


def test_theorem1_value_identity():
    w = W.random_dense(5, 13, T=2.0, Nt=40, N=4)
    phi = C.intermediate_states(w, w.u0)
    _, Jn = C.subinterval_all(w, phi, w.u0)
    beta = O.interval_weights(w.T, w.Nt, w.N)[4]
    J, _ = C.objective(w, w.u0)
    assert abs(np.sum(beta * Jn) + 1.0 - J) <= 1e-12


@pytest.mark.parametrize("objective", ["overlap", "observable"])
def test_theorem2_gradient_decomposition(objective):
    w = W.random_dense(5, 14, T=2.0, Nt=41, N=6, objective=objective)
    phi = C.intermediate_states(w, w.u0)
    g, _ = C.subinterval_all(w, phi, w.u0)
    j, _, _, _, beta = O.interval_weights(w.T, w.Nt, w.N)
    bj = np.repeat(beta, np.diff(j))
    assert np.max(np.abs(bj * g - C.global_gradient(w, w.u0))) <= 1e-12


def test_n_independence_and_gradient_method():
    w = W.config("rotor41", Nt=300, N=1).with_(H0=W.config("rotor41").H0[:9, :9],
                                               H1=W.config("rotor41").H1[:9, :9], O=W.config("rotor41").O[:9, :9],
                                               psi_i=np.eye(9)[0])
    u_ref, J_ref = C.gradient_method(w, w.u0, 3, 0.5)
    for N in (1, 5, 30):
        u, J, _, _ = C.ism_solve(w.with_(N=N), w.u0, 3, 0.5)
        assert np.max(np.abs(u - u_ref)) <= 1e-12
        assert np.max(np.abs(J - J_ref)) <= 1e-12
