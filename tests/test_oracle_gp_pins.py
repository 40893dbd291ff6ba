"""Pins of the Gross-Pitaevskii oracle (Strang split-step, reverse-mode adjoint, nonlinear ISM)
against finite differences, conservation laws, a closed form and the ISM invariants.  CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import gp_oracle as G


def _small(g=1.0, n=32, Nt=20, N=4, T=0.8, seed=3, u_amp=0.5):
    """32-point grid on [-10, 10) with the same structure as the benchmark problem."""
    rng = np.random.default_rng(seed)
    psi_i, psi_f = W.gp_stationary_states(n, 20.0, -10.0, g, dt=2e-3, steps=3000)
    return W.GPWorkload(name="gp-small", n=n, L=20.0, x_min=-10.0, g=g, psi_i=psi_i, psi_f=psi_f,
                        T=T, Nt=Nt, N=N, u0=rng.uniform(-u_amp, u_amp, Nt))


@pytest.mark.parametrize("g", [0.0, 1.0, 5.0])
def test_norm_is_conserved(g):
    w = _small(g=g, Nt=60)
    psi = G.forward(w, w.u0, w.psi_i, 0, w.Nt)
    nrm = np.sum(np.abs(psi) ** 2, axis=1) * w.dx
    assert np.allclose(nrm, 1.0, atol=1e-13)


@pytest.mark.parametrize("g", [0.0, 1.0, 3.0])
def test_adjoint_gradient_matches_finite_differences(g):
    w = _small(g=g)
    grad = G.global_gradient(w, w.u0)
    h = 1e-4
    fd = np.empty(w.Nt)
    for j in range(w.Nt):
        def J_at(s):
            v = w.u0.copy()
            v[j] += s
            return G.objective(w, v)[0]
        fd[j] = (8 * (J_at(h) - J_at(-h)) - (J_at(2 * h) - J_at(-2 * h))) / (12 * h)
    assert np.linalg.norm(grad - fd) <= 1e-9 * np.linalg.norm(fd)


def test_harmonic_ground_state_is_stationary():
    """g = 0, u = 0: the discrete ground state of x^2/2 - d^2/2 only acquires the phase exp(-i E0 T),
    E0 = 1/2 (closed form for the harmonic oscillator), up to the O(tau^2) splitting error."""
    n, L = 128, 20.0
    g0, _ = W.gp_stationary_states(n, L, -10.0, 0.0, dt=1e-3, steps=20000)
    w = W.GPWorkload(name="ho", n=n, L=L, x_min=-10.0, g=0.0, psi_i=g0, psi_f=g0, T=2.0, Nt=400, N=1,
                     u0=np.zeros(400))
    psi = G.forward(w, w.u0, g0, 0, w.Nt)
    ov = np.sum(np.conj(g0) * psi[-1]) * w.dx
    assert abs(abs(ov) - 1.0) < 1e-6
    assert abs(np.angle(ov) - (-0.5 * w.T)) < 1e-4


def test_linear_limit_matches_unitary_adjoint():
    """For g = 0 the map is linear and unitary: the reverse-mode adjoint is U^H applied to psi_f."""
    w = _small(g=0.0, Nt=30)
    psi = G.forward(w, w.u0, w.psi_i, 0, w.Nt)
    lam, _ = G.adjoint_sweep(w, w.u0, psi, w.psi_f, 0, w.Nt)
    # <lambda_j|psi_j> is constant and equals <psi_f|psi(T)>
    ov = np.array([np.sum(np.conj(lam[j]) * psi[j]) * w.dx for j in range(w.Nt + 1)])
    assert np.allclose(ov, ov[-1], atol=1e-13)


def test_ism_subinterval_gradient_equals_global_gradient():
    w = _small(g=1.0, Nt=24, N=5)
    psi_t, chi_t = G.intermediate_pairs(w, w.u0)
    g, _ = G.subinterval_all(w, psi_t, chi_t, w.u0)
    assert np.allclose(g, G.global_gradient(w, w.u0), atol=1e-14)


def test_ism_iterates_do_not_depend_on_N():
    w = _small(g=1.0, Nt=24, N=1)
    res = [G.ism_solve(w.with_(N=N), w.u0, 3, 0.5)[0] for N in (1, 3, 8, 24)]
    for u in res[1:]:
        assert np.allclose(u, res[0], atol=1e-13)
    u_gm, _ = G.gradient_method(w, w.u0, 3, 0.5)
    assert np.allclose(res[0], u_gm, atol=1e-13)


def test_gp_rho_increases_J():
    w = _small(g=1.0, Nt=40, N=4, T=2.0)
    _, J, _, _ = G.ism_solve(w, w.u0, 4, 0.1)
    assert np.all(np.diff(J) > 0)
