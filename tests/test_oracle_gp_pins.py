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


# ------------------------------------------------------------------ double-well potential (Sec. 4)
def _dw_small(g=1.0, n=32, Nt=20, N=4, T=0.8, seed=4, dw=4.0):
    """Even initial state (harmonic ground state); the target is a random state, since the double
    well conserves parity and an odd target would have zero overlap for every control."""
    rng = np.random.default_rng(seed)
    psi_i, _ = W.gp_stationary_states(n, 20.0, -10.0, g, dt=2e-3, steps=3000)
    psi_f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    psi_f = psi_f / np.sqrt(np.sum(np.abs(psi_f) ** 2) * (20.0 / n))
    return W.GPWorkload(name="dw-small", n=n, L=20.0, x_min=-10.0, g=g, psi_i=psi_i, psi_f=psi_f, T=T, Nt=Nt,
                        N=N, u0=rng.uniform(0.2, 1.2, Nt), potential="double_well", dw=dw)


def test_double_well_potential_is_c1_and_its_derivative_matches_differences():
    """The two branches meet with equal value and slope at |x| = u d/4 (a dropped factor in either
    branch breaks this), and dV/du equals central differences of V in u away from that point."""
    w = _dw_small()
    for u in (0.3, 1.0, 1.7):
        xb = u * w.dw / 4.0
        for x0 in (xb, -xb):
            lo = G.potential(w, np.array([x0 * (1 - 1e-10)]), u)[0]
            hi = G.potential(w, np.array([x0 * (1 + 1e-10)]), u)[0]
            assert abs(lo - hi) < 1e-9
            dlo = G.potential_du(w, np.array([x0 * (1 - 1e-10)]), u)[0]
            dhi = G.potential_du(w, np.array([x0 * (1 + 1e-10)]), u)[0]
            assert abs(dlo - dhi) < 1e-8
    x = np.linspace(-9.7, 9.7, 97)
    for u in (-0.4, 0.3, 1.0, 1.7):
        h = 1e-5
        fd = (G.potential(w, x, u + h) - G.potential(w, x, u - h)) / (2 * h)
        far = np.abs(np.abs(x) - u * w.dw / 4.0) > 1e-3
        assert np.max(np.abs(fd - G.potential_du(w, x, u))[far]) < 1e-8


def test_double_well_at_zero_control_is_the_harmonic_trap():
    """V(x, 0) = x^2/2 = the harmonic trap at u = 0: identical trajectories."""
    w = _dw_small(Nt=40)
    h = w.with_(potential="harmonic", dw=0.0)
    zero = np.zeros(w.Nt)
    a = G.forward(w, zero, w.psi_i, 0, w.Nt)
    b = G.forward(h, zero, h.psi_i, 0, h.Nt)
    assert np.max(np.abs(a - b)) < 1e-14


def test_double_well_conserves_parity():
    """V(-x, u) = V(x, u): an even state stays even under any control (grid symmetric about 0)."""
    w = _dw_small(Nt=60)
    psi = G.forward(w, w.u0, w.psi_i, 0, w.Nt)[-1]
    mirror = psi[(-np.arange(w.n)) % w.n]
    assert np.max(np.abs(psi - mirror)) < 1e-12
    assert np.max(np.abs(w.psi_i - w.psi_i[(-np.arange(w.n)) % w.n])) < 1e-12


@pytest.mark.parametrize("g", [0.0, 1.0])
def test_double_well_gradient_matches_finite_differences(g):
    w = _dw_small(g=g)
    grad = G.global_gradient(w, w.u0)
    h = 1e-4
    fd = np.empty(w.Nt)
    for j in range(w.Nt):
        def J_at(s):
            v = w.u0.copy()
            v[j] += s
            return G.objective(w, v)[0]
        fd[j] = (8 * (J_at(h) - J_at(-h)) - (J_at(2 * h) - J_at(-2 * h))) / (12 * h)
    assert np.linalg.norm(grad - fd) <= 1e-8 * np.linalg.norm(fd)


def test_double_well_ism_iterates_do_not_depend_on_N():
    w = _dw_small(Nt=24, N=1)
    u1, J1, _, _ = G.ism_solve(w, w.u0, 3, 0.05)
    for N in (3, 8):
        uN, JN, _, _ = G.ism_solve(w.with_(N=N), w.u0, 3, 0.05)
        assert np.max(np.abs(uN - u1)) < 1e-12 and np.max(np.abs(JN - J1)) < 1e-12


def test_double_well_rho_increases_J():
    """The step size of the double-well problem (rho = 0.05) increases J monotonically over 5
    gradient iterations on a 128-point version of the benchmark set-up."""
    w = W.gp_double_well(n=128, Nt=1000, N=8, steps=20000)
    _, J = G.gradient_method(w, w.u0, 5, 0.05)
    assert np.all(np.diff(J) > 0)
