"""Pins of the seeded input generators (workloads/) against their textbook definitions.

The generators are shared by the oracle and the GPU path, so a mistake in one of them (a wrong
matrix element, a transposed bit order, an unconverged initial state) would pass every parity test.
Each test here rebuilds the model quantity from a definition that the generator does not use:
quadrature of Legendre polynomials for the rotor (Sec. 4, molecular orientation), Kronecker products
of Pauli matrices for the spin models (Sec. 4, spin systems), and the stationary Gross-Pitaevskii
equation for the condensate's initial and target states (Sec. 4, condensates).
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as L

import workloads as W


def _normalised_legendre(j: int):
    """Coefficients (Legendre basis) of sqrt((2j+1)/2) P_j, orthonormal on [-1, 1]."""
    c = np.zeros(j + 1)
    c[j] = np.sqrt((2.0 * j + 1.0) / 2.0)
    return c


@pytest.mark.parametrize("jmax", [4, 40])
def test_rotor_cos_theta_is_the_legendre_matrix_element(jmax):
    """<j|cos theta|k> for m = 0 is the integral of P~_j(x) x P~_k(x) over x = cos theta in [-1, 1];
    Gauss-Legendre quadrature with 64 nodes is exact for the degree <= 2 jmax + 1 integrands."""
    x, wq = L.leggauss(64)
    P = np.array([L.legval(x, _normalised_legendre(j)) for j in range(jmax + 1)])   # (d, nodes)
    C_quad = (P * (x * wq)[None, :]) @ P.T
    C = W.rotor_cos_theta(jmax)
    assert np.max(np.abs(C - C_quad)) <= 1e-13
    # the same quadrature gives the identity for <j|k>: the basis used is orthonormal
    assert np.max(np.abs((P * wq[None, :]) @ P.T - np.eye(jmax + 1))) <= 1e-13


def test_rotor_h0_is_the_angular_momentum_eigenvalue():
    """H0 = L^2 / (hbar^2) in units of B: the Legendre operator -(d/dx)(1 - x^2)(d/dx) applied to
    P_j gives j(j + 1) P_j; the rotor workload's H0 must be that diagonal."""
    w = W.config("rotor41", Nt=100, N=4)
    d = w.d
    for j in range(d):
        p = L.leg2poly(_normalised_legendre(j))                    # power-series coefficients
        dp = np.polynomial.polynomial.polyder(p)
        flux = np.polynomial.polynomial.polymul([1.0, 0.0, -1.0], dp)   # (1 - x^2) p'
        lp = -np.polynomial.polynomial.polyder(flux)
        lam = lp[j] / p[j]                                         # leading coefficients
        assert np.allclose(np.polynomial.polynomial.polysub(lp, lam * p), 0.0, atol=1e-9 * abs(p[j]))
        assert abs(w.H0[j, j] - lam) <= 1e-9 * max(1.0, lam)
    assert np.count_nonzero(w.H0 - np.diag(np.diag(w.H0))) == 0
    assert np.array_equal(w.H1, -W.rotor_cos_theta(d - 1))        # H1 = -cos theta


_I2 = np.eye(2)
_X = np.array([[0.0, 1.0], [1.0, 0.0]])
_Z = np.diag([1.0, -1.0])


def _site_op(q: int, i: int, op: np.ndarray) -> np.ndarray:
    """op on spin i of q, identity elsewhere; spin i is bit i of the basis index (spin 0 the last
    Kronecker factor)."""
    out = np.eye(1)
    for k in reversed(range(q)):
        out = np.kron(out, op if k == i else _I2)
    return out


@pytest.mark.parametrize("name,q", [("spin16", 4), ("ising_small", 6)])
def test_spin_hamiltonians_are_the_pauli_sums(name, q):
    """H0 = sum over the coupled pairs J_ij Z_i Z_j, H1 = sum_i X_i, |0..0> and |1..1> the all-up and
    all-down product states, built as Kronecker products of 2x2 Pauli matrices."""
    if name == "spin16":
        w = W.config("spin16", Nt=100, N=4)
    else:
        w = W.spin_chain(q, 77, T=1.0, Nt=10, N=2)
    pairs, J = w.meta["pairs"], w.meta["J"]
    if name == "spin16":
        assert pairs == [(i, j) for i in range(q) for j in range(i + 1, q)]
    else:
        assert pairs == [(i, i + 1) for i in range(q - 1)]
    H0 = sum(Jij * _site_op(q, i, _Z) @ _site_op(q, j, _Z) for (i, j), Jij in zip(pairs, J))
    H1 = sum(_site_op(q, i, _X) for i in range(q))
    assert np.max(np.abs(w.H0 - H0)) <= 1e-14
    assert np.max(np.abs(w.H1 - H1)) == 0.0
    up = np.array([1.0, 0.0])
    down = np.array([0.0, 1.0])
    all_up, all_down = np.ones(1), np.ones(1)
    for _ in range(q):
        all_up, all_down = np.kron(all_up, up), np.kron(all_down, down)
    assert np.array_equal(w.psi_i, all_up.astype(np.complex128))
    assert np.array_equal(w.psi_f, all_down.astype(np.complex128))
    assert np.all((J >= 0.5) & (J <= 1.5))


def _gp_residual(psi, x, dx, g, V):
    """Residual of the stationary GP equation (-1/2 d^2 + V + g|psi|^2) psi = mu psi, with the second
    derivative taken spectrally on the periodic grid; returns (mu, relative residual)."""
    n = x.size
    kk = 2.0 * np.pi * np.fft.fftfreq(n, d=dx)
    Hpsi = np.fft.ifft(0.5 * kk ** 2 * np.fft.fft(psi)) + (V + g * np.abs(psi) ** 2) * psi
    mu = float(np.real(np.sum(np.conj(psi) * Hpsi) * dx))
    res = np.sqrt(np.sum(np.abs(Hpsi - mu * psi) ** 2) * dx) / np.sqrt(np.sum(np.abs(psi) ** 2) * dx)
    return mu, float(res)


def test_gp_states_are_stationary_states_of_the_gp_equation():
    """The 512-point condensate's initial state (ground state) and target (lowest odd state) of
    -1/2 d^2 + x^2/2 + g|psi|^2 at g = 1 on [-10, 10): unit L2 norm, the parity of each state, and a
    stationary-equation residual that is first order in the imaginary-time step (the nonlinear
    factor of a step uses the density before that step's renormalisation, an O(dt) shift of the
    fixed point): it halves with dt, so the generator converges to the stationary states.  Also
    mu_0 < mu_1, both above the harmonic (g = 0) values 1/2 and 3/2 (g > 0 raises mu)."""
    n, Lbox, x_min, g = 512, 20.0, -10.0, 1.0
    dx = Lbox / n
    x = x_min + np.arange(n) * dx
    V = 0.5 * x ** 2
    mirror = (-np.arange(n)) % n
    res = {}
    for dt, steps in ((1e-3, 40000), (5e-4, 80000)):
        g0, e1 = W.gp_stationary_states(n, Lbox, x_min, g, dt=dt, steps=steps)
        for psi, parity in ((g0, 1.0), (e1, -1.0)):
            assert abs(np.sum(np.abs(psi) ** 2) * dx - 1.0) <= 1e-12
            assert np.max(np.abs(psi[mirror] - parity * psi)) <= 1e-10
        (mu0, r0), (mu1, r1) = _gp_residual(g0, x, dx, g, V), _gp_residual(e1, x, dx, g, V)
        assert 0.5 < mu0 < mu1 and 1.5 < mu1
        res[dt] = (r0, r1)
    assert res[1e-3][0] <= 1e-4 and res[1e-3][1] <= 2e-4, res          # the states the workload uses
    for k in range(2):
        assert 1.8 <= res[1e-3][k] / res[5e-4][k] <= 2.2, res            # first order in dt


def test_gp_generator_at_zero_coupling_gives_the_harmonic_eigenfunctions():
    """At g = 0 the generator's states are the harmonic-oscillator eigenfunctions (closed forms
    pi^(-1/4) exp(-x^2/2) and sqrt(2) pi^(-1/4) x exp(-x^2/2)) up to a global phase."""
    n, Lbox, x_min = 512, 20.0, -10.0
    dx = Lbox / n
    x = x_min + np.arange(n) * dx
    h0, h1 = W.gp_stationary_states(n, Lbox, x_min, 0.0, steps=20000)
    c0 = np.pi ** -0.25 * np.exp(-0.5 * x ** 2)
    c1 = np.sqrt(2.0) * np.pi ** -0.25 * x * np.exp(-0.5 * x ** 2)
    for psi, c in ((h0, c0), (h1, c1)):
        phase = np.sum(np.conj(c) * psi) * dx
        phase /= abs(phase)
        assert np.max(np.abs(psi - phase * c)) <= 1e-5
