"""FP64 CPU oracle for the Gross-Pitaevskii (condensate) variant of the Intermediate State Method.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this module.  It shares no code with the CUDA path.

Model (Sec. 4, condensates, with the readings listed in the design notes): on a periodic grid
x_k = x_min + k dx, k = 0..n-1, the state obeys i d/dt psi = (-1/2 d^2/dx^2 + V(x, u) + g |psi|^2) psi
with <a|b> = sum_k conj(a_k) b_k dx and J = Re<psi(T)|psi_f> (alpha = 0).  Two potentials:
  harmonic trap with a control-shifted centre, V(x, u) = (x - u)^2 / 2;
  the double well of Sec. 4 (radio-frequency splitting, control lambda = u, separation d > 0):
      V(x, u) = (|x| - u d/2)^2 / 2          for |x| > u d/4,
      V(x, u) = ((u d)^2 / 8 - x^2) / 2      otherwise,
  whose derivative is dV/du = -(d/2)(|x| - u d/2), resp. u d^2 / 8.

Time step (Strang splitting, Eq. (OS), written for -1/2 d^2 so the half kinetic factor in Fourier
space is exp(-i tau k^2 / 4)):  a = K psi_j with K = F^-1 diag(exp(-i tau k^2/4)) F,
b = exp(-i tau theta) a with theta = V(x, u_j) + g |a|^2 (|b| = |a|, so evaluating the density on the
half-kinetic state is exact for this sub-step), psi_{j+1} = K b.  numpy.fft is the FFT primitive.

Adjoint (reverse mode of the discrete map, Wirtinger calculus): with dJ = Re<lambda_j|d psi_j>,
lambda_Nt = psi_f and, for one step at w = a_j,
    mu = exp(+i tau theta) K^H lambda_{j+1},
    lambda_j = K^H [ mu + 2 tau g Im(conj(mu) w) w ],
    dJ/du_j = tau sum_k dV/du(x_k) Im(conj(mu_k) w_k) dx.
Nonlinear ISM (Sec. 4): initial states psi(t_n) on the forward trajectory, targets chi(t_n) on the
adjoint trajectory, J_n = Re<psi_n(t_{n+1})|chi(t_{n+1})>; chi(t_n) is read as the discrete adjoint
lambda_{j_n} of the full problem.
"""
from __future__ import annotations

import numpy as np

from .ism_oracle import partition

__all__ = ["potential", "potential_du", "strang_step", "forward", "objective", "adjoint_sweep", "global_gradient", "intermediate_pairs",
           "subinterval", "subinterval_all", "ism_iteration", "ism_solve", "gradient_method"]


def _half_kinetic(w):
    return np.exp(-0.25j * w.tau * w.k ** 2)


def _K(w, v):
    return np.fft.ifft(_half_kinetic(w) * np.fft.fft(v))


def _KH(w, v):
    return np.fft.ifft(np.conj(_half_kinetic(w)) * np.fft.fft(v))


def potential(w, x, u_j):
    """V(x, u_j) for the workload's potential (module docstring)."""
    x = np.asarray(x, dtype=np.float64)
    if getattr(w, "potential", "harmonic") == "harmonic":
        return 0.5 * (x - u_j) ** 2
    d = w.dw
    ax = np.abs(x)
    return np.where(ax > u_j * d / 4.0, 0.5 * (ax - u_j * d / 2.0) ** 2, 0.5 * ((u_j * d) ** 2 / 8.0 - x ** 2))


def potential_du(w, x, u_j):
    """dV/du at (x, u_j)."""
    x = np.asarray(x, dtype=np.float64)
    if getattr(w, "potential", "harmonic") == "harmonic":
        return -(x - u_j)
    d = w.dw
    ax = np.abs(x)
    return np.where(ax > u_j * d / 4.0, -(d / 2.0) * (ax - u_j * d / 2.0), u_j * d * d / 8.0 + 0.0 * x)


def _theta(w, a, u_j):
    return potential(w, w.x, u_j) + w.g * np.abs(a) ** 2


def strang_step(w, psi, u_j):
    """psi_{j+1} = K exp(-i tau theta) K psi_j (Eq. (OS))."""
    a = _K(w, psi)
    return _K(w, np.exp(-1j * w.tau * _theta(w, a, u_j)) * a)


def forward(w, u, psi0, j0: int, j1: int) -> np.ndarray:
    """States psi_j, j = j0..j1, from psi_{j0} = psi0."""
    out = np.empty((j1 - j0 + 1, w.n), dtype=np.complex128)
    out[0] = psi0
    for s in range(j1 - j0):
        out[s + 1] = strang_step(w, out[s], u[j0 + s])
    return out


def _inner(w, a, b):
    return np.sum(np.conj(a) * b) * w.dx


def objective(w, u, psi=None):
    """(J, F) = (Re<psi(T)|psi_f>, |<psi(T)|psi_f>|^2)."""
    if psi is None:
        psi = forward(w, u, w.psi_i, 0, w.Nt)
    ov = _inner(w, psi[-1], w.psi_f)
    return float(ov.real), float(abs(ov) ** 2)


def _adjoint_step(w, lam_next, psi_j, u_j):
    """(lambda_j, dJ/du_j) from lambda_{j+1} through the step taken at psi_j."""
    a = _K(w, psi_j)
    th = _theta(w, a, u_j)
    mu = np.exp(1j * w.tau * th) * _KH(w, lam_next)
    lam = _KH(w, mu + 2.0 * w.tau * w.g * np.imag(np.conj(mu) * a) * a)
    g = w.tau * np.sum(potential_du(w, w.x, u_j) * np.imag(np.conj(mu) * a)) * w.dx
    return lam, float(g)


def adjoint_sweep(w, u, psi, lam_end, j0: int, j1: int):
    """lambda_j, j = j0..j1, from lambda_{j1} = lam_end backward along the stored states psi
    (psi[s] = psi_{j0+s}); returns (lambdas, gradient (j1-j0,))."""
    lam = np.empty((j1 - j0 + 1, w.n), dtype=np.complex128)
    lam[-1] = lam_end
    g = np.empty(j1 - j0)
    for s in reversed(range(j1 - j0)):
        lam[s], g[s] = _adjoint_step(w, lam[s + 1], psi[s], u[j0 + s])
    return lam, g


def global_gradient(w, u):
    """Exact gradient of the discrete J (reverse mode over [0, T])."""
    psi = forward(w, u, w.psi_i, 0, w.Nt)
    _, g = adjoint_sweep(w, u, psi, np.asarray(w.psi_f, dtype=np.complex128), 0, w.Nt)
    return g


def intermediate_pairs(w, u):
    """(psi(t_n), chi(t_n)), n = 0..N: forward states and adjoint states at the partition."""
    j = partition(w.Nt, w.N)
    psi = forward(w, u, w.psi_i, 0, w.Nt)
    lam, _ = adjoint_sweep(w, u, psi, np.asarray(w.psi_f, dtype=np.complex128), 0, w.Nt)
    return psi[j], lam[j]


def subinterval(w, psi_n, chi_n1, u, n: int):
    """Sub-problem n: psi_n from psi(t_n), J_n = Re<psi_n(t_{n+1})|chi(t_{n+1})> and its gradient by
    reverse mode from chi(t_{n+1})."""
    j = partition(w.Nt, w.N)
    j0, j1 = int(j[n]), int(j[n + 1])
    p = forward(w, u, psi_n, j0, j1)
    _, g = adjoint_sweep(w, u, p, chi_n1, j0, j1)
    Jn = float(_inner(w, p[-1], chi_n1).real)
    return g, Jn


def subinterval_all(w, psi_t, chi_t, u):
    g = np.empty(w.Nt)
    Jn = np.empty(w.N)
    j = partition(w.Nt, w.N)
    for n in range(w.N):
        g[j[n]:j[n + 1]], Jn[n] = subinterval(w, psi_t[n], chi_t[n + 1], u, n)
    return g, Jn


def ism_iteration(w, u, rho: float, L: int = 1):
    """Algorithm 1 with the nonlinear intermediate states: (a)-(b) psi(t_n), chi(t_n); (c) L ascent
    steps u <- u + rho g / tau on each sub-problem with the targets fixed; (e) Err = sum |g|."""
    j = partition(w.Nt, w.N)
    psi_t, chi_t = intermediate_pairs(w, u)
    u_next = np.array(u, dtype=np.float64, copy=True)
    err = 0.0
    for n in range(w.N):
        j0, j1 = int(j[n]), int(j[n + 1])
        local = np.array(u, dtype=np.float64, copy=True)
        for ell in range(L):
            g, _ = subinterval(w, psi_t[n], chi_t[n + 1], local, n)
            if ell == 0:
                err += float(np.sum(np.abs(g)))
            local[j0:j1] = local[j0:j1] + rho * g / w.tau
        u_next[j0:j1] = local[j0:j1]
    return u_next, err


def ism_solve(w, u0, iters: int, rho: float, L: int = 1):
    """(u, J_hist (iters+1), F_hist (iters+1), err_hist (iters))."""
    u = np.array(u0, dtype=np.float64, copy=True)
    J_hist, F_hist, err_hist = [], [], []
    for _ in range(iters):
        J, F = objective(w, u)
        J_hist.append(J)
        F_hist.append(F)
        u, err = ism_iteration(w, u, rho, L)
        err_hist.append(err)
    J, F = objective(w, u)
    J_hist.append(J)
    F_hist.append(F)
    return u, np.array(J_hist), np.array(F_hist), np.array(err_hist)


def gradient_method(w, u0, iters: int, rho: float):
    """Plain sequential gradient ascent on J (no decomposition)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    J_hist = []
    for _ in range(iters):
        J_hist.append(objective(w, u)[0])
        u = u + rho * global_gradient(w, u) / w.tau
    J_hist.append(objective(w, u)[0])
    return u, np.array(J_hist)
