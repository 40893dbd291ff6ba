"""FP64 CPU oracle for the Intermediate State Method with the paper's Crank-Nicolson propagator.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this module.  It shares no code with the CUDA path.

Scheme (Sec. 3): each step solves (I + i tau H_j / 2) psi_{j+1} = (I - i tau H_j / 2) psi_j with
H_j = H0 + u_j H1, i.e. psi_{j+1} = U_j psi_j, U_j = A_j^{-1} B_j, A_j = I + i tau H_j/2,
B_j = I - i tau H_j/2 (a Cayley transform: unitary, second order in tau).  numpy.linalg.solve is the
linear-solve primitive (d <= 64).

Adjoint and gradient (the exact derivative of the discrete J): with lambda_Nt = chi(T) (psi_f, or
O psi(T) with weight w = 2), lambda_j = U_j^H lambda_{j+1} = A_j B_j^{-1} lambda_{j+1}.  Writing
xi_j = B_j^{-1} lambda_{j+1} (so lambda_j = A_j xi_j), dU_j/du psi_j = -(i tau/2) A_j^{-1} H1
(psi_j + psi_{j+1}) gives
    dJ/du_j = w (tau/2) Im<xi_j|H1|psi_j + psi_{j+1}> - tau alpha_j u_j,
the paper's pairing of psi_{j+1} + psi_j in its discrete gradient (Sec. 3) with the adjoint it
implies.  The ISM pieces (partition, intermediate states of Eq. (cible), sub-problems of Sec. 2,
Algorithm 1) are those of ism_oracle with this propagator and this gradient.
"""
from __future__ import annotations

import numpy as np

from .ism_oracle import _alpha, interval_weights, partition, penalty, terminal_adjoint, weight

__all__ = ["step_matrices", "propagate", "propagate_adjoint", "forward_trajectory", "backward_trajectory",
           "objective", "global_gradient", "intermediate_states", "subinterval", "subinterval_all",
           "ism_iteration", "ism_solve", "gradient_method"]


def step_matrices(w, u_j):
    """(A_j, B_j) = (I + i tau H/2, I - i tau H/2) for H = H0 + u_j H1."""
    tau = w.T / w.Nt
    H = w.H0 + float(u_j) * w.H1
    Id = np.eye(w.d)
    return Id + 0.5j * tau * H, Id - 0.5j * tau * H


def propagate(w, u, psi, j0: int, j1: int) -> np.ndarray:
    """psi_{j+1} = A_j^{-1} B_j psi_j for j = j0..j1-1; returns (j1-j0+1, d) states."""
    out = np.empty((j1 - j0 + 1, w.d), dtype=np.complex128)
    out[0] = psi
    for k in range(j1 - j0):
        A, B = step_matrices(w, u[j0 + k])
        out[k + 1] = np.linalg.solve(A, B @ out[k])
    return out


def propagate_adjoint(w, u, lam_end, j0: int, j1: int):
    """lambda_j = A_j B_j^{-1} lambda_{j+1} for j = j1-1..j0 from lambda_{j1} = lam_end.  Returns
    (lambda (j1-j0+1, d), xi (j1-j0, d)) with xi_j = B_j^{-1} lambda_{j+1}."""
    lam = np.empty((j1 - j0 + 1, w.d), dtype=np.complex128)
    xi = np.empty((j1 - j0, w.d), dtype=np.complex128)
    lam[-1] = lam_end
    for k in reversed(range(j1 - j0)):
        A, B = step_matrices(w, u[j0 + k])
        xi[k] = np.linalg.solve(B, lam[k + 1])
        lam[k] = A @ xi[k]
    return lam, xi


def forward_trajectory(w, u) -> np.ndarray:
    return propagate(w, u, w.psi_i, 0, w.Nt)


def backward_trajectory(w, u, chi_T):
    """(chi_j (Nt+1, d), xi_j (Nt, d)) with chi_Nt = chi(T)."""
    return propagate_adjoint(w, u, chi_T, 0, w.Nt)


def objective(w, u, psi=None):
    """(J, F) as in ism_oracle.objective, with the Crank-Nicolson trajectory."""
    if psi is None:
        psi = forward_trajectory(w, u)
    pT = psi[-1]
    if w.objective == "overlap":
        ov = np.vdot(pT, w.psi_f)
        return float(ov.real) - penalty(w, u), float(abs(ov) ** 2)
    val = float(np.vdot(pT, w.O @ pT).real)
    return val - penalty(w, u), val


def _grad_terms(w, psi, xi) -> np.ndarray:
    """Im<xi_j|H1|psi_j + psi_{j+1}>, j = 0..len(xi)-1."""
    s = psi[:-1] + psi[1:]
    return np.imag(np.einsum("jk,jk->j", xi.conj(), s @ w.H1.T))


def global_gradient(w, u) -> np.ndarray:
    """dJ/du_j = w (tau/2) Im<xi_j|H1|psi_j + psi_{j+1}> - tau alpha_j u_j (exact for the scheme)."""
    tau = w.T / w.Nt
    psi = forward_trajectory(w, u)
    _, xi = backward_trajectory(w, u, terminal_adjoint(w, psi[-1]))
    return weight(w) * 0.5 * tau * _grad_terms(w, psi, xi) - tau * _alpha(w) * np.asarray(u)


def intermediate_states(w, u) -> np.ndarray:
    """phi_n = a_n psi(t_n) + b_n chi(t_n) (Eq. (cible)) on the Crank-Nicolson trajectories."""
    j, t, a, b, _ = interval_weights(w.T, w.Nt, w.N)
    psi = forward_trajectory(w, u)
    chi, _ = backward_trajectory(w, u, terminal_adjoint(w, psi[-1]))
    return a[:, None] * psi[j] + b[:, None] * chi[j]


def subinterval(w, phi, u, n: int):
    """Sub-problem n (Sec. 2) with targets phi: psi_n from phi_n, J_n = w (-1/2 ||psi_n(t_{n+1}) -
    phi_{n+1}||^2) - (tau/2) sum (alpha_j / beta_n) u_j^2 and its exact gradient, the adjoint started
    from w phi_{n+1} (the -w psi_n(t_{n+1}) part of the cotangent contributes Im of a Hermitian form,
    i.e. nothing)."""
    j, t, a, b, beta = interval_weights(w.T, w.Nt, w.N)
    tau = w.T / w.Nt
    j0, j1 = int(j[n]), int(j[n + 1])
    p = propagate(w, u, phi[n], j0, j1)
    _, xi = propagate_adjoint(w, u, phi[n + 1], j0, j1)
    al = _alpha(w)[j0:j1] / beta[n]
    uu = np.asarray(u[j0:j1], dtype=np.float64)
    g = weight(w) * 0.5 * tau * _grad_terms(w, p, xi) - tau * al * uu
    Jn = weight(w) * (-0.5 * float(np.linalg.norm(p[-1] - phi[n + 1]) ** 2)) - 0.5 * tau * float(np.sum(al * uu ** 2))
    return g, Jn


def subinterval_all(w, phi, u):
    g = np.empty(w.Nt)
    Jn = np.empty(w.N)
    j = partition(w.Nt, w.N)
    for n in range(w.N):
        g[j[n]:j[n + 1]], Jn[n] = subinterval(w, phi, u, n)
    return g, Jn


def ism_iteration(w, u, rho: float, L: int = 1):
    """Algorithm 1 with the constant-step gradient sub-solver (as ism_oracle.ism_iteration)."""
    j, t, a, b, beta = interval_weights(w.T, w.Nt, w.N)
    tau = w.T / w.Nt
    phi = intermediate_states(w, u)
    u_next = np.array(u, dtype=np.float64, copy=True)
    err = 0.0
    for n in range(w.N):
        j0, j1 = int(j[n]), int(j[n + 1])
        local = np.array(u, dtype=np.float64, copy=True)
        for ell in range(L):
            g, _ = subinterval(w, phi, local, n)
            if ell == 0:
                err += float(np.sum(np.abs(g)))
            local[j0:j1] = local[j0:j1] + rho * beta[n] * g / tau
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
    """Plain sequential gradient ascent on J with the same step rule (the N = 1 case)."""
    tau = w.T / w.Nt
    u = np.array(u0, dtype=np.float64, copy=True)
    J_hist = []
    for _ in range(iters):
        J_hist.append(objective(w, u)[0])
        u = u + rho * global_gradient(w, u) / tau
    J_hist.append(objective(w, u)[0])
    return u, np.array(J_hist)
