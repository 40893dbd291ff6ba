"""FP64 CPU oracle for the Intermediate State Method with several controls (the five-spin example of
Sec. 4): H(t) = H0 + sum_c u_c(t) H_c.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this module.  It shares no code with the CUDA path.

Two statements of the same method:

* State form (``MCWorkload``: diagonal H0, H_c = sum_b ax[c,b] X_b + ay[c,b] Y_b on d = 2^q basis
  states).  The operators are built from their definition as Kronecker products of the 2 x 2 Pauli
  matrices (bit b of the basis index <-> tensor factor b counted from the right); each step applies
  the exact exponential exp(-i tau H(u_j)) (``numpy.linalg.eigh`` for d <= 64,
  ``scipy.sparse.linalg.expm_multiply`` above).  Gradient, intermediate states, sub-problems and
  the ascent step are those of the single-control oracle with a vector of controls per step: the
  trapezoid reading of Eq. (gradJ),
      g_{j,c} = (tau/2)[Im<chi_{j+1}|H_c|psi_{j+1}> + Im<chi_j|H_c|psi_j>],
  phi_n = a_n psi(t_n) + b_n chi(t_n) (Eq. (cible)), u_{j,c} += rho beta_n g_{j,c} / tau.  The overlap
  objective J = Re<psi(T)|psi_f>, alpha = 0 (as in the paper's spin example).

* Density-matrix form (``dm_*``, the formalism the paper uses for the five spins): rho_{j+1} =
  U_j rho_j U_j^H with U_j = exp(-i tau H_j) on the 2^5-dimensional Hilbert space, the adjoint
  chi_j = U_j^H chi_{j+1} U_j from the target, J = Re Tr(chi_Nt^H rho(T)), and
  g_{j,c} = (tau/2)[Im Tr(chi_{j+1}^H [H_c, rho_{j+1}]) + Im Tr(chi_j^H [H_c, rho_j])], the same
  trapezoid form with the Hilbert-Schmidt inner product.  Operators from the paper's definitions:
  I_x, I_y, I_z = sigma/2 on one spin, H0 = 2 pi Jp sum over the couplings of I_z I_z.
"""
from __future__ import annotations

import numpy as np

from .ism_oracle import interval_weights, partition

__all__ = ["pauli_1q", "control_operators", "hamiltonian", "propagate", "propagate_adjoint", "objective",
           "global_gradient", "intermediate_states", "subinterval", "subinterval_all", "ism_iteration",
           "ism_solve", "gradient_method", "dm_operators", "dm_forward", "dm_backward", "dm_objective",
           "dm_gradient"]

_PAULI = {"I": np.eye(2, dtype=np.complex128),
          "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
          "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
          "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128)}


def pauli_1q(q: int, b: int, a: str):
    """The Pauli matrix a on bit b of a q-bit index, as a sparse d x d matrix: kron over the factors
    q-1 .. 0 (bit 0 is the rightmost factor)."""
    from scipy.sparse import csr_matrix, identity, kron

    M = csr_matrix(np.ones((1, 1), dtype=np.complex128))
    for f in range(q - 1, -1, -1):
        M = kron(M, csr_matrix(_PAULI[a]) if f == b else identity(2, dtype=np.complex128, format="csr"), format="csr")
    return M


def control_operators(w):
    """H_c = sum_b ax[c, b] X_b + ay[c, b] Y_b, c = 0..m-1 (sparse, cached in w.meta)."""
    key = "_mc_ops"
    if key in w.meta:
        return w.meta[key]
    X = [pauli_1q(w.q, b, "X") for b in range(w.q)]
    Y = [pauli_1q(w.q, b, "Y") for b in range(w.q)]
    ops = []
    for c in range(w.m):
        Hc = 0 * X[0]
        for b in range(w.q):
            Hc = Hc + w.ax[c, b] * X[b] + w.ay[c, b] * Y[b]
        ops.append(Hc.tocsr())
    w.meta[key] = ops
    return ops


def hamiltonian(w, u_j):
    """H(u_j) = diag(H0d) + sum_c u_{j,c} H_c (sparse)."""
    from scipy.sparse import diags

    H = diags(np.asarray(w.H0d, dtype=np.complex128)).tocsr()
    for c, Hc in enumerate(control_operators(w)):
        H = H + float(u_j[c]) * Hc
    return H


def _step(w, u_j, v, sign):
    """exp(-i sign tau H(u_j)) v (sign = +1 forward, -1 for the adjoint U^H)."""
    H = hamiltonian(w, u_j)
    if w.d <= 64:
        lam, V = np.linalg.eigh(H.toarray())
        return V @ (np.exp(-1j * sign * w.tau * lam) * (V.conj().T @ v))
    from scipy.sparse.linalg import expm_multiply

    return expm_multiply((-1j * sign * w.tau) * H, v)


def propagate(w, u, psi, j0: int, j1: int) -> np.ndarray:
    out = np.empty((j1 - j0 + 1, w.d), dtype=np.complex128)
    out[0] = psi
    for k in range(j1 - j0):
        out[k + 1] = _step(w, u[j0 + k], out[k], +1)
    return out


def propagate_adjoint(w, u, chi_end, j0: int, j1: int) -> np.ndarray:
    out = np.empty((j1 - j0 + 1, w.d), dtype=np.complex128)
    out[-1] = chi_end
    for k in reversed(range(j1 - j0)):
        out[k] = _step(w, u[j0 + k], out[k + 1], -1)
    return out


def objective(w, u, psi=None):
    """(J, F) = (Re<psi(T)|psi_f>, |<psi(T)|psi_f>|^2)."""
    if psi is None:
        psi = propagate(w, u, w.psi_i, 0, w.Nt)
    ov = np.vdot(psi[-1], w.psi_f)
    return float(ov.real), float(abs(ov) ** 2)


def _im_terms(w, chi, psi) -> np.ndarray:
    """Im<chi_j|H_c|psi_j> for every row j and control c: (rows, m)."""
    out = np.empty((psi.shape[0], w.m))
    for c, Hc in enumerate(control_operators(w)):
        out[:, c] = np.imag(np.einsum("jk,jk->j", chi.conj(), (Hc @ psi.T).T))
    return out


def global_gradient(w, u) -> np.ndarray:
    """(Nt, m) trapezoid gradient of J on [0, T]."""
    psi = propagate(w, u, w.psi_i, 0, w.Nt)
    chi = propagate_adjoint(w, u, w.psi_f, 0, w.Nt)
    im = _im_terms(w, chi, psi)
    return 0.5 * w.tau * (im[1:] + im[:-1])


def intermediate_states(w, u) -> np.ndarray:
    j, t, a, b, _ = interval_weights(w.T, w.Nt, w.N)
    psi = propagate(w, u, w.psi_i, 0, w.Nt)
    chi = propagate_adjoint(w, u, w.psi_f, 0, w.Nt)
    return a[:, None] * psi[j] + b[:, None] * chi[j]


def subinterval(w, phi, u, n: int):
    """Sub-problem n (Sec. 2): psi_n from phi_n, chi_n back from phi_{n+1}; (g (steps, m), J_n)."""
    j = partition(w.Nt, w.N)
    j0, j1 = int(j[n]), int(j[n + 1])
    p = propagate(w, u, phi[n], j0, j1)
    c = propagate_adjoint(w, u, phi[n + 1], j0, j1)
    im = _im_terms(w, c, p)
    g = 0.5 * w.tau * (im[1:] + im[:-1])
    Jn = -0.5 * float(np.linalg.norm(p[-1] - phi[n + 1]) ** 2)
    return g, Jn


def subinterval_all(w, phi, u):
    g = np.empty((w.Nt, w.m))
    Jn = np.empty(w.N)
    j = partition(w.Nt, w.N)
    for n in range(w.N):
        g[j[n]:j[n + 1]], Jn[n] = subinterval(w, phi, u, n)
    return g, Jn


def ism_iteration(w, u, rho: float, L: int = 1):
    """Algorithm 1 with the constant-step gradient sub-solver and a vector of controls per step."""
    j, t, a, b, beta = interval_weights(w.T, w.Nt, w.N)
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
            local[j0:j1] = local[j0:j1] + rho * beta[n] * g / w.tau
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
    u = np.array(u0, dtype=np.float64, copy=True)
    J_hist = []
    for _ in range(iters):
        J_hist.append(objective(w, u)[0])
        u = u + rho * global_gradient(w, u) / w.tau
    J_hist.append(objective(w, u)[0])
    return u, np.array(J_hist)


# ----------------------------------------------------------------------------------------------
# Density-matrix form on the Hilbert space of the spins (the paper's formalism for Sec. 4's spins)
# ----------------------------------------------------------------------------------------------
def dm_operators(meta):
    """(H0, [H_c], rho0, rhof) from the spin description: I_a^(k) = sigma_a / 2 on spin k (spin k <->
    tensor factor k-1 from the right), H0 = 2 pi Jp sum_{(k,l)} I_z^(k) I_z^(l), controls ordered
    u_x^1..u_x^ns, u_y^1..u_y^ns; rho0, rhof the initial and target operators, Frobenius-normalised."""
    ns, Jp = meta["spins"], meta["Jp"]

    def I(a, k):
        M = np.ones((1, 1), dtype=np.complex128)
        for f in range(ns - 1, -1, -1):
            M = np.kron(M, 0.5 * _PAULI[a] if f == k - 1 else _PAULI["I"])
        return M

    H0 = 2.0 * np.pi * Jp * sum(I("Z", k) @ I("Z", l) for k, l in meta["couplings"])
    Hc = [I("X", k) for k in range(1, ns + 1)] + [I("Y", k) for k in range(1, ns + 1)]
    r0 = I(meta["initial"][0].upper(), meta["initial"][1])
    rf = I(meta["target"][0].upper(), meta["target"][1])
    return H0, Hc, r0 / np.linalg.norm(r0), rf / np.linalg.norm(rf)


def _dm_unitaries(H0, Hc, tau, u, j0, j1):
    """U_j = exp(-i tau H_j), H_j = H0 + sum_c u_{j,c} H_c, for j in [j0, j1): numpy.linalg.eigh of
    each Hermitian H_j, U_j = V_j diag(exp(-i tau lambda_j)) V_j^H."""
    uu = np.asarray(u[j0:j1], dtype=np.float64)
    Hs = np.asarray(Hc)
    d = H0.shape[0]
    H = H0[None] + (uu.astype(np.complex128) @ Hs.reshape(len(Hs), -1)).reshape(-1, d, d)
    out = []
    for k in range(j1 - j0):
        lam, V = np.linalg.eigh(H[k])
        out.append((V * np.exp(-1j * tau * lam)[None, :]) @ V.conj().T)
    return out


def _dm_chunks(Nt, size=2048):
    return [(a, min(Nt, a + size)) for a in range(0, Nt, size)]


def dm_forward(w, u):
    """rho_j, j = 0..Nt, rho_{j+1} = U_j rho_j U_j^H."""
    H0, Hc, r0, _ = dm_operators(w.meta)
    out = np.empty((w.Nt + 1,) + r0.shape, dtype=np.complex128)
    out[0] = r0
    for a, b in _dm_chunks(w.Nt):
        U = _dm_unitaries(H0, Hc, w.tau, u, a, b)
        for k in range(b - a):
            out[a + k + 1] = U[k] @ out[a + k] @ U[k].conj().T
    return out


def dm_backward(w, u):
    """chi_j, j = 0..Nt, chi_Nt = rho_f, chi_j = U_j^H chi_{j+1} U_j."""
    H0, Hc, _, rf = dm_operators(w.meta)
    out = np.empty((w.Nt + 1,) + rf.shape, dtype=np.complex128)
    out[-1] = rf
    for a, b in reversed(_dm_chunks(w.Nt)):
        U = _dm_unitaries(H0, Hc, w.tau, u, a, b)
        for k in reversed(range(b - a)):
            out[a + k] = U[k].conj().T @ out[a + k + 1] @ U[k]
    return out


def dm_objective(w, u) -> float:
    _, _, _, rf = dm_operators(w.meta)
    return float(np.trace(rf.conj().T @ dm_forward(w, u)[-1]).real)


def dm_gradient(w, u) -> np.ndarray:
    """(Nt, m) trapezoid gradient with Im Tr(chi^H [H_c, rho]) = Im Tr(H_c C), C = rho chi^H - chi^H rho
    (cyclic trace): Tr(H_c C) = sum_ab H_c[a, b] C[b, a]."""
    _, Hc, _, _ = dm_operators(w.meta)
    rho = dm_forward(w, u)
    chi = dm_backward(w, u)
    d = rho.shape[1]
    CT = np.empty((rho.shape[0], d * d), dtype=np.complex128)
    for j in range(rho.shape[0]):
        cH = chi[j].conj().T
        CT[j] = (rho[j] @ cH - cH @ rho[j]).T.reshape(-1)
    im = np.imag(CT @ np.asarray(Hc).reshape(len(Hc), -1).T)
    return 0.5 * w.tau * (im[1:] + im[:-1])
