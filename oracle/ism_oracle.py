"""FP64 CPU oracle for the Intermediate State Method (ISM), Riahi, Salomon, Glaser, Sugny,
"A fully efficient time-parallelized quantum optimal control algorithm" (arXiv:1603.01237).

TEST INFRASTRUCTURE.  This module is the slow, plain, obviously-correct statement of what the CUDA
path computes.  Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  It shares no code with the CUDA path;
the two meet only in the seeded arrays of the ``workloads`` package.

Everything is complex128 / float64; H0 and H1 may be real symmetric or complex Hermitian (Sec. 2 poses
the problem for any Hermitian pair), and every formula below is written for the Hermitian case.
Library primitives used as single steps: ``numpy.linalg.eigh``
(the exact exponential of a Hermitian matrix, U = V exp(-i tau Lambda) V^H) for d <= 64; for larger
d, ``scipy.sparse.linalg.expm_multiply`` (action of the exponential on a vector, Al-Mohy & Higham)
on the sparse H(u_j); and, for the exact discrete derivative pin only, ``scipy.linalg.expm``.  There is no blocking, fusion or reordering
beyond the definitions cited on each function.

Discretisation (Sec. 3): the control is piecewise constant, u_j on step j, j = 0..Nt-1, tau = T/Nt;
step j applies U_j = exp(-i tau H(u_j)) with H(u) = H0 + u H1 (Eq. (dir)).  The paper's Crank-
Nicolson / Strang schemes are replaced by this exponential (exact for piecewise-constant u); its
tau = (t_b - t_a)/(J-1) is read as Nt = J - 1 steps on J grid points.

Readings of the paper taken here (each also listed in the design notes):
 * partition: j_n = floor(n Nt / N), t_n = j_n tau (Sec. 2 allows any partition 0=t_0<...<t_N=T);
 * discrete gradient: trapezoid form g_j = w (tau/2)[Im<chi_{j+1}|H1|psi_{j+1}> + Im<chi_j|H1|psi_j>]
   - tau alpha_j u_j of Eq. (gradJ), which pairs psi_{j+1}+psi_j as the Sec. 3 discrete gradient does
   and is bilinear in (chi, psi), so Theorem 2 holds for it exactly;
 * update: gradient ASCENT u <- u + rho * (L2 gradient) (Eq. gradStep is written as descent while
   the figure of merit is maximised); the L2 gradient on sub-interval n is beta_n g_{n,j} / tau;
 * Err (Algorithm 1 (e)) = sum_n sum_j |g_{n,j}| taken at the first local iteration;
 * observable objective J = <psi(T)|O|psi(T)>: chi(T) = O psi(T) and weight w = 2 on the Im-terms,
   and the sub-functional J_n carries the same weight w so that Theorem 2 keeps the factor beta_n.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "partition", "interval_weights", "step_unitaries", "propagate", "propagate_adjoint",
    "forward_trajectory", "terminal_adjoint", "backward_trajectory", "objective", "weight",
    "global_gradient", "exact_gradient", "intermediate_states", "assembled_intermediate_states",
    "subinterval", "subinterval_all", "j_parallel", "ism_iteration", "ism_solve", "gradient_method",
]


# ----------------------------------------------------------------------------------------------
# Time partition (Sec. 2: [0,T] = U_n [t_n, t_{n+1}], beta_n = T/(t_{n+1}-t_n), alpha_n = alpha/beta_n)
# ----------------------------------------------------------------------------------------------
def partition(Nt: int, N: int) -> np.ndarray:
    """Step indices j_n = floor(n Nt / N), n = 0..N (so t_n = j_n tau)."""
    if not (1 <= N <= Nt):
        raise ValueError("need 1 <= N <= Nt")
    return np.array([(n * Nt) // N for n in range(N + 1)], dtype=np.int64)


def interval_weights(T: float, Nt: int, N: int):
    """t_n, a_n = (T - t_n)/T, b_n = t_n/T (Eq. (cible)), beta_n = T/(t_{n+1} - t_n) (Theorem 1)."""
    tau = T / Nt
    j = partition(Nt, N)
    t = j * tau
    a = (T - t) / T
    b = t / T
    beta = T / (t[1:] - t[:-1])
    return j, t, a, b, beta


# ----------------------------------------------------------------------------------------------
# Propagation (Eq. (dir), Eq. (adj)) with the exact step exponential
# ----------------------------------------------------------------------------------------------
def step_unitaries(w, u, j0: int, j1: int) -> np.ndarray:
    """U_j = exp(-i tau (H0 + u_j H1)) for j in [j0, j1), stacked (j1-j0, d, d)."""
    tau = w.T / w.Nt
    H = w.H0[None, :, :] + np.asarray(u[j0:j1], dtype=np.float64)[:, None, None] * w.H1[None, :, :]
    lam, V = np.linalg.eigh(H)
    return (V * np.exp(-1j * tau * lam)[:, None, :]) @ np.conj(np.swapaxes(V, 1, 2))


def _chunks(j0, j1, size=2048):
    a = j0
    while a < j1:
        b = min(j1, a + size)
        yield a, b
        a = b


DENSE_MAX = 64


def _sparse_H(w):
    from scipy.sparse import csr_matrix

    key = "_oracle_sparse"
    cache = getattr(w, "meta", None)
    if cache is not None and key in cache:
        return cache[key]
    pair = (csr_matrix(w.H0), csr_matrix(w.H1))
    if cache is not None:
        cache[key] = pair
    return pair


def _expm_step(w, u_j, v, sign):
    """exp(sign * -i tau H(u_j)) v for large d (sign = +1 forward, -1 adjoint)."""
    from scipy.sparse.linalg import expm_multiply

    H0s, H1s = _sparse_H(w)
    tau = w.T / w.Nt
    A = (-1j * sign * tau) * (H0s + float(u_j) * H1s)
    return expm_multiply(A, v)


def propagate(w, u, psi, j0: int, j1: int) -> np.ndarray:
    """psi_{j+1} = U_j psi_j for j = j0..j1-1 starting from psi; returns (j1-j0+1, d) states."""
    out = np.empty((j1 - j0 + 1, w.d), dtype=np.complex128)
    out[0] = psi
    if w.d > DENSE_MAX:
        for k in range(j1 - j0):
            out[k + 1] = _expm_step(w, u[j0 + k], out[k], +1)
        return out
    for a, b in _chunks(j0, j1):
        U = step_unitaries(w, u, a, b)
        for k in range(b - a):
            out[a - j0 + k + 1] = U[k] @ out[a - j0 + k]
    return out


def propagate_adjoint(w, u, chi_end, j0: int, j1: int) -> np.ndarray:
    """chi_j = U_j^dagger chi_{j+1} for j = j1-1..j0 ending at chi_{j1} = chi_end; (j1-j0+1, d)."""
    out = np.empty((j1 - j0 + 1, w.d), dtype=np.complex128)
    out[-1] = chi_end
    if w.d > DENSE_MAX:
        for k in reversed(range(j1 - j0)):
            out[k] = _expm_step(w, u[j0 + k], out[k + 1], -1)
        return out
    chunks = list(_chunks(j0, j1))
    for a, b in reversed(chunks):
        U = step_unitaries(w, u, a, b)
        for k in reversed(range(b - a)):
            out[a - j0 + k] = U[k].conj().T @ out[a - j0 + k + 1]
    return out


def forward_trajectory(w, u) -> np.ndarray:
    """psi_j, j = 0..Nt, from psi(0) = psi_i (Eq. (dir))."""
    return propagate(w, u, w.psi_i, 0, w.Nt)


def terminal_adjoint(w, psi_T) -> np.ndarray:
    """chi(T): psi_f for the overlap objective (Eq. (adj)); O psi(T) for <psi(T)|O|psi(T)>."""
    if w.objective == "overlap":
        return np.asarray(w.psi_f, dtype=np.complex128)
    return w.O @ psi_T


def backward_trajectory(w, u, chi_T) -> np.ndarray:
    """chi_j, j = 0..Nt, with chi_Nt = chi(T) (Eq. (adj) discretised with the same U_j)."""
    return propagate_adjoint(w, u, chi_T, 0, w.Nt)


def weight(w) -> float:
    """Factor on the Im<chi|H1|psi> terms: 1 for Re<psi(T)|psi_f>, 2 for <psi(T)|O|psi(T)>."""
    return 1.0 if w.objective == "overlap" else 2.0


def _alpha(w) -> np.ndarray:
    return np.zeros(w.Nt) if w.alpha is None else np.asarray(w.alpha, dtype=np.float64)


def penalty(w, u) -> float:
    """(tau/2) sum_j alpha_j u_j^2, the discrete control cost of J (Sec. 2, Sec. 3 J_tau)."""
    tau = w.T / w.Nt
    return 0.5 * tau * float(np.sum(_alpha(w) * np.asarray(u) ** 2))


def objective(w, u, psi=None):
    """(J, F): J = Re<psi(T)|psi_f> - penalty and F = |<psi(T)|psi_f>|^2 (overlap), or
    J = <psi(T)|O|psi(T)> - penalty and F = <psi(T)|O|psi(T)> (observable)."""
    if psi is None:
        psi = forward_trajectory(w, u)
    pT = psi[-1]
    if w.objective == "overlap":
        ov = np.vdot(pT, w.psi_f)
        return float(ov.real) - penalty(w, u), float(abs(ov) ** 2)
    val = float(np.vdot(pT, w.O @ pT).real)
    return val - penalty(w, u), val


def global_gradient(w, u) -> np.ndarray:
    """Discrete gradient of J on the full interval (Eq. (gradJ), trapezoid in each step):
    g_j = w (tau/2)[Im<chi_{j+1}|H1|psi_{j+1}> + Im<chi_j|H1|psi_j>] - tau alpha_j u_j."""
    tau = w.T / w.Nt
    psi = forward_trajectory(w, u)
    chi = backward_trajectory(w, u, terminal_adjoint(w, psi[-1]))
    im = np.imag(np.einsum("jk,jk->j", chi.conj(), psi @ w.H1.T))   # Im<chi_j|H1|psi_j>
    return weight(w) * 0.5 * tau * (im[1:] + im[:-1]) - tau * _alpha(w) * np.asarray(u)


def exact_gradient(w, u) -> np.ndarray:
    """Exact derivative dJ/du_j of the discrete J, via the block exponential (Van Loan 1978):
    exp([[A, E], [0, A]]) has dU/du in its top-right block for A = -i tau H(u_j), E = -i tau H1."""
    from scipy.linalg import expm

    tau = w.T / w.Nt
    d = w.d
    psi = forward_trajectory(w, u)
    chi = backward_trajectory(w, u, terminal_adjoint(w, psi[-1]))
    g = np.empty(w.Nt)
    Z = np.zeros((d, d))
    for j in range(w.Nt):
        A = -1j * tau * (w.H0 + u[j] * w.H1)
        E = -1j * tau * w.H1
        B = expm(np.block([[A, E], [Z, A]]))
        dU = B[:d, d:]
        g[j] = weight(w) * float(np.vdot(chi[j + 1], dU @ psi[j]).real)
    return g - tau * _alpha(w) * np.asarray(u)


# ----------------------------------------------------------------------------------------------
# Intermediate states (Eq. (cible)) and propagator assembly (Sec. 3)
# ----------------------------------------------------------------------------------------------
def intermediate_states(w, u) -> np.ndarray:
    """phi_n = ((T - t_n)/T) psi(t_n) + (t_n/T) chi(t_n), n = 0..N, from the full sweeps
    (Algorithm 1 steps (a) and (b)).  phi_0 = psi_i and phi_N = chi(T) up to rounding."""
    j, t, a, b, _ = interval_weights(w.T, w.Nt, w.N)
    psi = forward_trajectory(w, u)
    chi = backward_trajectory(w, u, terminal_adjoint(w, psi[-1]))
    return a[:, None] * psi[j] + b[:, None] * chi[j]


def assembled_intermediate_states(w, u) -> np.ndarray:
    """Same phi_n through the propagator-assembly route of Sec. 3: M_n = prod_{j in sub-interval n}
    U_j (later steps on the left), psi(t_{n+1}) = M_n psi(t_n), chi(t_n) = M_n^dagger chi(t_{n+1})."""
    j, t, a, b, _ = interval_weights(w.T, w.Nt, w.N)
    M = []
    for n in range(w.N):
        U = step_unitaries(w, u, int(j[n]), int(j[n + 1]))
        Mn = np.eye(w.d, dtype=np.complex128)
        for k in range(U.shape[0]):
            Mn = U[k] @ Mn
        M.append(Mn)
    psi = [np.asarray(w.psi_i, dtype=np.complex128)]
    for n in range(w.N):
        psi.append(M[n] @ psi[n])
    chi = [None] * (w.N + 1)
    chi[w.N] = terminal_adjoint(w, psi[w.N])
    for n in reversed(range(w.N)):
        chi[n] = M[n].conj().T @ chi[n + 1]
    return np.array([a[n] * psi[n] + b[n] * chi[n] for n in range(w.N + 1)])


# ----------------------------------------------------------------------------------------------
# Sub-interval problems (Sec. 2: J_n, Eq. (dirpara); gradient of J_n from the proof of Theorem 2)
# ----------------------------------------------------------------------------------------------
def subinterval(w, phi, u, n: int):
    """Sub-problem n with targets phi: psi_n from psi_n(t_n) = phi_n (Eq. (dirpara)), chi_n backward
    from chi_n(t_{n+1}) = phi_{n+1}.  Returns (g, J_n) with
      J_n = w * (-1/2 ||psi_n(t_{n+1}) - phi_{n+1}||^2) - (tau/2) sum_j (alpha_j / beta_n) u_j^2,
      g_j = w (tau/2)[Im<chi_n,j+1|H1|psi_n,j+1> + Im<chi_n,j|H1|psi_n,j>] - tau (alpha_j/beta_n) u_j,
    g_j being dJ_n/du_j in the trapezoid reading (alpha_n = alpha (t_{n+1}-t_n)/T)."""
    j, t, a, b, beta = interval_weights(w.T, w.Nt, w.N)
    tau = w.T / w.Nt
    j0, j1 = int(j[n]), int(j[n + 1])
    p = propagate(w, u, phi[n], j0, j1)
    c = propagate_adjoint(w, u, phi[n + 1], j0, j1)
    im = np.imag(np.einsum("jk,jk->j", c.conj(), p @ w.H1.T))
    al = _alpha(w)[j0:j1] / beta[n]
    uu = np.asarray(u[j0:j1], dtype=np.float64)
    g = weight(w) * 0.5 * tau * (im[1:] + im[:-1]) - tau * al * uu
    Jn = weight(w) * (-0.5 * float(np.linalg.norm(p[-1] - phi[n + 1]) ** 2)) - 0.5 * tau * float(np.sum(al * uu ** 2))
    return g, Jn


def subinterval_all(w, phi, u):
    """All N sub-problems at one control (Algorithm 1 step (c), one gradient evaluation each):
    returns the concatenated g (Nt,) and J_n (N,)."""
    g = np.empty(w.Nt)
    Jn = np.empty(w.N)
    j = partition(w.Nt, w.N)
    for n in range(w.N):
        g[j[n]:j[n + 1]], Jn[n] = subinterval(w, phi, u, n)
    return g, Jn


def j_parallel(w, phi, u) -> float:
    """J_par[u, phi] = sum_n beta_n J_n[u_n, phi] (Sec. 2, before Theorem 1)."""
    _, _, _, _, beta = interval_weights(w.T, w.Nt, w.N)
    _, Jn = subinterval_all(w, phi, u)
    return float(np.sum(beta * Jn))


# ----------------------------------------------------------------------------------------------
# Algorithm 1 with the constant-step gradient sub-solver (Eq. gradStep, ascent reading)
# ----------------------------------------------------------------------------------------------
def ism_iteration(w, u, rho: float, L: int = 1):
    """One pass of Algorithm 1 loop body: (a) psi, chi on [0,T]; (b) phi (Eq. (cible)); (c) on each
    sub-interval L steps u_n <- u_n + rho beta_n g_n / tau with phi fixed; (d) concatenate;
    (e) Err = sum_n sum_j |g_{n,j}| of the first local step.  Returns (u_next, Err, J_n at u)."""
    j, t, a, b, beta = interval_weights(w.T, w.Nt, w.N)
    tau = w.T / w.Nt
    phi = intermediate_states(w, u)
    u_next = np.array(u, dtype=np.float64, copy=True)
    err = 0.0
    Jn0 = np.empty(w.N)
    for n in range(w.N):
        j0, j1 = int(j[n]), int(j[n + 1])
        local = np.array(u, dtype=np.float64, copy=True)
        for ell in range(L):
            g, Jn = subinterval(w, phi, local, n)
            if ell == 0:
                err += float(np.sum(np.abs(g)))
                Jn0[n] = Jn
            local[j0:j1] = local[j0:j1] + rho * beta[n] * g / tau
        u_next[j0:j1] = local[j0:j1]
    return u_next, err, Jn0


def ism_solve(w, u0, iters: int, rho: float, L: int = 1):
    """Run Algorithm 1 for a fixed number of iterations.  Returns (u, J_hist (iters+1), F_hist
    (iters+1), err_hist (iters)); J_hist[k] = J[u^(k)]."""
    u = np.array(u0, dtype=np.float64, copy=True)
    J_hist, F_hist, err_hist = [], [], []
    for _ in range(iters):
        J, F = objective(w, u)
        J_hist.append(J)
        F_hist.append(F)
        u, err, _ = ism_iteration(w, u, rho, L)
        err_hist.append(err)
    J, F = objective(w, u)
    J_hist.append(J)
    F_hist.append(F)
    return u, np.array(J_hist), np.array(F_hist), np.array(err_hist)


def gradient_method(w, u0, iters: int, rho: float):
    """The plain sequential gradient method on J (no decomposition): u <- u + rho g / tau with g the
    full-interval discrete gradient.  ISM with N = 1 must reproduce it."""
    tau = w.T / w.Nt
    u = np.array(u0, dtype=np.float64, copy=True)
    J_hist = []
    for _ in range(iters):
        J_hist.append(objective(w, u)[0])
        u = u + rho * global_gradient(w, u) / tau
    J_hist.append(objective(w, u)[0])
    return u, np.array(J_hist)
