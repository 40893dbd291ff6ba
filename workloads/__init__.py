"""Seeded synthetic workloads for the Intermediate State Method (ISM) hot path.

Every generator draws its random numbers from ``numpy.random.default_rng(seed)`` in a fixed,
documented order and returns plain arrays: dense real-symmetric ``H0`` and ``H1`` (the control
Hamiltonian is H(u) = H0 + u*H1, Sec. 2, Eq. (dir)), the initial state, the target (a state for the
overlap objective of Sec. 2, or an observable for the variant the paper calls straightforward),
the time grid and the initial control.

Both the CUDA path and the FP64 oracle consume exactly these arrays.  This module computes
nothing of the method itself (no propagation, no intermediate states, no gradients): it only
builds the physical model matrices and draws random numbers.

Models
------
* ``spin_all_to_all``  : q spin-1/2 with H0 = sum_{i<j} J_ij Z_i Z_j, H1 = sum_i X_i.
  Basis index s, spin i <-> bit i of s, Z_i|s> = (1 - 2 bit_i(s))|s>.
* ``spin_chain``       : same with nearest-neighbour open-chain couplings only.
* ``rotor``            : rigid rotor in the |j, m=0> basis, j = 0..jmax, H0 = diag(j(j+1)) (units
  of B), H1 = -cos(theta) with <j|cos theta|j+1> = (j+1)/sqrt((2j+1)(2j+3)) (textbook m=0 matrix
  element); the orientation objective is <psi(T)|cos theta|psi(T)> (Sec. 4, molecular orientation).
* ``random_dense``     : random real-symmetric H0, H1 for generic parity tests.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "Workload",
    "spin_all_to_all",
    "spin_chain",
    "rotor",
    "random_dense",
    "random_hermitian",
    "gauge",
    "rabi",
    "config",
    "CONFIG_NAMES",
    "GPWorkload",
    "gp_bec",
    "gp_stationary_states",
    "gp_double_well",
    "gp_ground_state",
    "MCWorkload",
    "random_pauli",
    "spin5_liouville",
]


@dataclass
class Workload:
    """One ISM control problem (Sec. 2) plus the run settings used with it."""

    name: str
    kind: str                    # structure hint for the CUDA path: "bitflip" | "tridiag" | "dense"
    H0: np.ndarray               # (d, d) float64 real symmetric, or complex128 Hermitian (dense kind)
    H1: np.ndarray               # (d, d) float64 real symmetric, or complex128 Hermitian (dense kind)
    psi_i: np.ndarray            # (d,) complex128
    objective: str               # "overlap" (target psi_f) | "observable" (target O)
    psi_f: Optional[np.ndarray]  # (d,) complex128 when objective == "overlap"
    O: Optional[np.ndarray]      # (d, d) float64 when objective == "observable"
    T: float
    Nt: int                      # number of piecewise-constant steps, tau = T / Nt
    N: int                       # number of sub-intervals
    u0: np.ndarray               # (Nt,) float64 initial control
    alpha: Optional[np.ndarray] = None   # (Nt,) penalty weight at step midpoints, None = 0
    iters: int = 20
    rho: float = 0.1
    local_iters: int = 1
    precision: str = "fp64"      # "fp64" | "mixed"
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return int(self.H0.shape[0])

    @property
    def tau(self) -> float:
        return self.T / self.Nt

    def with_(self, **kw) -> "Workload":
        """Copy with some fields replaced (arrays are shared, not copied)."""
        import dataclasses

        return dataclasses.replace(self, **kw)


def _basis(d: int, k: int) -> np.ndarray:
    v = np.zeros(d, dtype=np.complex128)
    v[k] = 1.0
    return v


def _zz_diagonal(q: int, pairs, J) -> np.ndarray:
    d = 1 << q
    s = np.arange(d)
    z = 1.0 - 2.0 * ((s[:, None] >> np.arange(q)[None, :]) & 1)   # (d, q) eigenvalues of Z_i
    diag = np.zeros(d)
    for (i, j), Jij in zip(pairs, J):
        diag += Jij * z[:, i] * z[:, j]
    return diag


def _x_field(q: int, weights=None) -> np.ndarray:
    d = 1 << q
    w = np.ones(q) if weights is None else np.asarray(weights, dtype=np.float64)
    H1 = np.zeros((d, d))
    s = np.arange(d)
    for i in range(q):
        H1[s, s ^ (1 << i)] += w[i]
    return H1


def spin_all_to_all(q: int, seed: int, *, T: float, Nt: int, N: int, u_amp: float = 0.1,
                    name: str = "spin") -> Workload:
    """q spins, all pairs i<j in lexicographic order, J_ij ~ U[0.5, 1.5]; then u0 ~ U[-u_amp, u_amp].

    psi_i = |0...0>, psi_f = |1...1>, overlap objective, alpha = 0.
    """
    rng = np.random.default_rng(seed)
    pairs = [(i, j) for i in range(q) for j in range(i + 1, q)]
    J = rng.uniform(0.5, 1.5, size=len(pairs))
    u0 = rng.uniform(-u_amp, u_amp, size=Nt)
    d = 1 << q
    return Workload(name=name, kind="bitflip", H0=np.diag(_zz_diagonal(q, pairs, J)), H1=_x_field(q),
                    psi_i=_basis(d, 0), objective="overlap", psi_f=_basis(d, d - 1), O=None,
                    T=T, Nt=Nt, N=N, u0=u0, meta={"q": q, "pairs": pairs, "J": J})


def spin_chain(q: int, seed: int, *, T: float, Nt: int, N: int, u_amp: float = 0.1,
               name: str = "ising") -> Workload:
    """Open chain: J_i ~ U[0.5, 1.5] for bonds (i, i+1), i = 0..q-2; then u0 ~ U[-u_amp, u_amp]."""
    rng = np.random.default_rng(seed)
    pairs = [(i, i + 1) for i in range(q - 1)]
    J = rng.uniform(0.5, 1.5, size=len(pairs))
    u0 = rng.uniform(-u_amp, u_amp, size=Nt)
    d = 1 << q
    return Workload(name=name, kind="bitflip", H0=np.diag(_zz_diagonal(q, pairs, J)), H1=_x_field(q),
                    psi_i=_basis(d, 0), objective="overlap", psi_f=_basis(d, d - 1), O=None,
                    T=T, Nt=Nt, N=N, u0=u0, meta={"q": q, "pairs": pairs, "J": J})


def rotor_cos_theta(jmax: int) -> np.ndarray:
    """cos(theta) in the |j, m=0> basis, j = 0..jmax (tridiagonal, zero diagonal)."""
    d = jmax + 1
    j = np.arange(d - 1, dtype=np.float64)
    c = (j + 1.0) / np.sqrt((2.0 * j + 1.0) * (2.0 * j + 3.0))
    C = np.zeros((d, d))
    C[np.arange(d - 1), np.arange(1, d)] = c
    C[np.arange(1, d), np.arange(d - 1)] = c
    return C


def rotor(jmax: int, seed: int, *, T: float, Nt: int, N: int, u_amp: float = 1.0,
          alpha0: float = 1e-3, objective: str = "observable", name: str = "rotor") -> Workload:
    """Rigid rotor; u0 ~ U[-u_amp, u_amp] is the only random draw.

    alpha(t) = alpha0 * (10 * ((t - T/2)/(T/2))**6 + 1), the shape of the paper's rotor penalty
    (Sec. 4), sampled at step midpoints.  objective "observable" maximises <cos theta>(T);
    objective "overlap" targets the max-eigenvalue eigenvector of cos theta restricted to j <= 4.
    """
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(-u_amp, u_amp, size=Nt)
    d = jmax + 1
    jj = np.arange(d, dtype=np.float64)
    C = rotor_cos_theta(jmax)
    tau = T / Nt
    tm = (np.arange(Nt) + 0.5) * tau
    alpha = alpha0 * (10.0 * ((tm - T / 2) / (T / 2)) ** 6 + 1.0)
    psi_f = None
    O = None
    if objective == "observable":
        O = C
    else:
        w, V = np.linalg.eigh(C[:5, :5])
        psi_f = np.zeros(d, dtype=np.complex128)
        psi_f[:5] = V[:, -1] * np.sign(V[0, -1])
    return Workload(name=name, kind="tridiag", H0=np.diag(jj * (jj + 1.0)), H1=-C, psi_i=_basis(d, 0),
                    objective=objective, psi_f=psi_f, O=O, T=T, Nt=Nt, N=N, u0=u0, alpha=alpha,
                    meta={"jmax": jmax, "alpha0": alpha0})


def random_dense(d: int, seed: int, *, T: float, Nt: int, N: int, u_amp: float = 0.5,
                 objective: str = "overlap", name: str = "dense") -> Workload:
    """Random real-symmetric H0, H1 (entries N(0,1), symmetrised, scaled by 1/sqrt(d)), random unit
    psi_i and psi_f (or a random symmetric observable), u0 ~ U[-u_amp, u_amp].  Draw order: H0, H1,
    psi_i (re, im), target, u0."""
    rng = np.random.default_rng(seed)

    def sym():
        A = rng.standard_normal((d, d))
        return (A + A.T) / np.sqrt(2.0 * d)

    H0 = sym()
    H1 = sym()

    def unit():
        v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
        return v / np.linalg.norm(v)

    psi_i = unit()
    psi_f = None
    O = None
    if objective == "overlap":
        psi_f = unit()
    else:
        O = sym()
    u0 = rng.uniform(-u_amp, u_amp, size=Nt)
    return Workload(name=name, kind="dense", H0=H0, H1=H1, psi_i=psi_i, objective=objective,
                    psi_f=psi_f, O=O, T=T, Nt=Nt, N=N, u0=u0)


def random_hermitian(d: int, seed: int, *, T: float, Nt: int, N: int, u_amp: float = 0.5,
                     objective: str = "overlap", name: str = "hermitian") -> Workload:
    """Random complex Hermitian H0, H1: (A + A^H)/sqrt(4d) with Re A, Im A entries N(0,1) (so that
    E|H_ef|^2 = 1/d off the diagonal, as for random_dense), random unit psi_i and psi_f (or a random
    real symmetric observable), u0 ~ U[-u_amp, u_amp].  Draw order: Re A0, Im A0, Re A1, Im A1, psi_i
    (re, im), target, u0."""
    rng = np.random.default_rng(seed)

    def herm():
        A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
        return (A + A.conj().T) / np.sqrt(4.0 * d)

    H0 = herm()
    H1 = herm()

    def unit():
        v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
        return v / np.linalg.norm(v)

    psi_i = unit()
    psi_f = None
    O = None
    if objective == "overlap":
        psi_f = unit()
    else:
        A = rng.standard_normal((d, d))
        O = (A + A.T) / np.sqrt(2.0 * d)
    u0 = rng.uniform(-u_amp, u_amp, size=Nt)
    return Workload(name=name, kind="dense", H0=H0, H1=H1, psi_i=psi_i, objective=objective,
                    psi_f=psi_f, O=O, T=T, Nt=Nt, N=N, u0=u0)


def gauge(w: Workload, theta: np.ndarray) -> Workload:
    """The same control problem in the basis rotated by D = diag(exp(i theta)): H -> D H D^H,
    psi -> D psi (a real observable O is kept only when theta makes D O D^H = O, i.e. never here:
    the overlap objective only).  Every quantity of Algorithm 1 is invariant under this change."""
    if w.objective != "overlap":
        raise ValueError("gauge() keeps the overlap objective only")
    D = np.exp(1j * np.asarray(theta, dtype=np.float64))
    rot = lambda H: D[:, None] * H * D.conj()[None, :]   # noqa: E731
    return w.with_(H0=rot(w.H0), H1=rot(w.H1), psi_i=D * w.psi_i, psi_f=D * w.psi_f, name=w.name + "-gauge")


def rabi(delta: float, u: float, *, T: float, Nt: int, N: int = 1) -> Workload:
    """Two-level system H = (delta/2) sigma_z + (u/2) sigma_x with a constant control u."""
    H0 = np.diag([delta / 2.0, -delta / 2.0])
    H1 = np.array([[0.0, 0.5], [0.5, 0.0]])
    return Workload(name="rabi", kind="dense", H0=H0, H1=H1, psi_i=_basis(2, 0), objective="overlap",
                    psi_f=_basis(2, 1), O=None, T=T, Nt=Nt, N=N, u0=np.full(Nt, float(u)))


# ----------------------------------------------------------------------------------------------
# The named benchmark configurations.  Seed = 1000 + configuration index.
# ----------------------------------------------------------------------------------------------
def with_random_target(w: Workload, seed: int) -> Workload:
    """The same problem with a seeded random unit target (standard normal real and imaginary parts,
    normalised), so that overlaps and gradients are O(1) from any start."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(w.d) + 1j * rng.standard_normal(w.d)
    return w.with_(psi_f=v / np.linalg.norm(v))


CONFIG_NAMES = ("spin16", "rotor41", "gp512", "ising1024")


def config(name: str, *, N: Optional[int] = None, Nt: Optional[int] = None, iters: Optional[int] = None,
           precision: Optional[str] = None) -> Workload:
    """The synthetic stand-ins for the four benchmark problems.

    spin16    : 4 spins (d=16), all-to-all ZZ, X control, |0000> -> |1111>, T=10, Nt=1000, N=4,
                u0 ~ U[-0.1, 0.1], 20 iterations, FP64.
    rotor41   : rigid rotor j=0..40 (d=41), maximise <cos theta>(T), T=pi, Nt=20000, N=128 (16 and
                64 also used), u0 ~ U[-1, 1], 50 iterations, mixed precision.
    ising1024 : 10-spin open Ising chain (d=1024), |0^10> -> |1^10>, T=10, Nt=50000, N=256,
                u0 ~ U[-0.1, 0.1], 20 iterations, mixed precision.
    """
    if name == "spin16":
        w = spin_all_to_all(4, 1000, T=10.0, Nt=Nt or 1000, N=N or 4, name=name)
        w = w.with_(iters=iters or 20, rho=30.0, precision=precision or "fp64")
    elif name == "rotor41":
        w = rotor(40, 1001, T=float(np.pi), Nt=Nt or 20000, N=N or 128, name=name)
        w = w.with_(iters=iters or 50, rho=1.0, precision=precision or "mixed")
    elif name == "ising1024":
        w = spin_chain(10, 1003, T=10.0, Nt=Nt or 50000, N=N or 256, name=name)
        w = w.with_(iters=iters or 20, rho=0.2, precision=precision or "mixed")
    else:
        raise KeyError(name)
    return w


# ----------------------------------------------------------------------------------------------
# Gross-Pitaevskii condensate on a periodic grid (Sec. 4, Bose-Einstein condensates)
# ----------------------------------------------------------------------------------------------
@dataclass
class GPWorkload:
    """1D GP problem: i d/dt psi = (-1/2 d^2/dx^2 + V(x, u) + g |psi|^2) psi on a periodic grid,
    V(x, u) = (x - u)^2 / 2 (harmonic) or the double well of separation dw (potential =
    "double_well"), maximise J = Re<psi(T)|psi_f> with <a|b> = sum conj(a) b dx."""

    name: str
    n: int              # grid points
    L: float            # box length; x_k = x_min + k L / n
    x_min: float
    g: float
    psi_i: np.ndarray   # (n,) complex128, normalised sum |psi|^2 dx = 1
    psi_f: np.ndarray
    T: float
    Nt: int
    N: int
    u0: np.ndarray
    iters: int = 20
    rho: float = 0.1
    local_iters: int = 1
    precision: str = "mixed"
    kind: str = "gp"
    objective: str = "overlap"
    alpha: Optional[np.ndarray] = None
    potential: str = "harmonic"   # "harmonic": (x - u)^2/2; "double_well": the split trap, separation dw
    dw: float = 0.0

    @property
    def dx(self) -> float:
        return self.L / self.n

    @property
    def x(self) -> np.ndarray:
        return self.x_min + np.arange(self.n) * self.dx

    @property
    def k(self) -> np.ndarray:
        return 2.0 * np.pi * np.fft.fftfreq(self.n, d=self.dx)

    @property
    def tau(self) -> float:
        return self.T / self.Nt

    def with_(self, **kw) -> "GPWorkload":
        import dataclasses

        return dataclasses.replace(self, **kw)


def gp_stationary_states(n: int, L: float, x_min: float, g: float, *, dt: float = 1e-3, steps: int = 40000):
    """Ground state and lowest odd state of -1/2 d^2 + x^2/2 + g|psi|^2 on the periodic grid, by
    imaginary-time split steps with renormalisation (the odd state also antisymmetrised about x = 0
    and orthogonalised against the ground state at every step).  Model set-up only."""
    x = x_min + np.arange(n) * (L / n)
    dx = L / n
    kk = 2.0 * np.pi * np.fft.fftfreq(n, d=dx)
    half = np.exp(-0.25 * dt * kk ** 2)
    V = 0.5 * x ** 2

    def norm(v):
        return v / np.sqrt(np.sum(np.abs(v) ** 2) * dx)

    def mirror(v):   # v(-x) on the grid x_k = x_min + k dx with x_min = -L/2: index (n - k) mod n
        return v[(-np.arange(n)) % n]

    g0 = norm(np.exp(-0.5 * x ** 2).astype(np.complex128))
    e1 = norm((x * np.exp(-0.5 * x ** 2)).astype(np.complex128))
    for _ in range(steps):
        g0 = np.fft.ifft(half * np.fft.fft(g0))
        g0 = g0 * np.exp(-dt * (V + g * np.abs(g0) ** 2))
        g0 = norm(np.fft.ifft(half * np.fft.fft(g0)))
        e1 = np.fft.ifft(half * np.fft.fft(e1))
        e1 = e1 * np.exp(-dt * (V + g * np.abs(e1) ** 2))
        e1 = np.fft.ifft(half * np.fft.fft(e1))
        e1 = 0.5 * (e1 - mirror(e1))
        e1 = e1 - np.sum(np.conj(g0) * e1) * dx * g0
        e1 = norm(e1)
    return g0, e1


def gp_bec(n: int = 512, seed: int = 1002, *, T: float = 8.0, Nt: int = 10000, N: int = 64, g: float = 1.0,
           u_amp: float = 0.1, steps: int = 40000, name: str = "gp512", states=None) -> GPWorkload:
    """Grid of n points on [-10, 10) (periodic), g = 1, T = 8, ground state -> lowest odd state,
    u0 ~ U[-u_amp, u_amp] (the only random draw).  `states` = (psi_i, psi_f) reuses stationary states
    already computed for the same (n, g, steps)."""
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(-u_amp, u_amp, size=Nt)
    L, x_min = 20.0, -10.0
    psi_i, psi_f = states if states is not None else gp_stationary_states(n, L, x_min, g, steps=steps)
    return GPWorkload(name=name, n=n, L=L, x_min=x_min, g=g, psi_i=psi_i, psi_f=psi_f, T=T, Nt=Nt, N=N, u0=u0)


def double_well_values(x: np.ndarray, lam: float, dw: float) -> np.ndarray:
    """The double-well potential on a grid at control lam (model set-up for the stationary states)."""
    ax = np.abs(x)
    return np.where(ax > lam * dw / 4.0, 0.5 * (ax - lam * dw / 2.0) ** 2, 0.5 * ((lam * dw) ** 2 / 8.0 - x ** 2))


def gp_ground_state(n: int, L: float, x_min: float, g: float, V: np.ndarray, *, dt: float = 1e-3,
                    steps: int = 40000) -> np.ndarray:
    """Ground state of -1/2 d^2 + V + g|psi|^2 on the periodic grid by imaginary-time split steps with
    renormalisation, started from a Gaussian.  Model set-up only."""
    x = x_min + np.arange(n) * (L / n)
    dx = L / n
    kk = 2.0 * np.pi * np.fft.fftfreq(n, d=dx)
    half = np.exp(-0.25 * dt * kk ** 2)
    v = np.exp(-0.5 * x ** 2).astype(np.complex128)
    v = v / np.sqrt(np.sum(np.abs(v) ** 2) * dx)
    for _ in range(steps):
        v = np.fft.ifft(half * np.fft.fft(v))
        v = v * np.exp(-dt * (V + g * np.abs(v) ** 2))
        v = np.fft.ifft(half * np.fft.fft(v))
        v = v / np.sqrt(np.sum(np.abs(v) ** 2) * dx)
    return v


def gp_double_well(n: int = 512, seed: int = 1005, *, T: float = 8.0, Nt: int = 10000, N: int = 64,
                   g: float = 1.0, dw: float = 4.0, u_amp: float = 0.05, steps: int = 20000,
                   name: str = "gp512dw", states=None) -> GPWorkload:
    """Condensate splitting in the double well of Sec. 4 on the grid of gp_bec: psi_i = ground state
    of V(x, 0) (the harmonic trap), psi_f = ground state of V(x, 1) (two wells at +-dw/2), control
    lambda(t), initial guess the ramp t/T plus U[-u_amp, u_amp] (the only random draw)."""
    rng = np.random.default_rng(seed)
    tm = (np.arange(Nt) + 0.5) * (T / Nt)
    u0 = tm / T + rng.uniform(-u_amp, u_amp, size=Nt)
    L, x_min = 20.0, -10.0
    if states is None:
        x = x_min + np.arange(n) * (L / n)
        states = (gp_ground_state(n, L, x_min, g, double_well_values(x, 0.0, dw), steps=steps),
                  gp_ground_state(n, L, x_min, g, double_well_values(x, 1.0, dw), steps=steps))
    psi_i, psi_f = states
    return GPWorkload(name=name, n=n, L=L, x_min=x_min, g=g, psi_i=psi_i, psi_f=psi_f, T=T, Nt=Nt, N=N, u0=u0,
                      potential="double_well", dw=dw)


# ----------------------------------------------------------------------------------------------
# Several controls on a Pauli structure (the five-spin example of Sec. 4)
# ----------------------------------------------------------------------------------------------
@dataclass
class MCWorkload:
    """A control problem with m controls: H(t) = diag(H0d) + sum_c u_c(t) H_c, H_c = sum_b
    (ax[c, b] X_b + ay[c, b] Y_b) on d = 2^q basis states (bit b of the index <-> X_b, Y_b; Pauli
    Y = [[0, -i], [i, 0]]), maximise J = Re<psi(T)|psi_f>.  u0 is (Nt, m)."""

    name: str
    q: int
    H0d: np.ndarray      # (d,) float64
    ax: np.ndarray       # (m, q) float64
    ay: np.ndarray       # (m, q) float64
    psi_i: np.ndarray    # (d,) complex128
    psi_f: np.ndarray    # (d,) complex128
    T: float
    Nt: int
    N: int
    u0: np.ndarray       # (Nt, m) float64
    iters: int = 20
    rho: float = 0.1
    local_iters: int = 1
    precision: str = "mixed"
    kind: str = "pauli"
    objective: str = "overlap"
    alpha: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return 1 << self.q

    @property
    def m(self) -> int:
        return int(self.ax.shape[0])

    @property
    def tau(self) -> float:
        return self.T / self.Nt

    def with_(self, **kw) -> "MCWorkload":
        import dataclasses

        return dataclasses.replace(self, **kw)


def random_pauli(q: int, m: int, seed: int, *, T: float, Nt: int, N: int, u_amp: float = 1.0,
                 h0_scale: float = 2.0, name: str = "pauli") -> MCWorkload:
    """Random multi-control problem for parity tests.  Draws, in order: H0d ~ U[-h0_scale, h0_scale]
    (d), ax ~ U[-1, 1] (m x q), ay ~ U[-1, 1] (m x q), psi_i and psi_f (complex Gaussian, normalised),
    u0 ~ U[-u_amp, u_amp] (Nt x m)."""
    rng = np.random.default_rng(seed)
    d = 1 << q
    H0d = rng.uniform(-h0_scale, h0_scale, d)
    ax = rng.uniform(-1.0, 1.0, (m, q))
    ay = rng.uniform(-1.0, 1.0, (m, q))
    v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    f = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    u0 = rng.uniform(-u_amp, u_amp, (Nt, m))
    return MCWorkload(name=name, q=q, H0d=H0d, ax=ax, ay=ay, psi_i=v / np.linalg.norm(v), psi_f=f / np.linalg.norm(f),
                      T=T, Nt=Nt, N=N, u0=u0)


SPIN5_COUPLINGS = ((1, 2), (1, 3), (2, 3), (2, 5), (3, 4))


def spin5_liouville(seed: int = 1006, *, Nt: int = 32768, N: int = 128, Jp: float = 140.0,
                    T: Optional[float] = None, u_amp: Optional[float] = None, name: str = "spin5") -> MCWorkload:
    """The five-spin example of Sec. 4 in the density-matrix formalism, written as a state of the
    Liouville space: rho (32 x 32) <-> v[s + 32 s'] = rho[s, s'] (row index s on bits 0-4, column
    index s' on bits 5-9), i d rho/dt = [H, rho] <-> i dv/dt = (I (x) H - H^T (x) I) v.

    H = H0 + sum_k (u_x^k I_x^(k) + u_y^k I_y^(k)), I_a = sigma_a / 2 on spin k (spin k <-> bit k-1),
    H0 = 2 pi Jp sum_{(k,l)} I_z^(k) I_z^(l) over SPIN5_COUPLINGS (diagonal), so in Liouville space
    H0 -> E(s) - E(s') and the controls c = 0..4 (u_x^k) and 5..9 (u_y^k) act as
    u_x^k: (X on bit k-1 - X on bit k+4)/2,  u_y^k: (Y on bit k-1 + Y on bit k+4)/2
    (-H^T acts on the column index; X^T = X, Y^T = -Y).  rho(0) = I_x^(1), target I_x^(5), both
    normalised in the Frobenius norm, J = Re Tr(rho_f rho(T)).  T = 10/Jp (the paper prints "Jp/10";
    read as ten coupling periods), steps T/2^15; u0 ~ U[-u_amp, u_amp], u_amp = 2 pi Jp by default
    (the only random draw).  meta holds the Hilbert-space description for the density-matrix oracle."""
    rng = np.random.default_rng(seed)
    T = 10.0 / Jp if T is None else T
    u_amp = 2.0 * np.pi * Jp if u_amp is None else u_amp
    ns, q, m = 5, 10, 10
    s = np.arange(32)
    z = 1.0 - 2.0 * ((s[:, None] >> np.arange(ns)[None, :]) & 1)   # (32, 5): eigenvalues of sigma_z
    E = 2.0 * np.pi * Jp * sum(0.25 * z[:, k - 1] * z[:, l - 1] for k, l in SPIN5_COUPLINGS)
    e = np.arange(1024)
    row, col = e & 31, e >> 5
    H0d = E[row] - E[col]
    ax = np.zeros((m, q))
    ay = np.zeros((m, q))
    for k in range(1, ns + 1):
        ax[k - 1, k - 1], ax[k - 1, k + 4] = 0.5, -0.5
        ay[5 + k - 1, k - 1], ay[5 + k - 1, k + 4] = 0.5, 0.5
    rho0 = np.zeros(1024, dtype=np.complex128)
    rhof = np.zeros(1024, dtype=np.complex128)
    rho0[(row ^ 1) == col] = 0.5          # I_x^(1)[s, s'] = 1/2 for s' = s ^ bit 0
    rhof[(row ^ 16) == col] = 0.5         # I_x^(5): bit 4
    rho0 /= np.linalg.norm(rho0)
    rhof /= np.linalg.norm(rhof)
    u0 = rng.uniform(-u_amp, u_amp, (Nt, m))
    return MCWorkload(name=name, q=q, H0d=H0d, ax=ax, ay=ay, psi_i=rho0, psi_f=rhof, T=T, Nt=Nt, N=N, u0=u0,
                      meta={"spins": ns, "couplings": SPIN5_COUPLINGS, "Jp": Jp, "initial": ("x", 1), "target": ("x", 5)})
