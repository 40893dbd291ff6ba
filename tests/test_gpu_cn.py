"""Crank-Nicolson plans (the time step of Sec. 3) through the C ABI vs the Crank-Nicolson oracle on
identical seeded inputs, FP64, for the tridiagonal, bit-flip and dense kinds: intermediate states
by both step-1 paths (assembly + chain, plain and
blocked; direct sweeps), sub-problem gradients and J_n, Algorithm 1 iterations, the global gradient
(Theorem 2 form), and the plan's errors for controls beyond the Jacobi solve's range.

Tolerances are those of the FP64 Chebyshev plans: the Jacobi solve stops at rho^K <= 1e-17 per step,
so the two sides differ by rounding alone."""
import numpy as np
import pytest

import workloads as W
from oracle import cn_oracle as C

pytestmark = pytest.mark.gpu

PHI = 1e-11
GRAD = 1e-10


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1603_01237_gb300 as P

    return P


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _band(A):
    return np.triu(np.tril(A, 1), -1)


def _strong(d, seed, *, T, Nt, N, objective="overlap", h1diag=False, scale=15.0):
    """Random tridiagonal H0 (with off-diagonal) and H1, scaled up: the Jacobi solve of each step
    takes many iterations (rho ~ 0.1-0.3)."""
    w = W.random_dense(d, seed, T=T, Nt=Nt, N=N, objective=objective, u_amp=1.0)
    H1 = _band(w.H1) if h1diag else _band(w.H1) - np.diag(np.diag(w.H1))
    return w.with_(kind="tridiag", H0=scale * _band(w.H0), H1=scale * H1)


def _rho(w):
    off = lambda A: np.max(np.abs(A - np.diag(np.diag(A))).sum(axis=1))
    return 0.5 * w.T / w.Nt * (off(w.H0) + np.max(np.abs(w.u0)) * off(w.H1))


def _h1_diagonal(w, seed):
    rng = np.random.default_rng(seed)
    return w.with_(H1=w.H1 + np.diag(rng.uniform(-0.3, 0.3, w.d)))


CASES = [
    ("rotor41", W.config("rotor41", Nt=1000, N=16, precision="fp64")),
    ("rotor41-overlap-ragged", W.rotor(40, 5, T=np.pi, Nt=801, N=11, objective="overlap")),
    ("rotor41-h1diag", _h1_diagonal(W.config("rotor41", Nt=600, N=6, precision="fp64"), 21)),
    ("strong12", _strong(12, 71, T=2.0, Nt=120, N=7)),
    ("strong33-h1diag-obs", _strong(33, 72, T=2.0, Nt=150, N=9, objective="observable", h1diag=True)),
    ("tridiag2", W.rabi(0.7, 0.3, T=3.0, Nt=64, N=8).with_(kind="tridiag")),
    # the bit-flip and dense kinds (spin models, generic H)
    ("spin16", W.config("spin16", Nt=400, N=4)),
    ("bitflip64-ragged", W.with_random_target(W.spin_chain(6, 67, T=2.0, Nt=201, N=7, u_amp=1.5), 3)),
    ("bitflip2", W.with_random_target(W.spin_all_to_all(1, 5, T=3.0, Nt=64, N=4, u_amp=1.5), 1)),
    ("dense5", W.random_dense(5, 61, T=2.0, Nt=203, N=6)),
    ("dense41-obs", W.random_dense(41, 62, T=2.0, Nt=150, N=9, objective="observable")),
    ("dense64", W.random_dense(64, 63, T=2.0, Nt=120, N=5)),
]
IDS = [c[0] for c in CASES]


def test_strong_cases_exercise_the_jacobi_solve():
    assert 0.05 < _rho(CASES[3][1]) < 0.5
    assert 0.05 < _rho(CASES[4][1]) < 0.5


@pytest.mark.parametrize("step1", [1, 2])
@pytest.mark.parametrize("name,w", CASES, ids=IDS)
def test_cn_intermediate_states(P, name, w, step1):
    phi_o = C.intermediate_states(w, w.u0)
    with P.Plan(w, precision="fp64", scheme="crank_nicolson", step1=step1) as pl:
        assert pl.info(8) == 1 and pl.info(6) == step1
        phi = pl.intermediate_states(w.u0)[0]
    assert np.max(np.abs(phi - phi_o)) <= PHI, np.max(np.abs(phi - phi_o))
    assert np.array_equal(phi[0], phi_o[0])


@pytest.mark.parametrize("name,w", CASES, ids=IDS)
def test_cn_subinterval_grad(P, name, w):
    phi_o = C.intermediate_states(w, w.u0)
    g_o, Jn_o = C.subinterval_all(w, phi_o, w.u0)
    with P.Plan(w, precision="fp64", scheme="crank_nicolson") as pl:
        g, Jn = pl.subinterval_grad(phi_o, w.u0)
    assert rel_l2(g[0], g_o) <= GRAD, rel_l2(g[0], g_o)
    assert np.max(np.abs(Jn[0] - Jn_o)) <= 1e-12 * max(1.0, np.abs(Jn_o).max())


ITER = [CASES[i] for i in (0, 1, 2, 3, 6, 9)]


@pytest.mark.parametrize("step1", [1, 2])
@pytest.mark.parametrize("name,w", ITER, ids=[c[0] for c in ITER])
def test_cn_iterate_matches_algorithm1(P, name, w, step1):
    iters = 3
    u_o, J_o, F_o, E_o = C.ism_solve(w, w.u0, iters, w.rho)
    with P.Plan(w, precision="fp64", scheme="crank_nicolson", step1=step1) as pl:
        u, J, E = pl.iterate(w.u0, iters)
        Jf, Ff = pl.evaluate(u[0])
    assert np.max(np.abs(J[0] - J_o)) <= 1e-9
    assert abs(Ff[0] - F_o[-1]) <= 1e-9
    assert rel_l2(u[0] - w.u0, u_o - w.u0) <= 1e-9
    assert rel_l2(E[0], E_o) <= 1e-9


@pytest.mark.parametrize("name,w", [CASES[0], CASES[3]], ids=[IDS[0], IDS[3]])
def test_cn_local_iterations_and_theorem2_form(P, name, w):
    """L = 2 local steps (the second from the moved controls), and the Theorem 2 two-trajectory
    form of the first step, which equals the literal sub-problem at phi = phi^u."""
    u_o, J_o, _, _ = C.ism_solve(w, w.u0, 2, w.rho, L=2)
    with P.Plan(w, precision="fp64", scheme="crank_nicolson", local_iters=2) as pl:
        u, J, _ = pl.iterate(w.u0, 2)
    assert np.max(np.abs(J[0] - J_o)) <= 1e-9
    assert rel_l2(u[0] - w.u0, u_o - w.u0) <= 1e-9
    u_l, J_l, _, _ = C.ism_solve(w, w.u0, 2, w.rho)
    with P.Plan(w, precision="fp64", scheme="crank_nicolson", subproblem_form=2) as pl:
        u2, J2, _ = pl.iterate(w.u0, 2)
    assert np.max(np.abs(J2[0] - J_l)) <= 1e-9
    assert rel_l2(u2[0] - w.u0, u_l - w.u0) <= 1e-9


@pytest.mark.parametrize("step1", [1, 2])
@pytest.mark.parametrize("name,w", CASES, ids=IDS)
def test_cn_global_gradient(P, name, w, step1):
    g_o = C.global_gradient(w, w.u0)
    J_o, F_o = C.objective(w, w.u0)
    with P.Plan(w, precision="fp64", scheme="crank_nicolson", step1=step1) as pl:
        g, J = pl.gradient(w.u0)
        Je, Fe = pl.evaluate(w.u0)
    assert rel_l2(g[0], g_o) <= GRAD, rel_l2(g[0], g_o)
    assert abs(J[0] - J_o) <= 1e-12 and abs(Je[0] - J_o) <= 1e-12 and abs(Fe[0] - F_o) <= 1e-12


def test_cn_blocked_chain(P):
    """N = 64 sub-intervals: the chain runs over products of 8 consecutive propagators."""
    w = W.config("rotor41", Nt=1600, N=64, precision="fp64")
    phi_o = C.intermediate_states(w, w.u0)
    with P.Plan(w, precision="fp64", scheme="crank_nicolson", step1=1) as pl:
        assert pl.info(7) > 1
        phi = pl.intermediate_states(w.u0)[0]
    assert np.max(np.abs(phi - phi_o)) <= PHI


def test_cn_batch_equals_singles_and_differs_from_chebyshev(P):
    """A batch of 3 problems with different controls (direct sweeps when forced) equals three single
    plans; the Crank-Nicolson J differs from the Chebyshev (exact-step) J by the scheme's O(tau^2)."""
    w = W.config("rotor41", Nt=400, N=8, precision="fp64")
    rng = np.random.default_rng(5)
    U = rng.uniform(-1, 1, (3, w.Nt))
    with P.Plan(w, precision="fp64", scheme="crank_nicolson", batch=3, step1=2) as pl:
        Jb, _ = pl.evaluate(U)
        gb, _ = pl.gradient(U)
    for b in range(3):
        with P.Plan(w, precision="fp64", scheme="crank_nicolson") as pl:
            J1, _ = pl.evaluate(U[b])
            g1, _ = pl.gradient(U[b])
        assert abs(J1[0] - Jb[b]) <= 1e-13
        assert rel_l2(gb[b], g1[0]) <= 1e-11
        assert abs(J1[0] - C.objective(w, U[b])[0]) <= 1e-12
    with P.Plan(w, precision="fp64") as pl:
        Jc, _ = pl.evaluate(U[0])
    Jcn = C.objective(w, U[0])[0]
    assert 1e-9 < abs(Jc[0] - Jcn) < 1e-2


def test_cn_controls_beyond_the_solve_are_rejected(P):
    """Controls with (tau/2)(off-diagonal row sum) >= 1/2 make the plan fail with ISM_EUNSUPPORTED;
    the launch itself runs its capped iteration count and the plan stays usable."""
    w = _strong(12, 71, T=2.0, Nt=120, N=7)
    big = np.full(w.Nt, 20.0)
    with P.Plan(w, precision="fp64", scheme="crank_nicolson") as pl:
        with pytest.raises(P.IsmError) as ei:
            pl.evaluate(big)
        assert ei.value.status == 6
        J, _ = pl.evaluate(w.u0)
    assert abs(J[0] - C.objective(w, w.u0)[0]) <= 1e-12


@pytest.mark.parametrize("step1", [1, 2])
@pytest.mark.parametrize("N", [1, 24])
def test_cn_degenerate_partitions(P, N, step1):
    """N = 1 (no decomposition) and N = Nt (one step per sub-interval)."""
    w = _strong(12, 73, T=0.5, Nt=24, N=N)
    phi_o = C.intermediate_states(w, w.u0)
    g_o, Jn_o = C.subinterval_all(w, phi_o, w.u0)
    u_o, J_o, _, _ = C.ism_solve(w, w.u0, 2, 0.3)
    with P.Plan(w, precision="fp64", scheme="crank_nicolson", step1=step1, rho=0.3) as pl:
        phi = pl.intermediate_states(w.u0)[0]
        g, Jn = pl.subinterval_grad(phi_o, w.u0)
        u, J, _ = pl.iterate(w.u0, 2)
    assert np.max(np.abs(phi - phi_o)) <= PHI
    assert rel_l2(g[0], g_o) <= GRAD and np.max(np.abs(Jn[0] - Jn_o)) <= 1e-12
    assert np.max(np.abs(J[0] - J_o)) <= 1e-9 and rel_l2(u[0] - w.u0, u_o - w.u0) <= 1e-9


# ---------------------------------------------------------------- mixed precision (FP32 propagation)
MIXED = [
    ("rotor41", W.config("rotor41", Nt=1000, N=16, precision="fp64")),
    ("strong12", _strong(12, 71, T=2.0, Nt=120, N=7)),
    ("strong33-h1diag-obs", _strong(33, 72, T=2.0, Nt=150, N=9, objective="observable", h1diag=True)),
    ("spin16", W.config("spin16", Nt=400, N=4)),
    ("dense41-obs", W.random_dense(41, 62, T=2.0, Nt=150, N=9, objective="observable")),
]


@pytest.mark.parametrize("step1", [1, 2])
@pytest.mark.parametrize("name,w", MIXED, ids=[c[0] for c in MIXED])
def test_cn_mixed_states_gradient_iterate(P, name, w, step1):
    """FP32 propagation with FP64 states at the partition, overlaps and update: the mixed tolerances
    (states 2e-5, gradient relative 1e-4, J 1e-5)."""
    phi_o = C.intermediate_states(w, w.u0)
    g_o = C.global_gradient(w, w.u0)
    u_o, J_o, _, _ = C.ism_solve(w, w.u0, 2, w.rho)
    with P.Plan(w, precision="mixed", scheme="crank_nicolson", step1=step1) as pl:
        assert pl.info(8) == 1
        phi = pl.intermediate_states(w.u0)[0]
        g, _ = pl.gradient(w.u0)
        u, J, _ = pl.iterate(w.u0, 2)
    assert np.max(np.abs(phi - phi_o)) <= 2e-5, np.max(np.abs(phi - phi_o))
    assert rel_l2(g[0], g_o) <= 1e-4, rel_l2(g[0], g_o)
    assert np.max(np.abs(J[0] - J_o)) <= 1e-5, np.max(np.abs(J[0] - J_o))
    assert rel_l2(u[0] - w.u0, u_o - w.u0) <= 1e-4


def test_cn_mixed_rotor_full_size(P):
    """The rotor at the benchmark's size (Nt = 20000, N = 128) with the FP32 Crank-Nicolson step: J and
    the gradient at u0 against the FP64 Crank-Nicolson oracle, batched direct sweeps and one problem.
    J meets the mixed bar (1e-5) and the gradient the 1e-4 relative one: tau H_ee / 2 and the Jacobi
    diagonal inverse are formed in FP64 and carried as hi + lo pairs, since their FP32 roundings would
    repeat at every one of the 2 x 20000 global steps (plain FP32 coefficients leave 3e-4 here)."""
    w = W.config("rotor41", precision="fp64")
    J_o, F_o = C.objective(w, w.u0)
    g_o = C.global_gradient(w, w.u0)
    for batch in (1, 96):
        with P.Plan(w, precision="mixed", scheme="crank_nicolson", batch=batch) as pl:
            J, F = pl.evaluate(np.broadcast_to(w.u0, (batch, w.Nt)))
            g, _ = pl.gradient(np.broadcast_to(w.u0, (batch, w.Nt)))
        assert np.max(np.abs(J - J_o)) <= 1e-5 and np.max(np.abs(F - F_o)) <= 1e-5
        err = max(rel_l2(g[b], g_o) for b in range(batch))
        assert err <= 1e-4, err
