"""Gross-Pitaevskii variant (Sec. 4, condensates; harmonic trap with shifted centre and the double well)
through the C ABI vs the FP64 oracle: forward and adjoint sweeps (psi(t_n), chi(t_n)), sub-problem
gradients, ISM iterations."""
import numpy as np
import pytest

import workloads as W
from oracle import gp_oracle as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1603_01237_gb300 as P

    return P


def _gp(n, Nt, N, T, seed=5, g=1.0, steps=4000):
    rng = np.random.default_rng(seed)
    psi_i, psi_f = W.gp_stationary_states(n, 20.0, -10.0, g, dt=2e-3, steps=steps)
    return W.GPWorkload(name=f"gp{n}", n=n, L=20.0, x_min=-10.0, g=g, psi_i=psi_i, psi_f=psi_f, T=T, Nt=Nt,
                        N=N, u0=rng.uniform(-0.5, 0.5, Nt))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _dw(n, Nt, N, T, seed=6, steps=4000):
    """Double well (Sec. 4): harmonic ground state -> ground state of the split trap, ramp + noise."""
    return W.gp_double_well(n=n, seed=seed, T=T, Nt=Nt, N=N, steps=steps, u_amp=0.3)


CASES = [("gp64", _gp(64, 150, 6, 1.5)), ("gp512", _gp(512, 240, 8, 2.0)), ("gp512-ragged", _gp(512, 157, 5, 1.0)),
         ("dw64", _dw(64, 150, 6, 1.5)), ("dw512", _dw(512, 240, 8, 2.0)), ("dw512-ragged", _dw(512, 157, 5, 1.0))]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 2e-5)])
def test_gp_intermediate_pairs(P, name, w, prec, tol):
    ps_o, ch_o = G.intermediate_pairs(w, w.u0)
    with P.Plan(w, precision=prec) as pl:
        phi = pl.intermediate_states(w.u0)[0]
    assert np.max(np.abs(phi[0] - ps_o)) <= tol, np.max(np.abs(phi[0] - ps_o))
    assert np.max(np.abs(phi[1] - ch_o)) <= tol, np.max(np.abs(phi[1] - ch_o))


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_gp_subinterval_grad(P, name, w, prec, tol):
    ps_o, ch_o = G.intermediate_pairs(w, w.u0)
    g_o, Jn_o = G.subinterval_all(w, ps_o, ch_o, w.u0)
    with P.Plan(w, precision=prec) as pl:
        g, Jn = pl.subinterval_grad(np.stack([ps_o, ch_o]), w.u0)
    assert rel(g[0], g_o) <= tol, rel(g[0], g_o)
    assert np.max(np.abs(Jn[0] - Jn_o)) <= tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_gp_iterate(P, prec, tol):
    w = _gp(512, 200, 8, 2.0)
    u_o, J_o, F_o, E_o = G.ism_solve(w, w.u0, 3, 0.5)
    with P.Plan(w, precision=prec, rho=0.5) as pl:
        u, J, E = pl.iterate(w.u0, 3)
        _, F = pl.evaluate(u[0])
    assert np.max(np.abs(J[0] - J_o)) <= tol, np.max(np.abs(J[0] - J_o))
    assert abs(F[0] - F_o[-1]) <= tol
    assert rel(E[0], E_o) <= (1e-4 if prec == "mixed" else 1e-9), rel(E[0], E_o)


def test_gp_n_independence(P):
    w = _gp(64, 120, 1, 1.0)
    res = []
    for N in (1, 4, 120):
        with P.Plan(w.with_(N=N), precision="fp64", rho=0.5) as pl:
            res.append(pl.iterate(w.u0, 2)[0][0])
    for u in res[1:]:
        assert np.max(np.abs(u - res[0])) <= 1e-11


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_double_well_iterate(P, prec, tol):
    w = _dw(512, 200, 8, 2.0)
    u_o, J_o, F_o, E_o = G.ism_solve(w, w.u0, 3, 0.05)
    with P.Plan(w, precision=prec, rho=0.05) as pl:
        u, J, E = pl.iterate(w.u0, 3)
        _, F = pl.evaluate(u[0])
    assert np.max(np.abs(J[0] - J_o)) <= tol, np.max(np.abs(J[0] - J_o))
    assert abs(F[0] - F_o[-1]) <= tol
    assert rel(E[0], E_o) <= (1e-4 if prec == "mixed" else 1e-9), rel(E[0], E_o)


def test_double_well_full_size_mixed(P):
    """The double-well problem at the condensate benchmark's size (512 points, Nt = 10000, N = 64),
    mixed precision, two ISM iterations and the global gradient against the FP64 oracle."""
    w = W.gp_double_well(n=512, Nt=10000, N=64, steps=20000)
    u_o, J_o, F_o, _ = G.ism_solve(w, w.u0, 2, 0.05)
    g_o = G.global_gradient(w, w.u0)
    with P.Plan(w, precision="mixed", rho=0.05) as pl:
        u, J, _ = pl.iterate(w.u0, 2)
        g, Jg = pl.gradient(w.u0)
    assert np.max(np.abs(J[0] - J_o)) <= 1e-5, np.max(np.abs(J[0] - J_o))
    assert rel(g[0], g_o) <= 1e-4, rel(g[0], g_o)
    assert np.max(np.abs(u[0] - u_o)) <= 1e-4 * np.max(np.abs(u_o))


@pytest.mark.parametrize("N", [1, 40])
def test_double_well_degenerate_partitions(P, N):
    """N = 1 and N = Nt for the double well (FP64)."""
    w = _dw(64, 40, N, 0.5)
    ps_o, ch_o = G.intermediate_pairs(w, w.u0)
    u_o, J_o, _, _ = G.ism_solve(w, w.u0, 2, 0.05)
    with P.Plan(w, precision="fp64", rho=0.05) as pl:
        phi = pl.intermediate_states(w.u0)[0]
        u, J, _ = pl.iterate(w.u0, 2)
    assert np.max(np.abs(phi[0] - ps_o)) <= 1e-11 and np.max(np.abs(phi[1] - ch_o)) <= 1e-11
    assert np.max(np.abs(J[0] - J_o)) <= 1e-10 and np.max(np.abs(u[0] - u_o)) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("S", [1, 4, 13, 1000])
def test_gp_checkpoints_change_nothing(P, prec, S):
    """ckpt_stride S > 0 keeps the forward states every S steps of each sub-interval and recomputes
    each S-step segment before its adjoint steps (the global adjoint sweep and the sub-problems):
    every result equals the whole-trajectory plan's bit for bit (the recomputation repeats the same
    steps from a stored copy of the same state).  Ragged partition (Nt = 157, N = 5: 31-32 steps,
    the last segment of each sub-interval shorter than S); S = 1000 is clamped to one segment per
    sub-interval."""
    w = _dw(512, 157, 5, 1.0)
    rng = np.random.default_rng(12)
    ps_o, ch_o = G.intermediate_pairs(w, w.u0)
    phi_in = np.stack([ps_o, ch_o]) * (1 + 1e-3 * rng.standard_normal((2,) + ps_o.shape))
    out = []
    for s in (0, S):
        with P.Plan(w, precision=prec, rho=0.05, ckpt_stride=s) as pl:
            assert pl.info(11) == (0 if s == 0 else min(s, 32))
            phi = pl.intermediate_states(w.u0)[0]
            g, Jn = pl.subinterval_grad(phi_in, w.u0)
            u, J, E = pl.iterate(w.u0, 3)
            gg, Jg = pl.gradient(u[0])
        out.append((phi, g, Jn, u, J, E, gg, Jg))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_gp_checkpoints_full_size_footprint_and_parity(P):
    """The condensate benchmark's size (512 points, Nt = 10000, N = 64) with ckpt_stride 13: under a
    quarter of the whole-trajectory plan's memory, the same iterates, and the oracle's to the mixed bar."""
    w = W.gp_double_well(n=512, Nt=10000, N=64, steps=20000)
    from paper_1603_01237_gb300 import abi

    f0 = abi.footprint(w, precision="mixed")
    f13 = abi.footprint(w, precision="mixed", ckpt_stride=13)
    assert f13 < 0.25 * f0
    u_o, J_o, _, _ = G.ism_solve(w, w.u0, 2, 0.05)
    with P.Plan(w, precision="mixed", rho=0.05, ckpt_stride=13) as pl:
        u, J, _ = pl.iterate(w.u0, 2)
    with P.Plan(w, precision="mixed", rho=0.05) as pl:
        u0_, J0_, _ = pl.iterate(w.u0, 2)
    assert np.array_equal(u, u0_) and np.array_equal(J, J0_)
    assert np.max(np.abs(J[0] - J_o)) <= 1e-5


def test_gp_batched_launches_match_single_problem_plans(P):
    """640 problems per plan (Nt = 40, N = 8): the FP32 sweeps then run the kernels compiled for ten
    (sequential sweeps) and eight (sub-problems) resident CTAs per SM, a one-problem plan the
    unbounded ones.  Same arithmetic: three problems' controls, J and Err after two iterations agree
    with their one-problem plans, and with the FP64 oracle to the mixed bar."""
    w = _gp(512, 40, 8, 0.5)
    B = 640
    rng = np.random.default_rng(21)
    U = w.u0[None, :] + 0.2 * rng.standard_normal((B, w.Nt))
    with P.Plan(w, precision="mixed", rho=0.5, batch=B) as pl:
        u, J, E = pl.iterate(U, 2)
    for b in (0, 317, B - 1):
        with P.Plan(w, precision="mixed", rho=0.5) as pl1:
            u1, J1, E1 = pl1.iterate(U[b], 2)
        assert np.max(np.abs(u[b] - u1[0])) <= 1e-12 * np.max(np.abs(u1[0])), np.max(np.abs(u[b] - u1[0]))
        assert np.max(np.abs(J[b] - J1[0])) <= 1e-12 and np.max(np.abs(E[b] - E1[0])) <= 1e-12 * np.max(E1[0])
        u_o, J_o, _, _ = G.ism_solve(w, U[b], 2, 0.5)
        assert np.max(np.abs(J[b] - J_o)) <= 1e-5, np.max(np.abs(J[b] - J_o))
        assert np.max(np.abs(u[b] - u_o)) <= 1e-4 * np.max(np.abs(u_o)), np.max(np.abs(u[b] - u_o))


@pytest.mark.parametrize("S", [0, 7])
def test_gp_first_local_step_equals_literal_subproblems(P, S):
    """A first local step starts every sub-problem from phi_n = psi(t_n) under the controls of the
    forward sweep, so `ism_iterate` takes the sub-problems' forward trajectories from that sweep (or
    its checkpoints, S > 0) and runs only their adjoints.  In FP64 the update equals the literal
    sub-problems' (`subinterval_grad` at the sweep's own phi, forward propagated from phi_n) to
    rounding: u + rho g / tau, and Err = sum_j |g_j| per sub-interval."""
    w = _dw(512, 157, 5, 1.0)
    rho, tau = 0.05, w.T / w.Nt
    with P.Plan(w, precision="fp64", rho=rho, ckpt_stride=S) as pl:
        phi = pl.intermediate_states(w.u0)[0]
        g, Jn = pl.subinterval_grad(phi, w.u0)
        u1, J, E = pl.iterate(w.u0, 1)
    assert np.max(np.abs(u1[0] - (w.u0 + rho * g[0] / tau))) <= 1e-10 * np.max(np.abs(w.u0))
    assert abs(E[0, 0] - np.sum(np.abs(g[0]))) <= 1e-10 * np.sum(np.abs(g[0]))
