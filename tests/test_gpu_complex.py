"""Complex Hermitian H0, H1 (the dense kind with imaginary parts) through the C ABI against the FP64
oracle.  Sec. 2 states the control problem for any Hermitian H0, H1, and the gradient Im<chi|H1|psi>
of Eq. (gradJ) needs no change for complex H1.  The cases cover every lane layout of the dense
kernels (d = 5, 24, 41, 64: one to four elements per lane), both objectives and both precisions,
the assembly + chain route, direct sweeps and the blocked chain, the allocation-free entry point and
the serving loop.  Tolerances are those of the real dense kind.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ism_oracle as O

pytestmark = pytest.mark.gpu

FP64_PHI, FP64_GRAD = 1e-11, 1e-10
MIX_PHI, MIX_GRAD = 2e-5, 1e-4


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1603_01237_gb300 as P

    return P


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


CASES = [
    ("herm5-fp64", W.random_hermitian(5, 81, T=2.0, Nt=203, N=6), "fp64"),
    ("herm24-obs-fp64", W.random_hermitian(24, 82, T=2.0, Nt=150, N=9, objective="observable"), "fp64"),
    ("herm41-mixed", W.random_hermitian(41, 83, T=2.0, Nt=300, N=10), "mixed"),
    ("herm64-fp64", W.random_hermitian(64, 84, T=2.0, Nt=120, N=5), "fp64"),
    ("herm16-mixed", W.random_hermitian(16, 85, T=2.0, Nt=300, N=10), "mixed"),
]


@pytest.mark.parametrize("name,w,prec", CASES, ids=[c[0] for c in CASES])
def test_intermediate_states_and_objective(P, name, w, prec):
    phi_o = O.intermediate_states(w, w.u0)
    Jo, Fo = O.objective(w, w.u0)
    with P.Plan(w, precision=prec) as pl:
        phi = pl.intermediate_states(w.u0)[0]
        J, F = pl.evaluate(w.u0)
    tol = FP64_PHI if prec == "fp64" else MIX_PHI
    assert np.max(np.abs(phi - phi_o)) <= tol, np.max(np.abs(phi - phi_o))
    assert np.array_equal(phi[0], phi_o[0])
    assert abs(J[0] - Jo) <= (1e-11 if prec == "fp64" else 2e-5)
    assert abs(F[0] - Fo) <= (1e-11 if prec == "fp64" else 2e-5)


@pytest.mark.parametrize("name,w,prec", CASES, ids=[c[0] for c in CASES])
def test_subinterval_grad(P, name, w, prec):
    phi_o = O.intermediate_states(w, w.u0)
    g_o, Jn_o = O.subinterval_all(w, phi_o, w.u0)
    with P.Plan(w, precision=prec) as pl:
        g, Jn = pl.subinterval_grad(phi_o, w.u0)
    assert rel_l2(g[0], g_o) <= (FP64_GRAD if prec == "fp64" else MIX_GRAD), rel_l2(g[0], g_o)
    jt = 1e-12 if prec == "fp64" else 1e-5
    assert np.max(np.abs(Jn[0] - Jn_o)) <= jt * max(1.0, np.abs(Jn_o).max())


@pytest.mark.parametrize("name,w,prec", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_iterate_matches_algorithm1(P, name, w, prec):
    iters = 3
    u_o, J_o, F_o, E_o = O.ism_solve(w, w.u0, iters, w.rho)
    with P.Plan(w, precision=prec) as pl:
        u, J, E = pl.iterate(w.u0, iters)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert np.max(np.abs(J[0] - J_o)) <= tol
    assert rel_l2(u[0] - w.u0, u_o - w.u0) <= tol
    assert rel_l2(E[0], E_o) <= tol


@pytest.mark.parametrize("name,w,prec", [CASES[1], CASES[4]], ids=[CASES[1][0], CASES[4][0]])
def test_direct_sweeps(P, name, w, prec):
    """step1 = 2: psi(t_n), chi(t_n) by direct propagation, and the iterate that follows."""
    phi_o = O.intermediate_states(w, w.u0)
    u_o, J_o, _, _ = O.ism_solve(w, w.u0, 2, w.rho)
    with P.Plan(w, precision=prec, step1=2) as pl:
        assert pl.info(6) == 2
        phi = pl.intermediate_states(w.u0)[0]
        u, J, _ = pl.iterate(w.u0, 2)
    assert np.max(np.abs(phi - phi_o)) <= (FP64_PHI if prec == "fp64" else MIX_PHI)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert np.max(np.abs(J[0] - J_o)) <= tol
    assert rel_l2(u[0] - w.u0, u_o - w.u0) <= tol


def test_blocked_chain(P):
    """N = 37 sub-intervals: the chain over blocks of propagators."""
    w = W.random_hermitian(16, 86, T=2.0, Nt=370, N=37)
    phi_o = O.intermediate_states(w, w.u0)
    with P.Plan(w, precision="fp64") as pl:
        assert pl.info(7) > 1
        phi = pl.intermediate_states(w.u0)[0]
    assert np.max(np.abs(phi - phi_o)) <= FP64_PHI


def test_gauge_rotated_problem_gives_the_real_problems_results(P):
    """A real symmetric problem and its basis-rotated complex Hermitian copy (H -> D H D^H, psi -> D psi)
    give the same objective and gradient, through the real and the complex kernels."""
    w = W.random_dense(24, 87, T=2.0, Nt=200, N=8)
    wc = W.gauge(w, np.random.default_rng(88).uniform(0, 2 * np.pi, w.d))
    with P.Plan(w, precision="fp64") as pl:
        g, J = pl.gradient(w.u0)
    with P.Plan(wc, precision="fp64") as pl:
        gc, Jc = pl.gradient(w.u0)
    assert abs(J[0] - Jc[0]) <= 1e-12
    assert rel_l2(gc, g) <= 1e-10


def test_noalloc_and_server_take_the_imaginary_parts(P):
    """The allocation-free entry point equals the planned call bit for bit on a complex problem, and a
    complex request through the serving loop equals the same plan run alone."""
    import torch

    from paper_1603_01237_gb300 import abi

    w = W.random_hermitian(24, 89, T=2.0, Nt=240, N=8)
    phi = O.intermediate_states(w, w.u0)
    phi_d = torch.tensor(phi.view(np.float64), device="cuda")
    u_d = torch.tensor(w.u0, dtype=torch.float64, device="cuda")
    with P.Plan(w, precision="fp64") as pl:
        g_ref = torch.empty((1, w.Nt), dtype=torch.float64, device="cuda")
        J_ref = torch.empty((1, w.N), dtype=torch.float64, device="cuda")
        pl.ism_subinterval_grad(phi_d, u_d, g_ref, J_ref)
        u1, J1, _ = pl.iterate(w.u0, 3)
    g = torch.full((1, w.Nt), float("nan"), dtype=torch.float64, device="cuda")
    J = torch.full((1, w.N), float("nan"), dtype=torch.float64, device="cuda")
    abi.subinterval_grad_noalloc(w, "fp64", phi_d, u_d, g, J)
    assert torch.equal(g, g_ref) and torch.equal(J, J_ref)
    g_o, _ = O.subinterval_all(w, phi, w.u0)
    assert rel_l2(g.cpu().numpy()[0], g_o) <= FP64_GRAD
    with P.Server(slots=1, hbm_budget_bytes=4 << 30) as srv:
        u2, J2, _ = srv.result(srv.submit(w, iters=3, precision="fp64"))
    assert np.array_equal(u2, u1) and np.array_equal(J2, J1)


def test_checkpoint_stride_changes_nothing(P):
    w = CASES[4][1]
    phi_o = O.intermediate_states(w, w.u0)
    res = []
    for S in (1, 6, 0, 10 ** 6):
        with P.Plan(w, precision="mixed", ckpt_stride=S) as pl:
            res.append(pl.subinterval_grad(phi_o, w.u0))
    for g, Jn in res[1:]:
        assert np.array_equal(g, res[0][0]) and np.array_equal(Jn, res[0][1])
