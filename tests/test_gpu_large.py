"""Spin chains of 7 to 10 sites (d = 128 .. 1024): one state per CTA, direct global sweeps.

The CUDA path is compared with the FP64 oracle on the same seeded inputs, with the tolerances of the
small-d cases: FP64 |dJ| <= 1e-9 and element bounds on states and gradients; mixed gradient relative
L2 <= 1e-4.  Sizes span every warp count compiled (1, 2, 4, 8 warps per state), ragged partitions,
both objectives, both sub-problem forms and batches.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ism_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1603_01237_gb300 as P

    return P


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _random_target(w, seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(w.d) + 1j * rng.standard_normal(w.d)
    return w.with_(psi_f=v / np.linalg.norm(v))


def _magnetisation(w):
    """O = (1/q) sum_i Z_i, diagonal and real."""
    q = int(np.log2(w.d))
    s = np.arange(w.d)
    z = 1.0 - 2.0 * ((s[:, None] >> np.arange(q)[None, :]) & 1)
    return w.with_(objective="observable", O=np.diag(z.mean(axis=1)), psi_f=None)


CASES = [
    ("chain7-fp64", _random_target(W.spin_chain(7, 81, T=1.0, Nt=160, N=8, u_amp=1.0), 11), "fp64"),
    ("chain8-mixed", _random_target(W.spin_chain(8, 82, T=1.0, Nt=240, N=6, u_amp=1.0), 12), "mixed"),
    ("chain9-ragged-fp64", _random_target(W.spin_chain(9, 83, T=1.0, Nt=203, N=7, u_amp=1.0), 13), "fp64"),
    ("chain10-mixed", _random_target(W.spin_chain(10, 84, T=1.0, Nt=200, N=8, u_amp=1.0), 14), "mixed"),
    ("chain10-fp64", _random_target(W.spin_chain(10, 85, T=0.5, Nt=100, N=5, u_amp=1.0), 15), "fp64"),
    ("chain7-obs-fp64", _magnetisation(W.spin_chain(7, 86, T=1.0, Nt=150, N=5, u_amp=1.0)), "fp64"),
    ("chain8-obs-mixed", _magnetisation(W.spin_chain(8, 87, T=1.0, Nt=150, N=5, u_amp=1.0)), "mixed"),
    ("chain10-obs-mixed", _magnetisation(W.spin_chain(10, 90, T=0.5, Nt=120, N=5, u_amp=1.0)), "mixed"),
]
IDS = [c[0] for c in CASES]
TOL = {"fp64": dict(phi=1e-11, grad=1e-10, J=1e-11), "mixed": dict(phi=2e-5, grad=1e-4, J=1e-6)}


@pytest.mark.parametrize("name,w,prec", CASES, ids=IDS)
def test_intermediate_states_large(P, name, w, prec):
    phi_o = O.intermediate_states(w, w.u0)
    with P.Plan(w, precision=prec) as pl:
        phi = pl.intermediate_states(w.u0)[0]
        J, F = pl.evaluate(w.u0)
    assert np.max(np.abs(phi - phi_o)) <= TOL[prec]["phi"], np.max(np.abs(phi - phi_o))
    assert np.array_equal(phi[0], phi_o[0])
    Jo, Fo = O.objective(w, w.u0)
    assert abs(J[0] - Jo) <= TOL[prec]["phi"]
    assert abs(F[0] - Fo) <= TOL[prec]["phi"]


@pytest.mark.parametrize("name,w,prec", CASES, ids=IDS)
def test_subinterval_grad_large(P, name, w, prec):
    phi_o = O.intermediate_states(w, w.u0)
    g_o, Jn_o = O.subinterval_all(w, phi_o, w.u0)
    with P.Plan(w, precision=prec) as pl:
        g, Jn = pl.subinterval_grad(phi_o, w.u0)
    assert rel_l2(g[0], g_o) <= TOL[prec]["grad"], rel_l2(g[0], g_o)
    assert np.max(np.abs(Jn[0] - Jn_o)) <= TOL[prec]["J"] * max(1.0, np.abs(Jn_o).max())


@pytest.mark.parametrize("name,w,prec", CASES, ids=IDS)
def test_iterate_large(P, name, w, prec):
    """Algorithm 1, two outer iterations; mixed runs the Theorem 2 form, FP64 the literal form."""
    iters = 2
    rho = 0.5
    u_o, J_o, F_o, E_o = O.ism_solve(w, w.u0, iters, rho)
    with P.Plan(w, precision=prec, rho=rho) as pl:
        u, J, E = pl.iterate(w.u0, iters)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert np.max(np.abs(J[0] - J_o)) <= (1e-9 if prec == "fp64" else 2e-5)
    assert rel_l2(u[0] - w.u0, u_o - w.u0) <= tol
    assert rel_l2(E[0], E_o) <= tol


def test_large_batch_equals_singles(P):
    w = _random_target(W.spin_chain(9, 88, T=1.0, Nt=120, N=4, u_amp=1.0), 16)
    rng = np.random.default_rng(9)
    U = np.stack([w.u0, rng.uniform(-1, 1, w.Nt)])
    with P.Plan(w, precision="mixed", batch=2) as pl:
        ub, Jb, Eb = pl.iterate(U, 2)
    for b in range(2):
        with P.Plan(w, precision="mixed") as pl:
            u1, J1, E1 = pl.iterate(U[b], 2)
        assert np.array_equal(ub[b], u1[0])
        assert np.array_equal(Jb[b], J1[0])


def test_large_forms_agree_fp64(P):
    """Theorem 2: the two-trajectory form and the literal phi-form give the same first step."""
    w = _random_target(W.spin_chain(8, 89, T=1.0, Nt=160, N=8, u_amp=1.0), 17)
    res = []
    for form in (1, 2):
        with P.Plan(w, precision="fp64", subproblem_form=form) as pl:
            res.append(pl.iterate(w.u0, 1)[0][0])
    assert np.max(np.abs(res[0] - res[1])) <= 1e-12


def test_ising1024_mixed_sampled_full_length(P):
    """The 10-spin chain at the benchmark's step size (tau = 2e-4) over a reduced horizon (Nt = 2000,
    N = 16): intermediate states and the sub-interval gradient at u0 against the oracle."""
    w = W.config("ising1024", Nt=2000, N=16)
    w = _random_target(w.with_(T=2000 * 2e-4), 18)
    phi_o = O.intermediate_states(w, w.u0)
    g_o, _ = O.subinterval_all(w, phi_o, w.u0)
    with P.Plan(w, precision="mixed") as pl:
        phi = pl.intermediate_states(w.u0)[0]
        g, _ = pl.subinterval_grad(phi_o, w.u0)
    assert np.max(np.abs(phi - phi_o)) <= 2e-5
    assert rel_l2(g[0], g_o) <= 1e-4



@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_large_checkpoint_stride_changes_nothing(P, prec):
    """CTA-wide literal sub-problems (d = 512, ragged): the stored states every S steps and the
    recomputed segments give the same gradient and J_n bit for bit for every stride, and the oracle's."""
    w = _random_target(W.spin_chain(9, 92, T=1.0, Nt=203, N=7, u_amp=1.0), 22)
    phi_o = O.intermediate_states(w, w.u0)
    g_o, _ = O.subinterval_all(w, phi_o, w.u0)
    res = []
    for S in (1, 5, 0, 10 ** 6):
        with P.Plan(w, precision=prec, ckpt_stride=S) as pl:
            res.append(pl.subinterval_grad(phi_o, w.u0))
    for g, Jn in res[1:]:
        assert np.array_equal(g, res[0][0]) and np.array_equal(Jn, res[0][1])
    assert rel_l2(res[0][0][0], g_o) <= TOL[prec]["grad"]
