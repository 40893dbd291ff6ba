"""Dense d = 128 and 256 on the tensor cores (tcgen05, TF32 x 3 split operands, FP32 accumulators):
the stacked global sweeps of Algorithm 1 (a)-(b) and the stacked two-trajectory sub-problems of step
(c) against the FP64 oracle on random real-symmetric H0, H1, at the mixed-precision bars (states 2e-5,
gradient relative L2 1e-4, J 1e-5 per iteration on these fine steps), batched and with ragged
partitions; and the requests these plans refuse."""
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


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


CASES = [
    ("dense128", W.random_dense(128, 301, T=2.0, Nt=160, N=4)),
    ("dense128-ragged-obs", W.random_dense(128, 302, T=2.0, Nt=157, N=6, objective="observable")),
    ("dense256", W.random_dense(256, 303, T=1.5, Nt=120, N=3)),
]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_tc_intermediate_states_and_gradient(P, name, w):
    phi_o = O.intermediate_states(w, w.u0)
    g_o = O.global_gradient(w, w.u0)
    J_o, _ = O.objective(w, w.u0)
    with P.Plan(w, precision="mixed") as pl:
        assert pl.info(10) == 1                      # the tensor-core path
        phi = pl.intermediate_states(w.u0)[0]
        g, J = pl.gradient(w.u0)
    assert np.max(np.abs(phi - phi_o)) <= 2e-5, np.max(np.abs(phi - phi_o))
    assert np.array_equal(phi[0], phi_o[0])
    assert rel(g[0], g_o) <= 1e-4, rel(g[0], g_o)
    assert abs(J[0] - J_o) <= 1e-5, abs(J[0] - J_o)


@pytest.mark.parametrize("name,w", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_tc_iterate_matches_algorithm1(P, name, w):
    iters = 3
    u_o, J_o, F_o, E_o = O.ism_solve(w, w.u0, iters, 0.5)
    with P.Plan(w, precision="mixed", rho=0.5) as pl:
        u, J, E = pl.iterate(w.u0, iters)
    assert np.max(np.abs(J[0] - J_o)) <= 1e-5, np.max(np.abs(J[0] - J_o))
    assert rel(u[0] - w.u0, u_o - w.u0) <= 1e-4
    assert rel(E[0], E_o) <= 1e-4


def test_tc_batch_equals_single_problems(P):
    """Three problems with different controls in one plan (states of different problems stacked in
    the same tensor-core tiles) agree with their own one-problem plans and with the oracle."""
    w = CASES[0][1]
    rng = np.random.default_rng(9)
    U = np.stack([w.u0] + [rng.uniform(-0.5, 0.5, w.Nt) for _ in range(2)])
    with P.Plan(w, precision="mixed", batch=3) as pl:
        gB, JB = pl.gradient(U)
    for b in range(3):
        with P.Plan(w, precision="mixed") as p1:
            g1, J1 = p1.gradient(U[b])
        assert np.array_equal(gB[b], g1[0]) and JB[b] == J1[0]   # a column's arithmetic ignores its neighbours
        assert rel(gB[b], O.global_gradient(w, U[b])) <= 1e-4


def test_tc_refusals(P):
    from paper_1603_01237_gb300 import abi

    w = CASES[0][1]
    with pytest.raises(abi.IsmError) as ei:
        P.Plan(w, precision="fp64")
    assert ei.value.status == abi.ISM_EUNSUPPORTED
    with pytest.raises(abi.IsmError) as ei:
        P.Plan(w, precision="mixed", local_iters=2)
    assert ei.value.status == abi.ISM_EUNSUPPORTED
    with P.Plan(w, precision="mixed") as pl:
        phi = pl.intermediate_states(w.u0)
        with pytest.raises(abi.IsmError) as ei:
            pl.subinterval_grad(phi, w.u0)
        assert ei.value.status == abi.ISM_EUNSUPPORTED
