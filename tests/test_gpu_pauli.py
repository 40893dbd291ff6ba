"""Several controls on a Pauli structure (the five-spin example of Sec. 4 in Liouville space) through
the C ABI vs the several-control oracle: intermediate states, sub-problem gradients of every control,
Algorithm 1 iterations and the global gradient on random problems (FP64 and mixed), and the five-spin
problem at the paper's size (2^15 steps) against the density-matrix form of the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import mc_oracle as M

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-11, 1e-10, 1e-9), "mixed": (2e-5, 1e-4, 1e-5)}   # states, gradient (rel L2), J


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1603_01237_gb300 as P

    return P


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


CASES = [
    ("q7-m3", W.random_pauli(7, 3, 31, T=1.0, Nt=120, N=6)),
    ("q8-m2-ragged", W.random_pauli(8, 2, 32, T=1.0, Nt=101, N=7)),
    ("q10-m4", W.random_pauli(10, 4, 33, T=0.6, Nt=80, N=4)),
]
IDS = [c[0] for c in CASES]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,w", CASES, ids=IDS)
def test_pauli_intermediate_states(P, name, w, prec):
    phi_o = M.intermediate_states(w, w.u0)
    with P.Plan(w, precision=prec) as pl:
        phi = pl.intermediate_states(w.u0)[0]
    assert np.max(np.abs(phi - phi_o)) <= TOL[prec][0], np.max(np.abs(phi - phi_o))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,w", CASES, ids=IDS)
def test_pauli_subinterval_grad(P, name, w, prec):
    phi_o = M.intermediate_states(w, w.u0)
    g_o, Jn_o = M.subinterval_all(w, phi_o, w.u0)
    with P.Plan(w, precision=prec) as pl:
        g, Jn = pl.subinterval_grad(phi_o, w.u0)
    assert g.shape == (1, w.Nt, w.m)
    assert rel(g[0], g_o) <= TOL[prec][1], rel(g[0], g_o)
    assert np.max(np.abs(Jn[0] - Jn_o)) <= (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,w", CASES[:2], ids=IDS[:2])
def test_pauli_iterate_and_gradient(P, name, w, prec):
    u_o, J_o, F_o, E_o = M.ism_solve(w, w.u0, 3, 0.3)
    g_o = M.global_gradient(w, w.u0)
    with P.Plan(w, precision=prec, rho=0.3) as pl:
        u, J, E = pl.iterate(w.u0, 3)
        g, Jg = pl.gradient(w.u0)
    tj = TOL[prec][2] if prec == "fp64" else 1e-4
    assert np.max(np.abs(J[0] - J_o)) <= tj, np.max(np.abs(J[0] - J_o))
    assert rel(u[0] - w.u0, u_o - w.u0) <= (1e-9 if prec == "fp64" else 1e-4)
    assert rel(E[0], E_o) <= (1e-4 if prec == "mixed" else 1e-9), rel(E[0], E_o)
    assert rel(g[0], g_o) <= TOL[prec][1]
    assert abs(Jg[0] - J_o[0]) <= tj


def test_pauli_batch_equals_singles(P):
    w = CASES[0][1]
    rng = np.random.default_rng(3)
    U = rng.uniform(-1, 1, (3, w.Nt, w.m))
    with P.Plan(w, precision="fp64", batch=3) as pl:
        Jb, _ = pl.evaluate(U)
        gb, _ = pl.gradient(U)
    for b in range(3):
        with P.Plan(w, precision="fp64") as pl:
            J1, _ = pl.evaluate(U[b])
            g1, _ = pl.gradient(U[b])
        assert abs(J1[0] - Jb[b]) <= 1e-13 and rel(gb[b], g1[0]) <= 1e-12


def test_spin5_at_the_paper_size_against_the_density_matrix_oracle(P):
    """Five spins, density-matrix formalism, 2^15 steps, N = 128, mixed precision: J and the gradient
    of all 10 controls against the Hilbert-space density-matrix oracle, and one ISM iteration (L = 1,
    which by Theorem 2 is the gradient step u + rho g / tau)."""
    w = W.spin5_liouville()
    rho = 100.0
    J_o = M.dm_objective(w, w.u0)
    g_o = M.dm_gradient(w, w.u0)
    with P.Plan(w, precision="mixed", rho=rho) as pl:
        g, J = pl.gradient(w.u0)
        u1, Jh, _ = pl.iterate(w.u0, 1)
    assert abs(J[0] - J_o) <= 1e-5, abs(J[0] - J_o)
    assert rel(g[0], g_o) <= 1e-4, rel(g[0], g_o)
    u1_o = w.u0 + rho * g_o / w.tau
    assert rel(u1[0] - w.u0, u1_o - w.u0) <= 1e-4
    assert abs(Jh[0, 1] - M.dm_objective(w, u1_o)) <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pauli_most_controls_and_one_step_sub_intervals(P, prec):
    """32 controls (the most a plan takes) on d = 128, N = Nt (one step per sub-interval)."""
    w = W.random_pauli(7, 32, 34, T=0.3, Nt=20, N=20, u_amp=0.3)
    phi_o = M.intermediate_states(w, w.u0)
    g_o, _ = M.subinterval_all(w, phi_o, w.u0)
    u_o, J_o, _, _ = M.ism_solve(w, w.u0, 2, 0.3)
    with P.Plan(w, precision=prec, rho=0.3) as pl:
        phi = pl.intermediate_states(w.u0)[0]
        g, _ = pl.subinterval_grad(phi_o, w.u0)
        u, J, _ = pl.iterate(w.u0, 2)
    assert np.max(np.abs(phi - phi_o)) <= TOL[prec][0]
    assert rel(g[0], g_o) <= TOL[prec][1]
    assert np.max(np.abs(J[0] - J_o)) <= (1e-9 if prec == "fp64" else 1e-5)
    assert rel(u[0] - w.u0, u_o - w.u0) <= (1e-9 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pauli_checkpoint_stride_changes_nothing(P, prec):
    """Several controls, literal sub-problems: every stride gives the same gradients of all controls
    and J_n bit for bit."""
    w = CASES[1][1]
    res = []
    phi_o = M.intermediate_states(w, w.u0)
    for S in (1, 4, 0, 10 ** 6):
        with P.Plan(w, precision=prec, ckpt_stride=S) as pl:
            res.append(pl.subinterval_grad(phi_o, w.u0))
    for g, Jn in res[1:]:
        assert np.array_equal(g, res[0][0]) and np.array_equal(Jn, res[0][1])
    g_o, _ = M.subinterval_all(w, phi_o, w.u0)
    assert rel(res[0][0][0], g_o) <= TOL[prec][1]
