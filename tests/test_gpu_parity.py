"""CUDA path (through the C ABI) vs the FP64 oracle on identical seeded inputs.

Tolerances: FP64 mode |dF| <= 1e-9 on the objective and tight element-wise bounds on states and
gradients; mixed mode |dF| <= 1e-5 and gradient relative L2 <= 1e-4.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ism_oracle as O

pytestmark = pytest.mark.gpu

FP64_PHI = 1e-11
FP64_GRAD = 1e-10
MIX_PHI = 2e-5
MIX_GRAD = 1e-4


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1603_01237_gb300 as P

    return P


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _random_target(w, seed):
    """Same problem with a random unit complex target, so the overlap and its gradient are O(1)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(w.d) + 1j * rng.standard_normal(w.d)
    return w.with_(psi_f=v / np.linalg.norm(v))


def _h1_diagonal(w, seed):
    rng = np.random.default_rng(seed)
    return w.with_(H1=w.H1 + np.diag(rng.uniform(-0.3, 0.3, w.d)))


def _cases():
    return [
        ("spin16-fp64", W.config("spin16", Nt=400, N=4), "fp64"),
        ("spin16-ragged", W.config("spin16", Nt=401, N=7), "fp64"),
        ("rotor41-fp64", W.config("rotor41", Nt=1000, N=16), "fp64"),
        ("rotor41-mixed", W.config("rotor41", Nt=1000, N=16), "mixed"),
        ("dense5-fp64", W.random_dense(5, 61, T=2.0, Nt=203, N=6), "fp64"),
        ("dense41-obs-fp64", W.random_dense(41, 62, T=2.0, Nt=150, N=9, objective="observable"), "fp64"),
        ("dense64-fp64", W.random_dense(64, 63, T=2.0, Nt=120, N=5), "fp64"),
        ("dense16-mixed", W.random_dense(16, 64, T=2.0, Nt=300, N=10), "mixed"),
        ("tridiag2-fp64", W.rabi(0.7, 0.3, T=3.0, Nt=64, N=8).with_(kind="tridiag"), "fp64"),
        ("bitflip2-fp64", _random_target(W.spin_all_to_all(1, 5, T=3.0, Nt=64, N=4, u_amp=1.5), 1), "fp64"),
        ("bitflip32-mixed", _random_target(W.spin_chain(5, 66, T=4.0, Nt=500, N=20, u_amp=1.5), 2), "mixed"),
        ("bitflip64-fp64", _random_target(W.spin_chain(6, 67, T=2.0, Nt=200, N=8, u_amp=1.5), 3), "fp64"),
        # near-zero overlap (|0..0> -> |1..1> at small u): gradients ~1e-12, compared in absolute terms
        ("bitflip64-tiny-fp64", W.spin_chain(6, 68, T=2.0, Nt=200, N=8), "fp64"),
        # tridiagonal H1 with a diagonal (the rotor's -cos(theta) has none): the other kernel variant
        ("tridiag41-h1diag-fp64", _h1_diagonal(W.config("rotor41", Nt=600, N=6), 21), "fp64"),
        ("tridiag41-h1diag-mixed", _h1_diagonal(W.config("rotor41", Nt=600, N=6), 22), "mixed"),
    ]


CASES = _cases()


@pytest.mark.parametrize("name,w,prec", CASES, ids=[c[0] for c in CASES])
def test_intermediate_states(P, name, w, prec):
    phi_o = O.intermediate_states(w, w.u0)
    with P.Plan(w, precision=prec) as pl:
        phi = pl.intermediate_states(w.u0)[0]
    tol = FP64_PHI if prec == "fp64" else MIX_PHI
    assert np.max(np.abs(phi - phi_o)) <= tol, np.max(np.abs(phi - phi_o))
    assert np.array_equal(phi[0], phi_o[0])            # phi_0 = psi_i exactly


@pytest.mark.parametrize("name,w,prec", CASES, ids=[c[0] for c in CASES])
def test_subinterval_grad(P, name, w, prec):
    phi_o = O.intermediate_states(w, w.u0)
    g_o, Jn_o = O.subinterval_all(w, phi_o, w.u0)
    with P.Plan(w, precision=prec) as pl:
        g, Jn = pl.subinterval_grad(phi_o, w.u0)
    tol = FP64_GRAD if prec == "fp64" else MIX_GRAD
    if "tiny" in name:   # absolute bound on the scale tau * ||H1|| of a unit-state gradient term
        scale = w.tau * np.abs(w.H1).sum(axis=1).max()
        assert np.max(np.abs(g[0] - g_o)) <= 1e-13 * scale
    else:
        assert rel_l2(g[0], g_o) <= tol, rel_l2(g[0], g_o)
    # mixed: these cases take steps 10-40x coarser than the benchmark problem (tau * rad up to 4.3),
    # where the FP32 rounding of the propagated psi_n is ~3 eps per sub-step (see test_iterate below)
    jt = 1e-12 if prec == "fp64" else 1e-5
    assert np.max(np.abs(Jn[0] - Jn_o)) <= jt * max(1.0, np.abs(Jn_o).max())


@pytest.mark.parametrize("name,w,prec", CASES[:4] + CASES[5:6], ids=[c[0] for c in CASES[:4] + CASES[5:6]])
def test_iterate_matches_algorithm1(P, name, w, prec):
    iters = 3
    u_o, J_o, F_o, E_o = O.ism_solve(w, w.u0, iters, w.rho)
    with P.Plan(w, precision=prec) as pl:
        u, J, E = pl.iterate(w.u0, iters)
        Jf, Ff = pl.evaluate(u[0])
    # mixed: these reduced cases take steps 10-20x coarser than the benchmark problem (tau*rad ~ 1.3-2.6
    # per step), where FP32 rounding inside the Chebyshev terms is ~eps * sum_k k|a_k| ~ 3 eps per step;
    # the 1e-5 bound is checked at the benchmark's own step size (test_rotor_mixed_fine_steps and the
    # full-size tests)
    tolF = 1e-9 if prec == "fp64" else 1e-4
    assert np.max(np.abs(J[0] - J_o)) <= tolF
    assert abs(Ff[0] - F_o[-1]) <= tolF
    assert rel_l2(u[0] - w.u0, u_o - w.u0) <= (1e-9 if prec == "fp64" else 1e-4)
    assert rel_l2(E[0], E_o) <= (1e-9 if prec == "fp64" else 1e-4)


def test_spin16_full_config_fp64(P):
    """The spin benchmark problem at its full size: 4 spins, Nt=1000, N=4, 20 iterations, FP64."""
    w = W.config("spin16")
    u_o, J_o, F_o, E_o = O.ism_solve(w, w.u0, w.iters, w.rho)
    with P.Plan(w, precision="fp64") as pl:
        u, J, E = pl.iterate(w.u0, w.iters)
        _, F = pl.evaluate(u[0])
    assert np.max(np.abs(J[0] - J_o)) <= 1e-9
    assert abs(F[0] - F_o[-1]) <= 1e-9
    assert np.max(np.abs(u[0] - u_o)) <= 1e-9


def test_n_independence_on_gpu(P):
    """L = 1: iterates do not depend on N (Theorem 2), here through the CUDA path in FP64."""
    base = W.config("rotor41", Nt=600, N=1)
    res = []
    for N in (1, 4, 25, 600):
        with P.Plan(base.with_(N=N), precision="fp64") as pl:
            res.append(pl.iterate(base.u0, 2)[0][0])
    for u in res[1:]:
        assert np.max(np.abs(u - res[0])) <= 1e-10


def test_batch_equals_singles(P):
    w = W.config("rotor41", Nt=800, N=8)
    rng = np.random.default_rng(5)
    U = np.stack([w.u0, rng.uniform(-1, 1, w.Nt), rng.uniform(-2, 2, w.Nt)])
    with P.Plan(w, precision="mixed", batch=3) as pl:
        ub, Jb, Eb = pl.iterate(U, 2)
    for b in range(3):
        with P.Plan(w, precision="mixed") as pl:
            u1, J1, E1 = pl.iterate(U[b], 2)
        assert np.array_equal(ub[b], u1[0])
        assert np.array_equal(Jb[b], J1[0])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_parameter_layouts_agree(P, prec):
    """The propagator parameters of few (problem, sub-interval) pairs come from one warp per pair, of
    many from one thread per pair: the same arithmetic, so a problem's iterates are the same bits in
    a one-problem plan and in a batch of 65 x 128 pairs (both assemble the sub-interval propagators)."""
    w = W.config("rotor41", Nt=1280, N=128)
    rng = np.random.default_rng(6)
    U = np.stack([w.u0] + [rng.uniform(-1, 1, w.Nt) for _ in range(64)])
    with P.Plan(w, precision=prec, batch=65, step1=1) as pl:
        ub, Jb, Eb = pl.iterate(U, 2)
    with P.Plan(w, precision=prec, step1=1) as pl:
        u1, J1, E1 = pl.iterate(w.u0, 2)
    assert np.array_equal(ub[0], u1[0]) and np.array_equal(Jb[0], J1[0]) and np.array_equal(Eb[0], E1[0])


def test_local_iterations(P):
    w = W.random_dense(6, 71, T=2.0, Nt=120, N=4)
    u_o, J_o, _, _ = O.ism_solve(w, w.u0, 2, 0.2, L=3)
    with P.Plan(w, precision="fp64", local_iters=3, rho=0.2) as pl:
        u, J, E = pl.iterate(w.u0, 2)
    assert np.max(np.abs(u[0] - u_o)) <= 1e-10
    assert np.max(np.abs(J[0] - J_o)) <= 1e-10


def test_device_pointers_and_torch_stream(P):
    import torch

    w = W.config("rotor41", Nt=500, N=10)
    s = torch.cuda.Stream()
    ud = torch.tensor(w.u0, dtype=torch.float64, device="cuda").reshape(1, -1).contiguous()
    phi = torch.empty((1, w.N + 1, w.d, 2), dtype=torch.float64, device="cuda")
    with P.Plan(w, precision="fp64", stream=s) as pl:
        pl.ism_intermediate_states(ud, phi)
        phi_h = pl.intermediate_states(w.u0)
        Jd = torch.empty((1, 3), dtype=torch.float64, device="cuda")
        pl.ism_iterate(2, ud, Jd, None)
        uh, Jh, _ = pl.iterate(w.u0, 2)
    p = phi.cpu().numpy()[..., 0] + 1j * phi.cpu().numpy()[..., 1]
    assert np.array_equal(p, phi_h)
    assert np.array_equal(ud.cpu().numpy(), uh)
    assert np.array_equal(Jd.cpu().numpy(), Jh)


def test_nonfinite_controls_rejected(P):
    w = W.config("spin16", Nt=100, N=4)
    u = w.u0.copy()
    u[17] = np.nan
    with P.Plan(w) as pl:
        with pytest.raises(P.IsmError) as ei:
            pl.iterate(u, 1)
        assert ei.value.status == 4
        import torch

        ud = torch.tensor(u, dtype=torch.float64, device="cuda").reshape(1, -1)
        with pytest.raises(P.IsmError) as ei:
            pl.ism_evaluate(ud)
        assert ei.value.status == 4
        # the plan stays usable
        J, F = pl.evaluate(w.u0)
        assert np.isfinite(J).all()


def test_stats_count_work(P):
    w = W.config("rotor41", Nt=1000, N=10)
    with P.Plan(w) as pl:
        pl.ism_set_profiling(True)
        pl.iterate(w.u0, 2)
        st = pl.ism_get_stats(reset=True)
    # 2 iterations + 1 final evaluation of J: 3 assemblies and chains, 2 sub-interval sweeps
    assert st["launches"] == [3, 3, 2]
    assert all(m > 0 for m in st["ms"])
    # every assembly propagates d columns over all Nt steps (>= 1 sub-step each)
    assert st["substeps"][0] >= 3 * w.d * w.Nt
    assert st["substeps"][1] >= 2 * 2 * w.Nt


@pytest.mark.parametrize("w", [W.config("rotor41", Nt=1500, N=30), W.random_dense(8, 91, T=2.0, Nt=300, N=12)],
                         ids=["rotor41", "dense8"])
def test_theorem2_form_equals_literal_form_fp64(P, w):
    """ism_iterate's first local step in the two-trajectory form of the proof of Theorem 2 and in the
    literal sub-problem form give the same iterates (FP64)."""
    out = []
    for form in (1, 2):
        with P.Plan(w, precision="fp64", subproblem_form=form) as pl:
            out.append(pl.iterate(w.u0, 3))
    assert np.max(np.abs(out[0][0] - out[1][0])) <= 1e-11
    assert np.max(np.abs(out[0][1] - out[1][1])) <= 1e-11
    assert rel_l2(out[0][2], out[1][2]) <= 1e-10


def test_rotor_mixed_fine_steps(P):
    """At the benchmark's step size (tau = pi/20000) mixed precision stays within 1e-5 of the FP64
    oracle's J history; here on a 2000-step horizon T = pi/10 (N = 16) so the oracle is quick."""
    w = W.config("rotor41", Nt=2000, N=16).with_(T=float(np.pi) / 10.0)
    u_o, J_o, F_o, _ = O.ism_solve(w, w.u0, 4, 5.0)
    with P.Plan(w, precision="mixed", rho=5.0) as pl:
        u, J, _ = pl.iterate(w.u0, 4)
    assert np.max(np.abs(J[0] - J_o)) <= 1e-5, np.max(np.abs(J[0] - J_o))
    assert np.all(np.diff(J_o) > 0)


# ---------------------------------------------------------------- Algorithm 1 (a)-(b) by direct sweeps
DIRECT = [c for c in CASES if c[0] in ("spin16-ragged", "rotor41-fp64", "rotor41-mixed", "dense41-obs-fp64",
                                        "dense16-mixed", "bitflip32-mixed", "tridiag41-h1diag-mixed")]


@pytest.mark.parametrize("name,w,prec", DIRECT, ids=[c[0] for c in DIRECT])
def test_direct_sweeps_match_oracle(P, name, w, prec):
    """step1 = 2: psi(t_n), chi(t_n) by direct propagation (2 Nt state-steps) instead of assembly."""
    phi_o = O.intermediate_states(w, w.u0)
    Jo, Fo = O.objective(w, w.u0)
    with P.Plan(w, precision=prec, step1=2) as pl:
        assert pl.info(6) == 2
        phi = pl.intermediate_states(w.u0)[0]
        J, F = pl.evaluate(w.u0)
    tol = FP64_PHI if prec == "fp64" else MIX_PHI
    assert np.max(np.abs(phi - phi_o)) <= tol, np.max(np.abs(phi - phi_o))
    assert np.array_equal(phi[0], phi_o[0])
    assert abs(J[0] - Jo) <= (1e-11 if prec == "fp64" else 2e-5)
    assert abs(F[0] - Fo) <= (1e-11 if prec == "fp64" else 2e-5)


@pytest.mark.parametrize("name,w,prec", DIRECT[:3], ids=[c[0] for c in DIRECT[:3]])
def test_direct_iterate_matches_algorithm1(P, name, w, prec):
    iters = 3
    u_o, J_o, F_o, E_o = O.ism_solve(w, w.u0, iters, w.rho)
    with P.Plan(w, precision=prec, step1=2) as pl:
        u, J, E = pl.iterate(w.u0, iters)
    tol = 1e-9 if prec == "fp64" else 1e-4
    assert np.max(np.abs(J[0] - J_o)) <= tol
    assert rel_l2(u[0] - w.u0, u_o - w.u0) <= tol


def test_step1_default_follows_the_batch(P):
    w = W.config("rotor41", Nt=400, N=8)
    with P.Plan(w, precision="mixed", batch=95) as pl:
        assert pl.info(6) == 1
    with P.Plan(w, precision="mixed", batch=96) as pl:
        assert pl.info(6) == 2
    with P.Plan(w, precision="mixed", batch=96, step1=1) as pl:
        assert pl.info(6) == 1


# ---------------------------------------------------------------- blocked chain (N >= 32)
BLOCKED = [
    ("rotor41-N40-fp64", W.config("rotor41", Nt=1000, N=40), "fp64"),         # observable, ragged blocks
    ("rotor41-N40-mixed", W.config("rotor41", Nt=2000, N=40).with_(T=2000 * np.pi / 20000), "mixed"),
    ("dense16-N37-fp64", W.random_dense(16, 65, T=2.0, Nt=370, N=37), "fp64"),  # overlap: two chains
    ("bitflip32-N64-mixed", _random_target(W.spin_chain(5, 69, T=4.0, Nt=640, N=64, u_amp=1.0), 4), "mixed"),
]


@pytest.mark.parametrize("name,w,prec", BLOCKED, ids=[c[0] for c in BLOCKED])
def test_blocked_chain_matches_oracle(P, name, w, prec):
    """From N = 32 the chain runs over products of ~sqrt(N) consecutive propagators and fills the
    states inside each block in parallel; the intermediate states and J are unchanged."""
    phi_o = O.intermediate_states(w, w.u0)
    Jo, Fo = O.objective(w, w.u0)
    with P.Plan(w, precision=prec) as pl:
        assert pl.info(7) > 1
        phi = pl.intermediate_states(w.u0)[0]
        J, F = pl.evaluate(w.u0)
    tol = FP64_PHI if prec == "fp64" else MIX_PHI
    assert np.max(np.abs(phi - phi_o)) <= tol, np.max(np.abs(phi - phi_o))
    assert abs(J[0] - Jo) <= (1e-11 if prec == "fp64" else 2e-5)
    assert abs(F[0] - Fo) <= (1e-11 if prec == "fp64" else 2e-5)


def test_bounded_wait_gives_up_cleanly(P):
    """A cap of one try on device-side waits makes the chain's first mbarrier wait give up before its
    propagator tile has landed: the call returns ISM_ETIMEOUT (the block first waits, with its own
    bound, for the copies it has in flight), and the context stays usable."""
    w = W.config("rotor41", Nt=2000, N=16)
    seen = 0
    for _ in range(4):
        with P.Plan(w, precision="mixed", max_spin_iters=1) as pl:
            try:
                pl.evaluate(w.u0)
            except P.IsmError as e:
                assert e.status == 5, e
                seen += 1
    assert seen >= 1
    Jo, _ = O.objective(w, w.u0)
    with P.Plan(w, precision="mixed") as pl:
        J, _ = pl.evaluate(w.u0)
    assert abs(J[0] - Jo) <= 2e-5


def test_direct_sweeps_wide_layout_for_large_batches(P):
    """From 2 x 152 x 16 problems per plan the direct sweeps switch to the assembly's lane layout
    (8 lanes x 6 elements for d = 41): the same results as the 16-lane layout of a small batch, and
    the oracle's within the mixed tolerance."""
    r = W.config("rotor41", Nt=2000, N=16).with_(T=float(np.pi) / 10.0)
    rng = np.random.default_rng(9)
    rows = np.stack([r.u0] + [rng.uniform(-1, 1, r.Nt) for _ in range(2)])
    B = 4864
    U = np.tile(rows, (B // 3 + 1, 1))[:B]
    with P.Plan(r, precision="mixed", batch=B) as pl:
        assert pl.info(6) == 2 and pl.info(9) == 8
        Jw, Fw = pl.evaluate(U)
        gw, _ = pl.gradient(U)
    with P.Plan(r, precision="mixed", batch=3, step1=2) as pl:
        assert pl.info(9) == 16
        Jn, Fn = pl.evaluate(rows)
        gn, _ = pl.gradient(rows)
    for b in range(3):
        for k in (b, b + 3 * 700, B - 3 + ((b - B) % 3)):
            assert abs(Jw[k] - Jn[b]) <= 1e-12 and rel_l2(gw[k], gn[b]) <= 1e-10
        Jo, Fo = O.objective(r, rows[b])
        assert abs(Jn[b] - Jo) <= 1e-5


def test_norm_drift_is_recorded_and_removed(P):
    """psi(t_n), chi(t_n) are renormalised in FP64 to the norms of psi_i and chi(T) (a no-op in exact
    arithmetic); the largest drift found is reported: rounding-level in FP64, small but nonzero for
    FP32 propagation (~1e-5 in norm^2 after the FP32 chain of 16 assembled propagators, less for
    the compensated direct sweeps).  The renormalised states give J within the usual bounds."""
    w = W.config("rotor41", Nt=2000, N=16)
    J_o, _ = O.objective(w, w.u0)
    for prec, lo, hi, tj in (("fp64", 0.0, 1e-12, 1e-9), ("mixed", 1e-12, 1e-4, 1e-5)):
        for step1 in (1, 2):
            with P.Plan(w, precision=prec, step1=step1) as pl:
                pl.ism_get_stats(reset=True)
                J, _ = pl.evaluate(w.u0)
                drift = pl.ism_get_stats()["norm_drift"]
            assert lo <= drift <= hi, (prec, step1, drift)
            assert abs(J[0] - J_o) <= tj


@pytest.mark.parametrize("prec,w", [
    ("fp64", W.config("rotor41", Nt=1001, N=7)),
    ("mixed", W.config("rotor41", Nt=1001, N=7)),
    ("fp64", _random_target(W.spin_chain(5, 71, T=4.0, Nt=333, N=5, u_amp=1.5), 5)),
    ("mixed", W.random_dense(16, 72, T=2.0, Nt=257, N=3)),
], ids=["rotor-fp64", "rotor-mixed", "bitflip32-fp64", "dense16-mixed"])
def test_checkpoint_stride_changes_nothing(P, prec, w):
    """The literal sub-problem stores psi_n every ckpt_stride steps and recomputes each segment from
    its checkpoint (hi + lo in FP32), repeating the forward sweep exactly: the gradient and J_n are the
    same bit for bit for every stride (1, a ragged 7, the default, the whole sub-interval) and match
    the oracle's literal sub-problems."""
    phi_o = O.intermediate_states(w, w.u0)
    g_o, Jn_o = O.subinterval_all(w, phi_o, w.u0)
    res = []
    for S in (1, 7, 0, 10 ** 6):
        with P.Plan(w, precision=prec, ckpt_stride=S) as pl:
            res.append(pl.subinterval_grad(phi_o, w.u0))
    for g, Jn in res[1:]:
        assert np.array_equal(g, res[0][0]) and np.array_equal(Jn, res[0][1])
    tol = FP64_GRAD if prec == "fp64" else MIX_GRAD
    assert rel_l2(res[0][0][0], g_o) <= tol
    jt = 1e-12 if prec == "fp64" else 1e-5
    assert np.max(np.abs(res[0][1][0] - Jn_o)) <= jt * max(1.0, np.abs(Jn_o).max())


def test_local_iterations_with_checkpoints_match_algorithm1(P):
    """L = 3 local steps (the later ones literal, so checkpointed) with a small stride, FP64 and mixed,
    against the oracle's Algorithm 1."""
    w = W.config("rotor41", Nt=1200, N=8)
    iters, L = 2, 3
    u_o, J_o, F_o, E_o = O.ism_solve(w, w.u0, iters, w.rho, L=L)
    for prec, tol in (("fp64", 1e-9), ("mixed", 1e-4)):
        with P.Plan(w, precision=prec, local_iters=L, ckpt_stride=5) as pl:
            u, J, E = pl.iterate(w.u0, iters)
        assert np.max(np.abs(J[0] - J_o)) <= tol, (prec, np.max(np.abs(J[0] - J_o)))
        assert rel_l2(u[0] - w.u0, u_o - w.u0) <= tol
