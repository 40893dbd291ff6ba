"""Serving loop (ism_server_*): requests of different dimensions, step counts and N, submitted while
others run, each give exactly the result of the same solve run alone; admission by device footprint."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1603_01237_gb300 as P

    return P


def _gp(n=64, Nt=200, N=8, T=1.5, seed=9):
    rng = np.random.default_rng(seed)
    psi_i, psi_f = W.gp_stationary_states(n, 20.0, -10.0, 1.0, dt=2e-3, steps=4000)
    return W.GPWorkload(name="gp", n=n, L=20.0, x_min=-10.0, g=1.0, psi_i=psi_i, psi_f=psi_f, T=T, Nt=Nt, N=N,
                        u0=rng.uniform(-0.5, 0.5, Nt), rho=0.5)


def _mix():
    return [
        (W.config("spin16", Nt=400, N=4), "fp64", 6),
        (W.config("rotor41", Nt=1200, N=16), "mixed", 5),
        (W.with_random_target(W.spin_chain(7, 51, T=1.0, Nt=300, N=8, u_amp=1.0), 52), "mixed", 3),
        (W.random_dense(16, 53, T=2.0, Nt=250, N=5), "fp64", 4),
        (_gp(), "mixed", 3),
        (W.config("rotor41", Nt=3000, N=64), "mixed", 4),
        (W.with_random_target(W.spin_chain(9, 54, T=1.0, Nt=200, N=4, u_amp=1.0), 55), "mixed", 2),
        (W.config("spin16", Nt=1000, N=8), "mixed", 5),
    ]


def _alone(P, w, prec, iters, **kw):
    """The request alone: submitted to a server of its own and waited for (for the requests that share
    launches, a shared plan holding just this one)."""
    with P.Server(slots=1, hbm_budget_bytes=8 << 30, **kw) as srv:
        u, J, _ = srv.result(srv.submit(w, iters=iters, precision=prec))
    return u, J


def test_results_in_the_mix_equal_results_alone(P):
    """Requests arriving while others run, several of them sharing launches (rotor problems of one N and
    different step counts and controls; spin chains of one d with different couplings and steps) and
    joining shared plans between their passes, each give exactly the result they give alone."""
    mix = _mix() + [
        (W.config("rotor41", Nt=900, N=16).with_(u0=np.random.default_rng(5).uniform(-1, 1, 900)), "mixed", 4),
        (W.with_random_target(W.spin_chain(7, 58, T=0.8, Nt=260, N=8, u_amp=1.0), 59), "mixed", 6),
        (W.config("rotor41", Nt=1700, N=16), "mixed", 2),
    ]
    rng = np.random.default_rng(1)
    with P.Server(slots=3, hbm_budget_bytes=8 << 30) as srv:
        ids = []
        for w, prec, iters in mix:
            ids.append(srv.submit(w, iters=iters, precision=prec))
            time.sleep(rng.exponential(0.005))   # arrivals while earlier requests run
        got = [srv.result(i) for i in ids]
        st = srv.stats()
    # the FP64, dense and grid requests run on plans of their own; the mixed structured ones fall in
    # five groups (kind, d, N, objective), each opening at least one shared plan
    assert st["single"] == 3 and st["groups"] >= 5, st
    for (w, prec, iters), (u, J, t) in zip(mix, got):
        ua, Ja = _alone(P, w, prec, iters)
        assert np.array_equal(u, ua), w.name
        assert np.array_equal(J, Ja), w.name
        assert t[2] >= t[1] >= 0.0


def test_request_joins_a_running_shared_plan(P):
    """Continuous batching: a request submitted while another of its group is half-way through its
    solve is admitted into the same shared plan between two passes (one shared plan opened, two
    requests in one pass), and both results equal their solves alone."""
    a = W.config("rotor41", Nt=3000, N=16)
    b = W.config("rotor41", Nt=1000, N=16).with_(u0=np.random.default_rng(8).uniform(-1, 1, 1000))
    with P.Server(slots=1, hbm_budget_bytes=8 << 30) as srv:
        ia = srv.submit(a, iters=150, precision="mixed")
        for _ in range(2000):   # wait until the first request's plan is running
            if srv.poll(ia)[0] == P.abi.ISM_REQ_RUNNING:
                break
            time.sleep(0.001)
        time.sleep(0.02)
        ib = srv.submit(b, iters=3, precision="mixed")
        ua, Ja, _ = srv.result(ia)
        ub, Jb, _ = srv.result(ib)
        st = srv.stats()
    assert st["groups"] == 1 and st["max_rows"] == 2 and st["single"] == 0
    for (w, it), (u, J) in zip(((a, 150), (b, 3)), ((ua, Ja), (ub, Jb))):
        u0, J0 = _alone(P, w, "mixed", it)
        assert np.array_equal(u, u0) and np.array_equal(J, J0)
    # and the shared plan's results are the FP64 oracle's to the mixed-precision bar
    from oracle import ism_oracle as O

    u_o, J_o, _, _ = O.ism_solve(b, b.u0, 3, b.rho)
    assert np.max(np.abs(Jb[0] - J_o)) <= 1e-4


def test_admission_by_footprint(P):
    """A budget that holds one plan at a time still completes every request (one after another);
    a request larger than the whole budget is refused at submission."""
    w = W.config("rotor41", Nt=1500, N=16)
    one = P.footprint(w) + 16 * 4 + (1 << 20)
    with P.Server(slots=4, hbm_budget_bytes=int(one * 1.5)) as srv:
        ids = [srv.submit(w, iters=3, precision="mixed") for _ in range(3)]
        res = [srv.result(i) for i in ids]
        for u, J, t in res[1:]:
            assert np.array_equal(u, res[0][0])
        starts = sorted(t[0] for _, _, t in res)
        assert starts[2] > starts[0]   # queued behind the budget
        with pytest.raises(P.IsmError) as ei:
            srv.submit(W.config("rotor41", Nt=20000, N=128), iters=1, batch=64)
        assert ei.value.status == 2


def test_footprint_matches_plan_bytes(P):
    for w in (W.config("rotor41", Nt=2000, N=16), W.config("ising1024", Nt=500, N=8), _gp()):
        with P.Plan(w, precision="mixed") as pl:
            assert pl.info(3) == P.footprint(w, precision="mixed")


def test_concurrent_blocked_chains_of_different_sizes(P):
    """Plans whose chain kernels need different shared-memory sizes (blocked chains of d = 16, 41 and
    64 at N = 64 and 128) run concurrently on 6 slots, many times over: every request completes and
    equals its solve alone (the kernels' shared-memory caps are raised once, not per launch)."""
    base = [
        (W.config("spin16", Nt=640, N=64), "mixed", 2),
        (W.config("rotor41", Nt=1280, N=128), "mixed", 2),
        (W.random_dense(64, 56, T=1.0, Nt=256, N=64), "mixed", 2),
        (W.random_dense(57, 57, T=1.0, Nt=256, N=64), "fp64", 2),
    ]
    mix = base * 6
    with P.Server(slots=6, hbm_budget_bytes=16 << 30, group_capacity=-1) as srv:   # every request its own plan
        ids = [srv.submit(w, iters=it, precision=prec) for w, prec, it in mix]
        got = [srv.result(i) for i in ids]
    alone = []
    for w, prec, it in base:
        with P.Plan(w, precision=prec) as pl:
            assert pl.info(7) > 1   # blocked chain
            alone.append(pl.iterate(w.u0, it)[:2])
    for k, (u, J, t) in enumerate(got):
        ua, Ja = alone[k % len(base)]
        assert np.array_equal(u, ua) and np.array_equal(J, Ja)
