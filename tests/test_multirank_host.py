"""The multi-GPU path of bench.py is replicas with no data-path collective: every rank solves its own
batch and the job time is the slowest rank's.  Its host logic runs here on gloo ranks (CPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_env()
        ms = 100.0 + 50.0 * rank                      # rank 1 is slower
        job_ms = bench.slowest_rank_ms(ms, w, "cpu")
        out.put((r, lr, w, job_ms, bench.job_throughput(64, 10, w, job_ms)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replicas_time_is_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slow = 100.0 + 50.0 * (world - 1)
    for r, (rank, local, w, job_ms, thr) in enumerate(res):
        assert (rank, local, w) == (r, r, world)
        assert job_ms == slow
        assert thr == pytest.approx(64 * 10 * world / (slow / 1e3))


def test_single_rank_is_unchanged():
    import bench

    assert bench.slowest_rank_ms(12.5, 1, "cpu") == 12.5
    assert bench.job_throughput(8, 5, 1, 1000.0) == 40.0
