"""The multi-GPU path (replicas only) on CPU ranks: two gloo processes run
the host logic bench.py uses under torchrun -- the barrier, the
max-over-ranks time and the whole-job rate of weak scaling (the units of
all ranks over the slowest rank's time).  One process (no process group)
reduces to its own numbers.  No data moves between ranks: the path has no
exchange step."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_0907_3390_gb300 import replicas as R  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = [0.5, 2.0, 1.25, 0.75][rank]
        rate, t_max = R.whole_job_rate(100.0, seconds, dist)
        R.barrier(dist)
        m = R.max_over_ranks(float(rank), dist)
        q.put((rank, rate, t_max, m, R.world_size(dist)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_gloo_ranks_combine_timings(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == list(range(world))
    for rank, rate, t_max, m, w in out:
        assert w == world
        assert t_max == 2.0                     # the slowest rank
        assert rate == 100.0 * world / 2.0      # every rank's units over the slowest time
        assert m == float(world - 1)


def test_one_process_is_its_own_job():
    assert R.world_size(None) == 1
    assert R.max_over_ranks(3.5, None) == 3.5
    assert R.whole_job_rate(100.0, 0.5, None) == (200.0, 0.5)
    R.barrier(None)
