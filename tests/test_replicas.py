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


def _worker_dies(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)          # as torchrun sets them
    os.environ["WORLD_SIZE"] = str(world)
    R.init(dist, "gloo", timeout_s=5.0)
    if rank == 1:
        os._exit(0)                     # a rank that leaves between steps, without a word
    import time
    t0 = time.perf_counter()
    try:
        R.barrier(dist)
        q.put(("no error", time.perf_counter() - t0))
    except Exception as e:              # the failure surfaces on the host as an error
        q.put((type(e).__name__, time.perf_counter() - t0))


def test_dead_rank_is_detected_on_the_host():
    """A rank that exits between steps: the other rank's next barrier ends
    with an error within the process group's timeout (here 5 s), instead of
    waiting for ever."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_dies, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    what, waited = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert what != "no error"
    assert waited < 60.0, waited
