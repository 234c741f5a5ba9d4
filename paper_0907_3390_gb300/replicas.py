"""The multi-GPU path: replicas only.

Patch groups shard naturally, but a sharded hierarchy needs the halo
exchange of ghost slabs per level and step and the global reductions of dt
and of the conservation sums (the MPI buffer patches of Sec. 2.4); with one
GPU per call nothing of that is built.  N processes, one per GPU, each
advance their own copy of the workload; the whole-job rate is the work all
ranks did over the slowest rank's time (weak scaling).  These helpers take
the ``torch.distributed`` module (or None for one process) and only
combine timings: no data moves between ranks.
"""
from __future__ import annotations

import datetime


def init(dist, backend: str, timeout_s: float = 300.0) -> None:
    """Join the process group (rank, world size and rendezvous from the
    environment, as torchrun sets them) with a bounded timeout: a rank that
    dies between steps makes the others' next barrier or reduction fail
    with an error within timeout_s instead of waiting for ever."""
    dist.init_process_group(backend=backend, timeout=datetime.timedelta(seconds=timeout_s))


def world_size(dist) -> int:
    return 1 if dist is None else dist.get_world_size()


def barrier(dist) -> None:
    if dist is not None:
        dist.barrier()


def max_over_ranks(x: float, dist, device="cpu") -> float:
    """The largest x over all ranks (x itself for one process).  device:
    where the reduction tensor lives (a CUDA device under NCCL, the CPU
    under gloo)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds: float, dist, device="cpu"):
    """(rate, slowest time): every rank did units_per_rank units in its own
    `seconds`; the job's rate is the sum of the units over the slowest
    rank's time."""
    t_max = max_over_ranks(seconds, dist, device)
    return units_per_rank * world_size(dist) / t_max, t_max
