"""Replica data parallelism for the search path (one process per GPU).

Greedy search over a fixed index is independent per query (Algorithms 1 and 4
of arXiv 2206.11408 run one query at a time), so the path shards by queries
with no exchange step: every rank holds a full copy of the index and serves its
own contiguous slice of the query set.  The only collectives are the ones a
benchmark needs around the timed region: a barrier, the agreement on a common
setting (max over ranks) and the max/sum reductions of timings and counts.
They work with any torch.distributed backend (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def query_slice(nq_per_rank: int, rank: int) -> tuple[int, int]:
    """[start, stop) of this rank's queries in a set of nq_per_rank x world rows."""
    return rank * nq_per_rank, (rank + 1) * nq_per_rank


def _reduce(values, op: str, device):
    import torch
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(x) for x in t.cpu()]


def max_over_ranks(values, device="cpu") -> list[float]:
    """Element-wise maximum over ranks (slowest rank's time, agreed settings)."""
    return _reduce(values, "max", device)


def sum_over_ranks(values, device="cpu") -> list[float]:
    """Element-wise sum over ranks (total work, hit counts)."""
    return _reduce(values, "sum", device)


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
