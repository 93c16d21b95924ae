"""Database-partitioned search across processes (one GPU each).

The database is split into contiguous parts; every process holds the index
(graph and FINGER tables) of its own part, searches every query there, and
the parts' K nearest are exchanged and merged into the K nearest of the whole
database (the kNN problem of Sec. 1 of arXiv 2206.11408 over the union of the
parts).  Unlike query replicas (``replicas.py``) this path has a real exchange
step: an all-gather of nq x K (id, distance) pairs per part, then the top-K
merge on the device (``finger_merge_topk``).  Results differ from one index
over the whole database because each part has its own graph.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of part `rank` of n rows split into `world` contiguous parts
    whose sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def exchange(ids, dists):
    """All parts' nq x K results, stacked part-major (S x nq x K) in rank
    order.  Works on CPU tensors with gloo and CUDA tensors with NCCL; one
    process returns its own results with S = 1."""
    import torch
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return ids.unsqueeze(0).contiguous(), dists.unsqueeze(0).contiguous()
    ws = dist.get_world_size()
    gi = [torch.empty_like(ids) for _ in range(ws)]
    gd = [torch.empty_like(dists) for _ in range(ws)]
    dist.all_gather(gi, ids.contiguous())
    dist.all_gather(gd, dists.contiguous())
    return torch.stack(gi), torch.stack(gd)


def offsets(lo: int, device="cpu") -> list[int]:
    """Every part's first global id, in rank order."""
    import torch
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return [int(lo)]
    t = torch.tensor([int(lo)], dtype=torch.int64, device=device)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return [int(x.item()) for x in out]


def search_partitioned(ix, queries, K: int, ef: int, lo: int, stream=None):
    """Search this process's part, exchange, and merge: the K nearest of the
    whole database for every query (CUDA tensors nq x K, global ids)."""
    from . import merge_topk
    ids, d = ix.search(queries, K, ef, stream=stream)
    gi, gd = exchange(ids, d)
    return merge_topk(gi, gd, offsets(lo, device=queries.device), stream=stream)
