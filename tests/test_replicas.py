"""Multi-rank host logic of the replica path on CPU (gloo, world size 2): the
query slices partition the query set, ranks agree on a setting by the max, and
timings/work reduce by max and sum.  The search path itself has no exchange
step (each query is an independent Algorithm 4 run), so these reductions are
all the collectives a multi-GPU run performs."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2206_11408_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, lr = replicas.world()
        lo, hi = replicas.query_slice(1000, r)
        ef = [140 + 10 * r, 120 - r]                   # each rank's own choice
        agreed = replicas.max_over_ranks(ef)
        ms = replicas.max_over_ranks([5.0 + r])
        hits = replicas.sum_over_ranks([r + 1, 10])
        replicas.barrier()
        out[r] = (ws, r, lr, lo, hi, agreed, ms, hits)
    finally:
        dist.destroy_process_group()


def test_replica_collectives_gloo_world_2():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    slices = sorted((v[3], v[4]) for v in res.values())
    assert slices == [(0, 1000), (1000, 2000)]         # a partition of 2 x 1000 queries
    for r, (ws, rr, lr, lo, hi, agreed, ms, hits) in res.items():
        assert (ws, rr, lr) == (2, r, r)
        assert agreed == [150.0, 120.0]                # max of the ranks' settings
        assert ms == [6.0]                             # slowest rank
        assert hits == [3.0, 20.0]                     # totals


def test_single_process_reductions_are_identity():
    assert replicas.max_over_ranks([1.5, 2]) == [1.5, 2.0]
    assert replicas.sum_over_ranks([3]) == [3.0]
    assert replicas.query_slice(10, 0) == (0, 10)
