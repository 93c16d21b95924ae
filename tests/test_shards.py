"""Host logic of the partitioned-database path on CPU (gloo, world size 2):
the parts partition the rows, and the exchange returns every rank's results
and first ids in rank order, which is what the device merge expects."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2206_11408_gb300 import shards  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = shards.shard_range(1001, rank, world)
        ids = torch.arange(6, dtype=torch.int64).view(2, 3) + 100 * rank
        d = torch.full((2, 3), float(rank), dtype=torch.float32)
        gi, gd = shards.exchange(ids, d)
        offs = shards.offsets(lo)
        out[rank] = (lo, hi, gi.tolist(), gd.tolist(), offs)
    finally:
        dist.destroy_process_group()


def test_partition_exchange_gloo_world_2():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    assert [(res[r][0], res[r][1]) for r in (0, 1)] == [(0, 501), (501, 1001)]
    for r in (0, 1):
        lo, hi, gi, gd, offs = res[r]
        assert gi == [[[0, 1, 2], [3, 4, 5]], [[100, 101, 102], [103, 104, 105]]]
        assert gd == [[[0.0] * 3] * 2, [[1.0] * 3] * 2]
        assert offs == [0, 501]


def test_shard_range_partitions_rows():
    for n, w in ((10, 3), (7, 7), (5, 8), (1_000_000, 6)):
        parts = [shards.shard_range(n, r, w) for r in range(w)]
        assert parts[0][0] == 0 and parts[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        sizes = [hi - lo for lo, hi in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shards.shard_range(10, 3, 3)


def test_single_process_exchange_is_identity():
    ids = torch.arange(6).view(2, 3)
    d = torch.zeros(2, 3)
    gi, gd = shards.exchange(ids, d)
    assert gi.shape == (1, 2, 3) and (gi[0] == ids).all()
    assert shards.offsets(7) == [7]
