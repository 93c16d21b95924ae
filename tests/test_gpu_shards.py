"""Partitioned-database search through the C ABI against the FP64 oracle.

* finger_merge_topk on the oracle's exact kNN of three uneven parts (FP32
  distances, local ids, one part smaller than K) equals the oracle's merge of
  the same lists bit for bit, pads when the parts hold fewer than K results,
  and rejects bad arguments.
* Two halves of the 10,000-point Gaussian mixture, each with its own oracle
  HNSW graph and FINGER tables: plain and FINGER search on every part, merged
  on the device, against the oracle's per-part searches merged by the oracle.
  Bars as for one index: merged lists identical on >= 99 % of queries,
  distances within 1e-5 relative of FP64, recall@10 within 0.002.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_11408_gb300 as fg  # noqa: E402

REL = 1e-5


def _fp32_canonical(oi, od):
    """Lists reordered by (FP32 distance, id): the kernels compare FP32
    distances, so FP64 values that round to the same FP32 are a tie there."""
    d32 = od.astype(np.float32)
    out = oi.copy()
    for qi in range(oi.shape[0]):
        valid = oi[qi] >= 0
        order = np.lexsort((oi[qi][valid], d32[qi][valid]))
        out[qi, :valid.sum()] = oi[qi][valid][order]
    return out


def test_device_merge_equals_oracle_merge():
    X = workloads.base_vectors(1)
    Q = workloads.query_vectors(1)
    K = 10
    cuts = [0, 7, 4000, 10000]
    parts = [oracle.bruteforce(X[lo:hi], Q, K) for lo, hi in zip(cuts[:-1], cuts[1:])]
    ids = np.stack([p[0] for p in parts])
    d32 = np.stack([p[1].astype(np.float32) for p in parts])
    oi, od = oracle.merge_topk(list(ids), list(d32), cuts[:-1], K)
    ti, td = torch.from_numpy(ids).cuda(), torch.from_numpy(d32).cuda()
    gi, gd = fg.merge_topk(ti, td, cuts[:-1])
    torch.cuda.synchronize()
    assert (gi.cpu().numpy() == oi).all()
    assert (gd.cpu().numpy() == od).all()
    # the union holds fewer than K results: padded with -1 / +inf
    small = [oracle.bruteforce(X[lo:hi], Q, K) for lo, hi in ((0, 3), (3, 7))]
    si = torch.from_numpy(np.stack([p[0] for p in small])).cuda()
    sd = torch.from_numpy(np.stack([p[1].astype(np.float32) for p in small])).cuda()
    gi, gd = fg.merge_topk(si, sd, [0, 3])
    oi, od = oracle.merge_topk([p[0] for p in small], [p[1].astype(np.float32) for p in small],
                               [0, 3], K)
    assert (gi.cpu().numpy() == oi).all() and (gd.cpu().numpy() == od).all()
    assert (oi[:, 7:] == -1).all()
    with pytest.raises(fg.FingerError):
        fg.merge_topk(ti, td, [0, -1, 5])
    with pytest.raises(ValueError):
        fg.merge_topk(ti, td, [0, 7])


@pytest.fixture(scope="module")
def two_parts():
    X = workloads.base_vectors(1)
    Q = workloads.query_vectors(1)
    cuts = [0, 5000, 10000]
    parts = []
    for p, (lo, hi) in enumerate(zip(cuts[:-1], cuts[1:])):
        Xp = X[lo:hi]
        g = oracle.hnsw_build(Xp, 16, 100, 3101 + p)
        fp, _ = oracle.build_tables(Xp, g, 16, 4101 + p)
        ix = fg.Index(Xp)
        ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
        ix.build_tables(16, 4101 + p, basis=fp.P, stats=fp.stats())
        parts.append((Xp, g, fp, ix))
    gt, _ = oracle.bruteforce(X, Q, 10)
    yield dict(X=X, Q=Q, q=torch.from_numpy(Q).cuda(), cuts=cuts, parts=parts, gt=gt)
    for p in parts:
        p[3].close()


@pytest.mark.parametrize("mode", [fg.MODE_PLAIN, fg.MODE_FINGER])
@pytest.mark.parametrize("ef", [20, 50])
def test_partitioned_search_matches_oracle(two_parts, mode, ef):
    K = 10
    offs = two_parts["cuts"][:-1]
    gids, gds, oids, ods = [], [], [], []
    for Xp, g, fp, ix in two_parts["parts"]:
        ix.set_mode(mode, 5)
        i, d = ix.search(two_parts["q"], K, ef)
        gids.append(i)
        gds.append(d)
        oi, od, _ = oracle.search(g, Xp, two_parts["Q"], K, ef,
                                  fp if mode == fg.MODE_FINGER else None)
        oids.append(oi)
        ods.append(od)
    mi, md = fg.merge_topk(torch.stack(gids), torch.stack(gds), offs)
    torch.cuda.synchronize()
    mi, md = mi.cpu().numpy(), md.cpu().numpy()
    oi, od = oracle.merge_topk(oids, ods, offs, K)
    oi = _fp32_canonical(oi, od)
    match = (mi == oi).all(axis=1)
    assert match.mean() >= 0.99, match.mean()
    ok = oi[match] >= 0
    rel = np.abs(md[match][ok] - np.sort(od, axis=1)[match][ok]) / np.maximum(
        np.sort(od, axis=1)[match][ok], 1e-30)
    assert rel.max() < REL
    r_g, r_o = oracle.recall(mi, two_parts["gt"], K), oracle.recall(oi, two_parts["gt"], K)
    assert abs(r_g - r_o) <= 0.002, (r_g, r_o)
    # global ids: every returned id is in range and lists are sorted by (distance, id)
    assert ((mi >= 0) & (mi < two_parts["X"].shape[0])).all()
    keys_sorted = (md[:, 1:] > md[:, :-1]) | ((md[:, 1:] == md[:, :-1]) & (mi[:, 1:] > mi[:, :-1]))
    assert keys_sorted.all()
