"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Workload: the 10,000-point, 64-dimensional 16-cluster Gaussian mixture with
200 queries, an HNSW graph (M = 16, efConstruction = 100) built by the oracle,
FINGER rank 16.  Bars (tests/parity_util.py): result lists identical to the
oracle on >= 99 % of queries, per-pair distances within 1e-5 relative of FP64,
recall@10 within 0.002 of the oracle's at the same ef, traversal counters
identical on >= 97 % of the queries whose lists match.
"""
import dataclasses
import json
import os

import numpy as np
import pytest

import oracle
import parity_util
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_11408_gb300 as fg  # noqa: E402

REL = 1e-5


@pytest.fixture(scope="module")
def cfg1():
    X = workloads.base_vectors(1)
    Q = workloads.query_vectors(1)
    g = oracle.hnsw_build(X, 16, 100, 3001)
    fp, pairs = oracle.build_tables(X, g, 16, 4001)
    gt, gd = oracle.bruteforce(X, Q, 10)
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(16, 4001, basis=fp.P, stats=fp.stats(), half_codes=True, fp8_codes=True)
    q = torch.from_numpy(Q).cuda()
    yield dict(X=X, Q=Q, g=g, fp=fp, pairs=pairs, gt=gt, gd=gd, ix=ix, q=q)
    ix.close()


_gpu_search = parity_util.gpu_search
_compare = parity_util.compare


def _f16(fp):
    """The oracle's FINGER parameters with the per-edge codes stored as binary16."""
    return dataclasses.replace(fp, codes=16)


def _f8(fp, deg0=32):
    """The oracle's FINGER parameters with the per-edge codes stored as FP8 E4M3
    codes of 256 u: u_q split into E4M3 parts where the kernel multiplies in
    FP8 (at most four products per code block: not both deg0 > 32 and r > 32),
    else u_q itself."""
    tiles, kp = (4 if deg0 > 32 else 2), (2 if fp.P.shape[0] > 32 else 1)
    return dataclasses.replace(fp, codes=8 if tiles * kp <= 4 else 9)


def _modes(fp, deg0=32):
    return ((fg.MODE_PLAIN, None), (fg.MODE_FINGER, fp), (fg.MODE_FINGER_F16, _f16(fp)),
            (fg.MODE_FINGER_F8, _f8(fp, deg0)))


def test_bruteforce_knn_matches_oracle(cfg1):
    ids, d = cfg1["ix"].knn(cfg1["q"], 10)
    torch.cuda.synchronize()
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    assert (ids == cfg1["gt"]).mean() > 0.999
    np.testing.assert_allclose(d, cfg1["gd"], rtol=REL)


@pytest.mark.parametrize("ef", [10, 20, 50, 100])
def test_plain_search_parity(cfg1, ef):
    gi, gd, gc = _gpu_search(cfg1["ix"], cfg1["q"], 10, ef, fg.MODE_PLAIN)
    oi, od, oc = oracle.search(cfg1["g"], cfg1["X"], cfg1["Q"], 10, ef)
    _compare(gi, gd, gc, oi, od, oc, cfg1["gt"], 10, f"plain ef={ef}")


@pytest.mark.parametrize("ef", [10, 20, 50, 100])
def test_finger_search_parity(cfg1, ef):
    gi, gd, gc = _gpu_search(cfg1["ix"], cfg1["q"], 10, ef, fg.MODE_FINGER)
    oi, od, oc = oracle.search(cfg1["g"], cfg1["X"], cfg1["Q"], 10, ef, cfg1["fp"])
    _compare(gi, gd, gc, oi, od, oc, cfg1["gt"], 10, f"finger ef={ef}")
    assert gc[:, 3].sum() > 0          # the gate skipped neighbours


@pytest.mark.parametrize("ef", [10, 20, 50, 100])
def test_finger_f16_search_parity(cfg1, ef):
    """FINGER with the codes stored as binary16 (whole code block read with the
    adjacency row) against the oracle's Algorithm 4 on binary16 codes."""
    gi, gd, gc = _gpu_search(cfg1["ix"], cfg1["q"], 10, ef, fg.MODE_FINGER_F16)
    oi, od, oc = oracle.search(cfg1["g"], cfg1["X"], cfg1["Q"], 10, ef, _f16(cfg1["fp"]))
    _compare(gi, gd, gc, oi, od, oc, cfg1["gt"], 10, f"finger-f16 ef={ef}")
    assert gc[:, 3].sum() > 0


@pytest.mark.parametrize("ef", [10, 20, 50, 100])
def test_finger_f8_search_parity(cfg1, ef):
    """FINGER with FP32 rows and the codes stored as FP8 E4M3 of 256 u against
    the oracle's Algorithm 4 on the same FP8 codes."""
    gi, gd, gc = _gpu_search(cfg1["ix"], cfg1["q"], 10, ef, fg.MODE_FINGER_F8)
    oi, od, oc = oracle.search(cfg1["g"], cfg1["X"], cfg1["Q"], 10, ef, _f8(cfg1["fp"]))
    _compare(gi, gd, gc, oi, od, oc, cfg1["gt"], 10, f"finger-f8 ef={ef}")
    assert gc[:, 3].sum() > 0


def test_alg4_hand_trace_on_gpu():
    """The hand-traced Algorithm 4 instance (tests/golden/alg4_hand_trace.json:
    one estimate exactly equal to ub) through the FINGER modes of the kernel
    (r = 1: the unit codes are +-1, exact in FP16 and, as 256, in FP8)."""
    t = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "alg4_hand_trace.json")))
    names = sorted(t["ids"], key=t["ids"].get)
    X = np.array([t["points"][k] for k in names], np.float32)
    adj = np.full((len(names), 2), -1, np.int32)
    for k in names:
        row = [t["ids"][v] for v in t["adjacency"][k]]
        adj[t["ids"][k], :len(row)] = row
    st = t["stats"]
    stats = [st["mu"], st["sigma"], st["mu_hat"], st["sigma_hat"], st["eps"]]
    ix = fg.Index(X)
    ix.set_graph(adj, np.zeros(len(names), np.int32), np.full(len(names), -1, np.int64),
                 np.zeros((0, 1), np.int32), t["ids"][t["entry"]], 0, 1)
    ix.build_tables(1, 1, basis=np.array(t["P"], np.float32), stats=stats, half_codes=True, fp8_codes=True)
    q = torch.tensor([t["query"]], dtype=torch.float32, device="cuda")
    for mode in (fg.MODE_FINGER, fg.MODE_FINGER_F16, fg.MODE_FINGER_F8):
        for key, warmup in (("warmup1_strict", 1), ("warmup2_strict", 2)):
            exp = t["expected"][key]
            ids, d, c = _gpu_search(ix, q, t["K"], t["ef"], mode, warmup)
            assert [names[i] for i in ids[0]] == exp["ids"], (mode, key)
            assert d[0].tolist() == exp["dists"], (mode, key)
            got = dict(zip(fg.COUNTER_NAMES, c[0].tolist()))
            for k in ("expansions", "examined", "estimates", "skipped", "exact", "admitted"):
                assert got[k] == exp[k], (mode, key, k, got[k], exp[k])
    ix.close()


def test_finger_without_skipping_equals_plain(cfg1):
    a = _gpu_search(cfg1["ix"], cfg1["q"], 10, 50, fg.MODE_PLAIN)
    b = _gpu_search(cfg1["ix"], cfg1["q"], 10, 50, fg.MODE_FINGER, warmup=10 ** 9)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()
    assert (a[2][:, [0, 1, 4, 5, 6]] == b[2][:, [0, 1, 4, 5, 6]]).all()


def test_search_host_equals_device(cfg1):
    ix = cfg1["ix"]
    ix.set_mode(fg.MODE_FINGER, 5)
    ids, d = ix.search(cfg1["q"], 10, 50)
    hi, hd = ix.search_host(cfg1["Q"], 10, 50)
    assert (ids.cpu().numpy() == hi).all() and (d.cpu().numpy() == hd).all()


def test_edge_tables_match_oracle(cfg1):
    t = cfg1["ix"].get_tables()
    X, g, fp = cfg1["X"], cfg1["g"], cfg1["fp"]
    nodes = np.arange(0, X.shape[0], 7)
    u, dn, b = oracle.edge_tables(X, g.adj0, fp.P, nodes)
    np.testing.assert_allclose(t["b"][nodes], b, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(t["dres_norm"][nodes], dn, rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(t["edge_u"][nodes], u, atol=2e-5)
    Pc = X[nodes].astype(np.float64) @ fp.P.T
    np.testing.assert_allclose(t["node_proj"][nodes], Pc, rtol=1e-5, atol=1e-5)


def test_matching_stats_match_oracle(cfg1):
    """GPU statistics from the oracle's basis vs the oracle's own (FP64)."""
    X, g, fp = cfg1["X"], cfg1["g"], cfg1["fp"]
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(16, 4001, basis=fp.P)
    st = ix.get_tables()["stats"]
    np.testing.assert_allclose(st, fp.stats(), rtol=1e-5, atol=1e-6)
    ix.close()


def test_device_basis_is_the_svd_basis(cfg1):
    """P from the device Gram + Jacobi spans the top-r left singular subspace:
    orthonormal rows, captured energy equal to the sum of the r largest
    eigenvalues of the oracle's Gram matrix (Proposition 1)."""
    X, g, fp, pairs = cfg1["X"], cfg1["g"], cfg1["fp"], cfg1["pairs"]
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(16, 4001)
    t = ix.get_tables()
    P = t["P"].astype(np.float64)
    np.testing.assert_allclose(P @ P.T, np.eye(16), atol=1e-5)
    G = oracle.gram(X, pairs)
    w = np.sort(np.linalg.eigvalsh(G))[::-1]
    energy = np.trace(P @ G @ P.T)
    assert energy == pytest.approx(w[:16].sum(), rel=1e-5)
    gap = (w[15] - w[16]) / w[0]
    if gap > 1e-3:
        np.testing.assert_allclose(P.T @ P, fp.P.T @ fp.P, atol=1e-3)
    np.testing.assert_allclose(t["stats"], fp.stats(), rtol=2e-3, atol=1e-4)
    ix.close()


def test_full_rank_finger_equals_plain(cfg1):
    X, g = cfg1["X"], cfg1["g"]
    fpf, _ = oracle.build_tables(X, g, 64, 4001)
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(64, 4001, basis=fpf.P, stats=fpf.stats())
    a = _gpu_search(ix, cfg1["q"], 10, 50, fg.MODE_PLAIN)
    b = _gpu_search(ix, cfg1["q"], 10, 50, fg.MODE_FINGER)
    assert (a[0] == b[0]).all(axis=1).mean() >= 0.99
    assert b[2][:, 2].sum() > 0
    ix.close()


def test_limits_and_padding(cfg1):
    ix = cfg1["ix"]
    with pytest.raises(fg.FingerError):
        ix.search(cfg1["q"], 10, 5)                     # K > ef
    ids, d = ix.search(cfg1["q"][:0], 10, 20)           # empty batch
    assert ids.shape == (0, 10)
    small = fg.Index(cfg1["X"][:5])
    adj = np.full((5, 4), -1, np.int32)
    adj[:, :2] = [[1, 2], [0, 2], [0, 1], [4, -1], [3, -1]]
    small.set_graph(adj, np.zeros(5, np.int32), np.full(5, -1, np.int64),
                    np.zeros((0, 2), np.int32), 0, 0, 2)
    small.set_mode(fg.MODE_PLAIN)
    ids, d = small.search(cfg1["q"][:3], 8, 8)          # only 3 nodes reachable
    ids = ids.cpu().numpy()
    assert (ids[:, 3:] == -1).all() and set(ids[0, :3]) == {0, 1, 2}
    assert torch.isinf(d[:, 3:]).all()
    small.close()


def test_ragged_batch_and_odd_dimension():
    X = workloads.base_vectors(1, 1500)[:, :50].copy()      # m = 50, not a multiple of 4
    Q = workloads.query_vectors(1, 203)[:, :50].copy()
    g = oracle.hnsw_build(X, 12, 60, 99)                   # deg0 = 24
    fp, _ = oracle.build_tables(X, g, 10, 5)
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(10, 5, basis=fp.P, stats=fp.stats(), half_codes=True, fp8_codes=True)
    q = torch.from_numpy(Q).cuda()
    for mode, f in _modes(fp):
        gi, gd, gc = _gpu_search(ix, q, 7, 33, mode)
        oi, od, oc = oracle.search(g, X, Q, 7, 33, f)
        gt, _ = oracle.bruteforce(X, Q, 7)
        _compare(gi, gd, gc, oi, od, oc, gt, 7, f"m=50 mode={mode}")
    ix.close()


def test_two_neighbour_slots_per_lane():
    """deg0 = 48 > 32 (two neighbour slots per lane), M = 24."""
    X = workloads.base_vectors(1, 3000)
    Q = workloads.query_vectors(1, 100)
    g = oracle.hnsw_build(X, 24, 80, 11)
    fp, _ = oracle.build_tables(X, g, 16, 12)
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(16, 12, basis=fp.P, stats=fp.stats(), half_codes=True, fp8_codes=True)
    q = torch.from_numpy(Q).cuda()
    gt, _ = oracle.bruteforce(X, Q, 10)
    for mode, f in _modes(fp):
        gi, gd, gc = _gpu_search(ix, q, 10, 64, mode)
        oi, od, oc = oracle.search(g, X, Q, 10, 64, f)
        _compare(gi, gd, gc, oi, od, oc, gt, 10, f"deg0=48 mode={mode}")
    ix.close()


def test_wide_rows_k1_and_ef_equal_k():
    """m = 300 (the GIST-like distribution's first 300 coordinates): every lane
    holds several 16-byte chunks of a row; K = 1 and ef = K are the smallest
    result and candidate lists."""
    X = np.ascontiguousarray(workloads.base_vectors(5, 2500)[:, :300])
    Q = np.ascontiguousarray(workloads.query_vectors(5, 120)[:, :300])
    g = oracle.hnsw_build(X, 16, 60, 21)
    fp, _ = oracle.build_tables(X, g, 32, 22)
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(32, 22, basis=fp.P, stats=fp.stats(), half_codes=True, fp8_codes=True)
    q = torch.from_numpy(Q).cuda()
    for K, ef in ((1, 1), (1, 16), (10, 10), (10, 48)):
        gt, _ = oracle.bruteforce(X, Q, K)
        for mode, f in _modes(fp):
            gi, gd, gc = _gpu_search(ix, q, K, ef, mode)
            oi, od, oc = oracle.search(g, X, Q, K, ef, f)
            _compare(gi, gd, gc, oi, od, oc, gt, K, f"m=300 K={K} ef={ef} mode={mode}")
    ix.close()


def test_wide_codes_two_row_groups():
    """deg0 = 64 (M = 32) with r = 64: the FP16 code block of a centre is 16
    loads per lane, taken as two row groups of eight (the second once the
    first is consumed)."""
    X = workloads.base_vectors(2, 3000)
    Q = workloads.query_vectors(2, 100)
    g = oracle.hnsw_build(X, 32, 100, 41)
    fp, _ = oracle.build_tables(X, g, 64, 42)
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(64, 42, basis=fp.P, stats=fp.stats(), half_codes=True, fp8_codes=True)
    assert ix.info()["deg0"] == 64
    q = torch.from_numpy(Q).cuda()
    gt, _ = oracle.bruteforce(X, Q, 10)
    for mode, f in _modes(fp, 64)[1:]:
        gi, gd, gc = _gpu_search(ix, q, 10, 80, mode)
        oi, od, oc = oracle.search(g, X, Q, 10, 80, f)
        _compare(gi, gd, gc, oi, od, oc, gt, 10, f"deg0=64 r=64 mode={mode}")
    # ef 2 and 4: the expansion that fills T leaves up to 63 new neighbours for
    # the gate replay, most of them below ub, so expansions with 32 or more
    # candidates take the serial replay
    gt2, _ = oracle.bruteforce(X, Q, 2)
    for ef in (2, 4):
        for mode, f in _modes(fp, 64):
            gi, gd, gc = _gpu_search(ix, q, 2, ef, mode)
            oi, od, oc = oracle.search(g, X, Q, 2, ef, f)
            _compare(gi, gd, gc, oi, od, oc, gt2, 2, f"deg0=64 ef={ef} mode={mode}")
    ix.close()


def test_flat_graph_parity_and_device_builder():
    """FINGER over a non-HNSW graph (single layer, entry node 0): parity with
    the oracle on the oracle's flat graph; the device builder's flat graph has
    no hierarchy and is searchable."""
    X = workloads.base_vectors(1, 4000)
    Q = workloads.query_vectors(1, 150)
    g = oracle.hnsw_build(X, 16, 80, 31, flat=True)
    fp, _ = oracle.build_tables(X, g, 16, 32)
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(16, 32, basis=fp.P, stats=fp.stats())
    q = torch.from_numpy(Q).cuda()
    gt, _ = oracle.bruteforce(X, Q, 10)
    for mode, f in ((fg.MODE_PLAIN, None), (fg.MODE_FINGER, fp)):
        gi, gd, gc = _gpu_search(ix, q, 10, 50, mode)
        oi, od, oc = oracle.search(g, X, Q, 10, 50, f)
        _compare(gi, gd, gc, oi, od, oc, gt, 10, f"flat mode={mode}")
    ix.build_graph(16, 80, 31, flat=True)
    gg = ix.get_graph()
    assert (gg["level"] == 0).all() and gg["maxlevel"] == 0 and gg["entry"] == 0
    ix.build_tables(16, 32)
    ix.set_mode(fg.MODE_FINGER)
    ids, _ = ix.search(q, 10, 100)
    ix.sync()
    assert oracle.recall(ids.cpu().numpy(), gt, 10) > 0.9
    ix.close()


@pytest.mark.parametrize("m,K", [(64, 10), (64, 1), (64, 40), (64, 64), (50, 10), (300, 16)])
def test_bruteforce_paths_match_oracle(m, K):
    """Exact kNN on the tensor cores (K <= 40: BF16 split products in tensor
    memory, FP32 re-rank) and on FFMA (K > 40), against the FP64 oracle; n and
    nq not multiples of the 128-row tiles, m = 50 (zero-filled K tail) and
    m = 300 (five K chunks)."""
    cfg = 5 if m > 64 else 1
    X = np.ascontiguousarray(workloads.base_vectors(cfg, 3001)[:, :m])
    Q = np.ascontiguousarray(workloads.query_vectors(cfg, 77)[:, :m])
    ix = fg.Index(X)
    ids, d = ix.knn(torch.from_numpy(Q).cuda(), K)
    torch.cuda.synchronize()
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    gt, gd = oracle.bruteforce(X, Q, K)
    assert (ids == gt).mean() > 0.999, (ids != gt).sum()
    np.testing.assert_allclose(d, gd, rtol=REL)
    ix.close()


@pytest.mark.parametrize("bits", [0, 32])
def test_maximum_ef_and_k(cfg1, bits):
    """ef at the compiled maximum (1024) and K = 256 on the 10,000-point index:
    the result list holds 1024 entries, most visits go through the spill path
    (and, with 16-bit slots, through full probe sequences), and the traversal
    still equals the oracle's with either visited-set slot width."""
    q = cfg1["q"][:40]
    Q = cfg1["Q"][:40]
    gt, _ = oracle.bruteforce(cfg1["X"], Q, 256)
    cfg1["ix"].set_visited_slots(bits)
    try:
        for mode, f in ((fg.MODE_PLAIN, None), (fg.MODE_FINGER, cfg1["fp"])):
            gi, gd, gc = _gpu_search(cfg1["ix"], q, 256, 1024, mode)
            oi, od, oc = oracle.search(cfg1["g"], cfg1["X"], Q, 256, 1024, f)
            _compare(gi, gd, gc, oi, od, oc, gt, 256, f"ef=1024 K=256 mode={mode} bits={bits}")
    finally:
        cfg1["ix"].set_visited_slots(0)
    with pytest.raises(fg.FingerError):
        cfg1["ix"].search(q, 10, 1025)                  # above the compiled maximum


@pytest.mark.parametrize("ef", [20, 100])
def test_visited_slot_widths_give_the_same_traversal(cfg1, ef):
    """The visited set is exact with 16-bit and with 32-bit slots, so plain and
    FINGER search return identical lists, distances and counters; the 32-bit
    tables also meet the oracle bars."""
    ix = cfg1["ix"]
    for mode, f in ((fg.MODE_PLAIN, None), (fg.MODE_FINGER, cfg1["fp"])):
        a = _gpu_search(ix, cfg1["q"], 10, ef, mode)
        ix.set_visited_slots(32)
        try:
            b = _gpu_search(ix, cfg1["q"], 10, ef, mode)
        finally:
            ix.set_visited_slots(0)
        for x, y in zip(a, b):
            assert (x == y).all()
        oi, od, oc = oracle.search(cfg1["g"], cfg1["X"], cfg1["Q"], 10, ef, f)
        _compare(*b, oi, od, oc, cfg1["gt"], 10, f"32-bit slots mode={mode} ef={ef}")
    with pytest.raises(fg.FingerError):
        ix.set_visited_slots(16)
