"""Oracle parity at the benchmark's kernel instance.

Workload: a 20,000-row prefix of the SIFT-like integer mixture (64 clusters,
per-dimension gamma draws rounded to 0..255, m = 128: many exact distance
ties), 500 fresh queries, HNSW M = 16 (layer-0 degree 32), efConstruction
200, built by the oracle; FINGER rank 64.  This is the kernel variant the
benchmark times at full size: exact rows on 16 lanes x 2 chunks, edge rows on
16 lanes with the transpose-reduce of the row sums.

1. FINGER (Algorithm 4; FP32, binary16 and FP8 codes) and plain search
   (Algorithm 1) at ef 40 and 140 against the oracle, with the oracle's basis
   and matching statistics.
2. The product path: FINGER tables built on the device from the graph alone
   (its own pair draw, D_res Gram matrix, Jacobi basis and statistics,
   Algorithm 2), then FINGER search, against oracle.build_tables followed by
   oracle.search.
3. Uneven batches: per-query K in {1, 10, 100} and ef in [max(K, 10), 400] in
   one finger_search_batch launch, against oracle.search of each query.

Bars: tests/parity_util.py.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import parity_util
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_11408_gb300 as fg  # noqa: E402

N, NQ, R = 20_000, 500, 64


@pytest.fixture(scope="module")
def sift_like():
    X = workloads.base_vectors(2, N)
    Q = workloads.query_vectors(2, NQ)
    g = oracle.hnsw_build(X, 16, 200, 3002)
    fp, _ = oracle.build_tables(X, g, R, 4002)
    gt, _ = oracle.bruteforce(X, Q, 100)
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(R, 4002, basis=fp.P, stats=fp.stats(), half_codes=True, fp8_codes=True)
    q = torch.from_numpy(Q).cuda()
    yield dict(X=X, Q=Q, g=g, fp=fp, gt=gt, ix=ix, q=q)
    ix.close()


@pytest.mark.parametrize("ef", [40, 140])
@pytest.mark.parametrize("mode", [fg.MODE_PLAIN, fg.MODE_FINGER, fg.MODE_FINGER_F16,
                                  fg.MODE_FINGER_F8])
def test_benchmark_instance_parity(sift_like, mode, ef):
    s = sift_like
    gi, gd, gc = parity_util.gpu_search(s["ix"], s["q"], 10, ef, mode)
    fp = {fg.MODE_PLAIN: None, fg.MODE_FINGER: s["fp"],
          fg.MODE_FINGER_F16: dataclasses.replace(s["fp"], codes=16),
          fg.MODE_FINGER_F8: dataclasses.replace(s["fp"], codes=8)}[mode]
    oi, od, oc = oracle.search(s["g"], s["X"], s["Q"], 10, ef, fp)
    parity_util.compare(gi, gd, gc, oi, od, oc, s["gt"][:, :10], 10,
                        f"mode {mode} m=128 r=64 ef={ef}")
    if fp is not None:
        assert gc[:, 3].sum() > 0.5 * gc[:, 2].sum()   # most estimates skip


def test_device_built_tables_product_path(sift_like):
    """Algorithm 2 on the device, then Algorithm 4, against the same two steps
    in the oracle.  The device basis equals the oracle's up to column signs
    and FP32 rounding of the D_res Gram matrix, so the sign-invariant
    statistics agree closely and the searches meet the parity bars."""
    s = sift_like
    ix = fg.Index(s["X"])
    g = s["g"]
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(R, 4002)
    st = ix.stats()
    fp = s["fp"]
    for k, want in (("mu", fp.mu), ("sigma", fp.sigma), ("mu_hat", fp.mu_hat),
                    ("sigma_hat", fp.sigma_hat), ("eps", fp.eps)):
        assert st[k] == pytest.approx(want, rel=1e-4, abs=1e-6), k
    for ef in (40, 140):
        gi, gd, gc = parity_util.gpu_search(ix, s["q"], 10, ef, fg.MODE_FINGER)
        oi, od, oc = oracle.search(g, s["X"], s["Q"], 10, ef, fp)
        parity_util.compare(gi, gd, gc, oi, od, oc, s["gt"][:, :10], 10,
                            f"device tables ef={ef}")
    ix.close()


@pytest.mark.parametrize("mode", [fg.MODE_PLAIN, fg.MODE_FINGER, fg.MODE_FINGER_F8])
def test_uneven_batch_matches_oracle(sift_like, mode):
    s = sift_like
    ix = s["ix"]
    rng = np.random.default_rng(7)
    nq = 300
    K = rng.choice(np.array([1, 10, 100], np.int32), nq)
    ef = np.array([rng.integers(max(k, 10), 401) for k in K], np.int32)
    ix.set_mode(mode, 5)
    q = s["q"][:nq]
    ids, d, off = ix.search_batch(q, torch.from_numpy(K).cuda(), torch.from_numpy(ef).cuda())
    torch.cuda.synchronize()
    ix.sync()
    ids, d, off = ids.cpu().numpy(), d.cpu().numpy(), off.cpu().numpy()
    fp = {fg.MODE_PLAIN: None, fg.MODE_FINGER: s["fp"],
          fg.MODE_FINGER_F8: dataclasses.replace(s["fp"], codes=8)}[mode]
    same, hits_g, hits_o, tot, worst = 0, 0, 0, 0, 0.0
    for i in range(nq):
        k = int(K[i])
        oi, od, _ = oracle.search(s["g"], s["X"], s["Q"][i:i + 1], k, int(ef[i]), fp)
        oi = parity_util.fp32_canonical(oi, od)[0]
        od = np.sort(od[0])
        gi, gdi = ids[off[i]:off[i] + k], d[off[i]:off[i] + k]
        if (gi == oi).all():
            same += 1
            ok = oi >= 0
            worst = max(worst, float((np.abs(gdi[ok] - od[ok]) / np.maximum(od[ok], 1e-30)).max()))
        gt = set(s["gt"][i, :k].tolist())
        hits_g += len(gt & set(gi.tolist()))
        hits_o += len(gt & set(oi.tolist()))
        tot += k
    print(f"uneven batch mode {mode}: lists identical {same / nq:.4f}, "
          f"recall {hits_g / tot:.4f} vs oracle {hits_o / tot:.4f}")
    assert same / nq >= 0.99
    assert worst < parity_util.REL
    assert abs(hits_g - hits_o) / tot <= 0.002
