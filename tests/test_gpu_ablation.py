"""GPU parity of the ablation switches (Sec. 4.3) and of the rank rule
(Supplementary E) against the FP64 oracle, on the oracle's own HNSW graph of
the 10,000-point, 64-dimensional Gaussian mixture.

* statistics (mu, sigma, mu_hat, sigma_hat, eps) and corr(X, Y) of the device
  build for the full method, no matching, no eps, and a random Gaussian
  (RPLSH) basis passed in, against the oracle's on the same drawn pairs;
* FINGER search with the ablated statistics against the oracle's search;
* the rank rule picks the same rank with the same correlations;
* a rebuild at another rank reuses the cached eigenvectors: the basis of rank
  8 is the first 8 rows of the basis of rank 16, and rebuilding at 16 gives
  bit-identical tables.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_11408_gb300 as fg  # noqa: E402

STAT_TOL = 2e-5


@pytest.fixture(scope="module")
def cfg1():
    X = workloads.base_vectors(1)
    Q = workloads.query_vectors(1)
    g = oracle.hnsw_build(X, 16, 100, 3001)
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    q = torch.from_numpy(Q).cuda()
    yield dict(X=X, Q=Q, g=g, ix=ix, q=q)
    ix.close()


def _gpu_stats(ix):
    s = ix.stats()
    return np.array([s["mu"], s["sigma"], s["mu_hat"], s["sigma_hat"], s["eps"]]), s["corr"]


@pytest.mark.parametrize("variant", ["full", "no_matching", "no_eps", "rplsh", "rplsh_no_matching"])
def test_ablation_stats_match_oracle(cfg1, variant):
    X, g, ix = cfg1["X"], cfg1["g"], cfg1["ix"]
    r = 16
    basis = None
    if variant.startswith("rplsh"):
        basis = np.random.default_rng(17).standard_normal((r, X.shape[1]))
    matching = "no_matching" not in variant
    use_eps = variant != "no_eps"
    fp, _ = oracle.build_tables(X, g, r, 4001, basis=basis, matching=matching, use_eps=use_eps)
    ix.build_tables(r, 4001, basis=basis, matching=matching, use_eps=use_eps)
    st, corr = _gpu_stats(ix)
    np.testing.assert_allclose(st, fp.stats(), atol=STAT_TOL)
    assert corr == pytest.approx(fp.corr, abs=STAT_TOL)
    if not matching:
        assert tuple(st[:4]) == (0.0, 1.0, 0.0, 1.0)
    if not use_eps:
        assert st[4] == 0.0


@pytest.mark.parametrize("variant", ["no_matching", "rplsh"])
def test_ablated_search_matches_oracle(cfg1, variant):
    """Same basis and statistics on both sides (the oracle's), FINGER search
    lists identical on >= 99 % of the queries, recall within 0.002."""
    X, Q, g, ix, q = cfg1["X"], cfg1["Q"], cfg1["g"], cfg1["ix"], cfg1["q"]
    r = 16
    basis = None
    if variant == "rplsh":
        basis = np.random.default_rng(17).standard_normal((r, X.shape[1]))
    fp, _ = oracle.build_tables(X, g, r, 4001, basis=basis, matching=variant != "no_matching")
    ix.build_tables(r, 4001, basis=fp.P, stats=fp.stats())
    gt, _ = oracle.bruteforce(X, Q, 10)
    ix.set_mode(fg.MODE_FINGER, 5)
    for ef in (20, 60):
        ids, d = ix.search(q, 10, ef)
        ix.sync()
        gi, gd = ids.cpu().numpy(), d.cpu().numpy()
        oi, od, oc = oracle.search(g, X, Q, 10, ef, fp)
        match = (gi == oi).all(axis=1)
        assert match.mean() >= 0.99, (variant, ef, match.mean())
        np.testing.assert_allclose(gd[match], od[match], rtol=1e-5)
        assert oc[:, 3].sum() > 0
        assert abs(oracle.recall(gi, gt, 10) - oracle.recall(oi, gt, 10)) <= 0.002


def test_rank_rule_matches_oracle(cfg1):
    X, g, ix = cfg1["X"], cfg1["g"], cfg1["ix"]
    r_o, trace_o = oracle.select_rank(X, g, 4001)
    r_g, trace_g = ix.select_rank(4001)
    assert len(trace_g) == len(trace_o)
    np.testing.assert_allclose(trace_g, [c for _, c in trace_o], atol=STAT_TOL)
    # the decision is the same unless a correlation sits on the threshold
    assert all(abs(c - 0.7) > 1e-3 for _, c in trace_o)
    assert r_g == r_o
    assert ix.info()["r"] == r_g
    _, corr = _gpu_stats(ix)
    assert corr == pytest.approx(trace_o[-1][1], abs=STAT_TOL)
    # an unreachable threshold walks every candidate up to r_max
    r_all, trace_all = ix.select_rank(4001, threshold=1.5, r_max=40)
    assert r_all == 40 and len(trace_all) == 5


def test_rebuild_reuses_eigenvectors(cfg1):
    ix = cfg1["ix"]
    ix.build_tables(16, 4001)
    t16 = ix.get_tables()
    ix.build_tables(8, 4001)
    t8 = ix.get_tables()
    np.testing.assert_array_equal(t8["P"], t16["P"][:8])
    ix.build_tables(16, 4001)
    t16b = ix.get_tables()
    for k in ("P", "node_proj", "edge_u", "dres_norm", "b", "stats"):
        np.testing.assert_array_equal(t16b[k], t16[k])
    # another draw seed gives another basis (the cache is keyed by the draw)
    ix.build_tables(16, 4002)
    assert not np.array_equal(ix.get_tables()["P"], t16["P"])
