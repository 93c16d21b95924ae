"""GPU tests of the learned angle predictor (extension; not in the paper).

* gradients of the hand-written training kernels against the FP64 oracle's
  analytic gradients (which are pinned by finite differences), same BF16
  weights and inputs;
* harvested features and targets against the oracle's definitions computed on
  the same (query, centre, neighbour) triples;
* the MLP-gated search against the oracle's MLP-gated Algorithm 4 with the same
  (seeded, oracle-initialised) predictor, on every estimate and with the
  predictor gated to the margin around ub;
* what training buys: on held-out harvested triples the trained network's
  cosine error is below that of distribution matching.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_11408_gb300 as fg  # noqa: E402


@pytest.fixture(scope="module")
def deep_like():
    """3,000 unit vectors, m = 96, 128-cluster mixture (configuration 4's
    distribution), HNSW M = 16, r = 24 (28 predictor inputs)."""
    X = workloads.base_vectors(4, 3000)
    Q = workloads.query_vectors(4, 120)
    g = oracle.hnsw_build(X, 16, 80, 3004)
    fp, _ = oracle.build_tables(X, g, 24, 4004)
    ix = fg.Index(X)
    ix.set_graph(g.adj0, g.level, g.up_off, g.up_adj, g.entry, g.maxlevel, g.M)
    ix.build_tables(24, 4004, basis=fp.P, stats=fp.stats())
    yield X, Q, g, fp, ix
    ix.close()


def test_training_gradients_match_oracle(deep_like):
    X, Q, g, fp, ix = deep_like
    nf = 28
    rng = np.random.default_rng(7)
    w = mlp.quantize_weights(mlp.init(nf, 11) + rng.normal(0, 0.02, mlp.n_weights(nf)), nf)
    F = rng.standard_normal((512, nf)).astype(np.float32)
    T = rng.uniform(-1, 1, 512).astype(np.float32)
    loss_g, grad_g = ix.mlp_loss_grad(w.astype(np.float32), torch.from_numpy(F).cuda(),
                                      torch.from_numpy(T).cuda())
    loss_o, grad_o = mlp.loss_and_grad(w, F.astype(np.float64), T.astype(np.float64), nf, True)
    assert loss_g == pytest.approx(loss_o, rel=1e-4)
    scale = np.abs(grad_o).max()
    np.testing.assert_allclose(grad_g, grad_o, rtol=1e-3, atol=1e-4 * scale)


def test_harvest_features_match_oracle(deep_like):
    X, Q, g, fp, ix = deep_like
    ix.set_mode(fg.MODE_FINGER, 5)
    feat, tgt, trip = ix.harvest(torch.from_numpy(Q).cuda(), 40, 100000)
    n = feat.shape[0]
    assert n > 1000
    feat, tgt, trip = feat.cpu().numpy(), tgt.cpu().numpy(), trip.cpu().numpy()
    sel = np.random.default_rng(3).choice(n, 300, replace=False)
    for i in sel:
        qi, c, d = trip[i]
        f, t = mlp.features(Q[qi], X[c], X[d], fp.P)
        np.testing.assert_allclose(feat[i], f, atol=2e-4, rtol=1e-3)
        assert tgt[i] == pytest.approx(t, abs=3e-3)


def test_mlp_search_matches_oracle(deep_like):
    """Same predictor on both sides (oracle-initialised, BF16-valued weights):
    the MLP-gated traversal equals the oracle's on >= 99 % of the queries."""
    X, Q, g, fp, ix = deep_like
    nf = 28
    w = mlp.init(nf, 21) * 0.3
    w[-1] = fp.mu                       # predictions scatter around the mean cosine
    wq = mlp.quantize_weights(w, nf)
    eps = float(np.float32(fp.eps))
    ix.set_predictor(wq.astype(np.float32), eps)
    ix.set_mode(fg.MODE_FINGER_MLP, 5)
    q = torch.from_numpy(Q).cuda()
    gt, _ = oracle.bruteforce(X, Q, 10)
    # delta < 0: the predictor on every estimate; delta >= 0: only where the
    # matched estimate lies within delta * ub of ub (the gated rule)
    for delta in (-1.0, 0.1, 0.3):
        ix.set_predictor_gate(delta)
        for ef in (20, 60):
            cnt = torch.zeros((Q.shape[0], 8), dtype=torch.int32, device="cuda")
            ix.set_counters(cnt)
            ids, d = ix.search(q, 10, ef)
            torch.cuda.synchronize()
            ix.sync()
            ix.set_counters(None)
            gi, gd, gc = ids.cpu().numpy(), d.cpu().numpy(), cnt.cpu().numpy()
            oi, od, oc = oracle.search(g, X, Q, 10, ef, fp, mlp_weights=wq, mlp_eps=eps,
                                       mlp_delta=delta)
            match = (gi == oi).all(axis=1)
            assert match.mean() >= 0.99, (delta, ef, match.mean())
            np.testing.assert_allclose(gd[match], od[match], rtol=1e-5)
            same = (gc[match][:, :7] == oc[match][:, :7]).all(axis=1)
            assert same.mean() >= 0.97, (delta, ef, same.mean())
            assert oc[:, 3].sum() > 0                       # the gate skips
            assert abs(oracle.recall(gi, gt, 10) - oracle.recall(oi, gt, 10)) <= 0.002
    ix.set_predictor_gate(-1.0)


def test_trained_predictor_beats_matching(deep_like):
    """Harvest on training queries (a seed disjoint from the test queries),
    train on the GPU, then compare cosine errors on held-out triples."""
    X, Q, g, fp, ix = deep_like
    ix.set_mode(fg.MODE_FINGER, 5)
    Qtr = np.random.default_rng(99).standard_normal((400, X.shape[1])).astype(np.float32)
    Qtr = X[np.random.default_rng(98).choice(X.shape[0], 400)] + 0.05 * Qtr
    Qtr = (Qtr / np.linalg.norm(Qtr, axis=1, keepdims=True)).astype(np.float32)
    feat, tgt, _ = ix.harvest(torch.from_numpy(Qtr).cuda(), 60, 200000)
    n = feat.shape[0]
    n_val = n // 5
    losses = ix.train_predictor(feat.contiguous(), tgt.contiguous(), n_val, epochs=12,
                                batch=2048, lr=2e-3, seed=5004)
    assert losses[-1] < losses[0]
    w, eps = ix.get_predictor()
    assert eps > 0
    fv, tv = feat[n - n_val:].contiguous(), tgt[n - n_val:].cpu().numpy()
    pred = ix.mlp_predict(fv).cpu().numpy()
    that = fv[:, 24].cpu().numpy()
    ratio = fp.sigma / fp.sigma_hat
    matched = (that - fp.mu_hat) * ratio + fp.mu
    mae_mlp = np.abs(pred - tv).mean()
    mae_match = np.abs(matched - tv).mean()
    assert mae_mlp < mae_match, (mae_mlp, mae_match)
    # the trained predictor also runs in the search without faults
    ix.set_mode(fg.MODE_FINGER_MLP, 5)
    ids, _ = ix.search(torch.from_numpy(Q).cuda(), 10, 40)
    ix.sync()
    gt, _ = oracle.bruteforce(X, Q, 10)
    assert oracle.recall(ids.cpu().numpy(), gt, 10) > 0.8
