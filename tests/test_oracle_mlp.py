"""Pins of the oracle's learned angle predictor (an extension; the paper has no
learned predictor): BF16 rounding against the IEEE definition and torch's
conversion, analytic gradients against central finite differences, the
features against their defining identities, and the predictor hook of the
oracle search against predictors whose effect is known in closed form."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import mlp


def test_bf16_round_to_nearest_even():
    # spacing of bfloat16 at 1.0 is 2^-7
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1 + 2 ** -8) == 1.0                       # tie -> even mantissa
    assert mlp.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6           # tie -> even mantissa
    assert mlp.bf16(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7    # above the tie
    assert mlp.bf16(-2.5) == -2.5 and mlp.bf16(0.0) == 0.0
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).uniform(-6, 6, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    nf = 12
    w = mlp.init(nf, 3) + rng.normal(0, 0.05, mlp.n_weights(nf))
    w[mlp.H * nf:mlp.H * nf + mlp.H] = rng.normal(0, 0.5, mlp.H)     # non-zero b1
    X = rng.standard_normal((40, nf))
    t = rng.standard_normal(40)
    loss, g = mlp.loss_and_grad(w, X, t, nf, round_act=False)
    idx = rng.choice(len(w), 120, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_and_grad(wp, X, t, nf, False)[0] - mlp.loss_and_grad(wm, X, t, nf, False)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9)


def test_features_identities():
    rng = np.random.default_rng(4)
    m, r = 16, 5
    P = np.linalg.qr(rng.standard_normal((m, m)))[0][:r]
    for _ in range(20):
        q, c, d = rng.standard_normal((3, m))
        f, target = mlp.features(q, c, d, P)
        assert f[:r].sum() == pytest.approx(f[r], abs=1e-12)      # sum of products = t_hat
        cc = c @ c
        qr, dr = q - (c @ q) / cc * c, d - (c @ d) / cc * c
        assert target == pytest.approx(qr @ dr / np.linalg.norm(qr) / np.linalg.norm(dr))
        assert f[r + 1] == pytest.approx(np.linalg.norm(qr) / np.linalg.norm(q))
    # full rank: cos(P q_res, P d_res) = cos(q_res, d_res), i.e. t_hat = target
    Pf = np.linalg.qr(rng.standard_normal((m, m)))[0]
    f, target = mlp.features(q, c, d, Pf)
    assert f[m] == pytest.approx(target, abs=1e-12)


@pytest.fixture(scope="module")
def small():
    X = workloads.base_vectors(4, 2000)
    Q = workloads.query_vectors(4, 40)
    g = oracle.hnsw_build(X, 8, 60, 3004)
    fp, _ = oracle.build_tables(X, g, 8, 4004)
    return X, Q, g, fp


def _const_predictor(nf, value):
    w = np.zeros(mlp.n_weights(nf))
    w[-1] = value                           # b3: the output is this constant
    return w


def test_predictor_hook_large_cosine_is_no_skip(small):
    """A predictor that always says cos = +1e6 makes every estimate -inf-like:
    nothing is skipped and the search is Algorithm 1."""
    X, Q, g, fp = small
    nf = fp.P.shape[0] + 4
    i1, d1, c1 = oracle.search(g, X, Q, 10, 30)
    i2, d2, c2 = oracle.search(g, X, Q, 10, 30, fp, mlp_weights=_const_predictor(nf, 1e6))
    assert (i1 == i2).all() and (d1 == d2).all()
    assert c2[:, 3].sum() == 0 and c2[:, 2].sum() > 0


def test_predictor_hook_constant_equals_matching(small):
    """A constant predictor c0 with eps' = e0 gives t = c0 + e0, the same t as
    distribution matching with sigma = 0, mu = c0, eps = e0."""
    X, Q, g, fp = small
    nf = fp.P.shape[0] + 4
    c0, e0 = -0.5, 0.05
    flat = oracle.FingerParams(fp.P, c0, 0.0, 0.0, 1.0, e0)
    i1, d1, c1 = oracle.search(g, X, Q, 10, 30, flat)
    i2, d2, c2 = oracle.search(g, X, Q, 10, 30, fp, mlp_weights=_const_predictor(nf, c0),
                               mlp_eps=e0)
    assert (i1 == i2).all() and (c1 == c2).all()
    assert c1[:, 3].sum() > 0


def test_c_predictor_matches_numpy_forward():
    """The predictor inside the oracle's search (oracle.c: features assembled in
    Algorithm 3, then the r+4 -> 64 -> 64 -> 1 network) against the numpy
    definition in oracle/mlp.py, on random BF16 weights with non-zero biases
    (every layer matters), random triples and both signs of every feature."""
    rng = np.random.default_rng(11)
    m, r = 24, 6
    nf = r + 4
    P = np.linalg.qr(rng.standard_normal((m, m)))[0][:r]
    w = mlp.init(nf, 12)
    w[mlp.H * nf:mlp.H * nf + mlp.H] = rng.normal(0, 0.3, mlp.H)            # b1
    w[-(2 * mlp.H + 1):-(mlp.H + 1)] = rng.normal(0, 0.3, mlp.H)             # b2
    w[-1] = 0.125                                                            # b3
    w = mlp.quantize_weights(w, nf)
    fp = oracle.FingerParams(P, 0.1, 0.9, 0.05, 1.1, 0.02)
    eps_p = 0.03
    outs = []
    for _ in range(50):
        q, c, d = rng.standard_normal((3, m))
        est, f_c, y_c = oracle.estimate_mlp(q, c, d, fp, w, eps_p)
        f_np, _ = mlp.features(q, c, d, P)
        np.testing.assert_allclose(f_c, f_np, rtol=1e-12, atol=1e-14)
        y_np, _ = mlp.forward(w, f_np[None, :], nf, round_act=True)
        assert y_c == pytest.approx(float(y_np[0]), rel=1e-12, abs=1e-12)
        # the estimate uses t = prediction + eps' in Eq. (2)
        cc = c @ c
        a, b = (c @ q) / cc, (c @ d) / cc
        qr, dr = q - a * c, d - b * c
        ref = (a - b) ** 2 * cc + qr @ qr + dr @ dr - 2 * np.linalg.norm(qr) * np.linalg.norm(dr) * (y_c + eps_p)
        assert est == pytest.approx(ref, rel=1e-12, abs=1e-12)
        outs.append(y_c)
    assert np.std(outs) > 1e-3          # the network is not constant on these inputs


def test_predictor_gate(small):
    """The gated predictor (extension): it runs only where the matched estimate
    lies within delta * ub of the ub at the start of the centre's expansion.
    delta = 0 leaves every matched estimate (an exact tie with ub has measure
    zero): the traversal of FINGER without a predictor.  With a predictor that
    says cos = 1e6 (its estimates never skip), the skipped neighbours fall
    from distribution matching's count (delta = 0) through a gated count to
    none (ungated), and widening the margin only removes skips."""
    X, Q, g, fp = small
    nf = fp.P.shape[0] + 4
    big = _const_predictor(nf, 1e6)
    i0, d0, c0 = oracle.search(g, X, Q, 10, 30, fp)
    i1, d1, c1 = oracle.search(g, X, Q, 10, 30, fp, mlp_weights=big, mlp_delta=0.0)
    assert (i0 == i1).all() and (d0 == d1).all() and (c0 == c1).all()
    skips = [c0[:, 3].sum()]
    for delta in (0.05, 0.5):
        _, _, c = oracle.search(g, X, Q, 10, 30, fp, mlp_weights=big, mlp_delta=delta)
        skips.append(c[:, 3].sum())
    _, _, c = oracle.search(g, X, Q, 10, 30, fp, mlp_weights=big, mlp_delta=-1.0)
    skips.append(c[:, 3].sum())
    assert skips[0] > skips[1] > skips[2] > skips[3] == 0, skips
