"""Pins of the oracle's ablation switches (Sec. 4.3: RPLSH basis, no
distribution matching, no error term) and of the rank rule (Supplementary E),
each against something other than the oracle itself: a library routine, a
closed form, or an algorithmic reduction."""
import numpy as np
import pytest

import oracle
import workloads


@pytest.fixture(scope="module")
def small():
    X = workloads.base_vectors(1, 2000)
    Q = workloads.query_vectors(1, 60)
    g = oracle.hnsw_build(X, 8, 60, 3001)
    return X, Q, g


def test_correlation_library_and_closed_forms():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(5000)
    y = 0.6 * x + 0.8 * rng.standard_normal(5000)
    assert oracle.correlation(x, y) == pytest.approx(np.corrcoef(x, y)[0, 1], abs=1e-12)
    assert oracle.correlation(x, 3.0 * x - 2.0) == pytest.approx(1.0, abs=1e-12)
    assert oracle.correlation(x, -0.5 * x + 1.0) == pytest.approx(-1.0, abs=1e-12)
    assert oracle.correlation(x, np.full_like(x, 0.3)) == 0.0


def test_no_matching_no_eps_full_rank_is_plain(small):
    """Without matching and without eps, t = t_hat; at full rank t_hat is the
    true residual cosine, so the estimate is the exact distance and the
    traversal is Algorithm 1's."""
    X, Q, g = small
    fp, _ = oracle.build_tables(X, g, X.shape[1], 4001, matching=False, use_eps=False)
    assert (fp.mu, fp.sigma, fp.mu_hat, fp.sigma_hat, fp.eps) == (0.0, 1.0, 0.0, 1.0, 0.0)
    assert fp.corr == pytest.approx(1.0, abs=1e-12)
    for ef in (10, 40):
        i1, d1, c1 = oracle.search(g, X, Q, 10, ef)
        i2, d2, c2 = oracle.search(g, X, Q, 10, ef, fp)
        assert (i1 == i2).all() and (d1 == d2).all()
        assert (c2[:, 2] > 0).any() and (c1[:, 0] == c2[:, 0]).all()


def test_no_matching_keeps_identity_map(small):
    """Matching off: the map is the identity (mu = mu_hat = 0, sigma =
    sigma_hat = 1) and eps is the mean |Y - X|, which vanishes at full rank."""
    X, Q, g = small
    lo, _ = oracle.build_tables(X, g, 8, 4001, matching=False)
    assert (lo.mu, lo.sigma, lo.mu_hat, lo.sigma_hat) == (0.0, 1.0, 0.0, 1.0)
    assert lo.eps > 0
    full, _ = oracle.build_tables(X, g, X.shape[1], 4001, matching=False)
    assert full.eps < 1e-12
    on, _ = oracle.build_tables(X, g, 8, 4001)
    off, _ = oracle.build_tables(X, g, 8, 4001, use_eps=False)
    assert off.eps == 0.0
    assert (off.mu, off.sigma, off.mu_hat, off.sigma_hat) == (on.mu, on.sigma, on.mu_hat,
                                                              on.sigma_hat)
    # matching is an affine map of Y: it leaves the correlation unchanged
    assert lo.corr == pytest.approx(on.corr, abs=1e-12)


def test_orthogonal_basis_preserves_angles(small):
    """A basis passed in is used as is: an orthogonal m x m matrix preserves
    every angle, so Y = X, corr = 1, mu = mu_hat, sigma = sigma_hat, eps = 0."""
    X, Q, g = small
    m = X.shape[1]
    R = np.linalg.qr(np.random.default_rng(5).standard_normal((m, m)))[0]
    fp, _ = oracle.build_tables(X, g, m, 4001, basis=R)
    np.testing.assert_array_equal(fp.P, R)
    assert fp.corr == pytest.approx(1.0, abs=1e-12)
    assert fp.mu == pytest.approx(fp.mu_hat, abs=1e-12)
    assert fp.sigma == pytest.approx(fp.sigma_hat, abs=1e-12)
    assert fp.eps < 1e-12


def test_random_basis_captures_less_than_svd(small):
    """Sec. 3.3 / Proposition 1: at equal rank the SVD basis of D_res estimates
    residual angles better (higher corr(X, Y)) than a random Gaussian basis."""
    X, Q, g = small
    r, m = 8, X.shape[1]
    svd, _ = oracle.build_tables(X, g, r, 4001)
    G = np.random.default_rng(6).standard_normal((r, m))
    rp, _ = oracle.build_tables(X, g, r, 4001, basis=G)
    assert svd.corr > rp.corr + 0.05


def test_rank_rule_low_dimensional_residuals():
    """Data on a 4-dimensional linear subspace of R^16: every residual lies in
    that subspace, the first candidate rank (8) already spans it, Y = X and the
    rule stops at r = 8 with corr = 1."""
    rng = np.random.default_rng(7)
    B = np.linalg.qr(rng.standard_normal((16, 4)))[0]
    X = (rng.standard_normal((600, 4)) @ B.T + 0.0).astype(np.float32)
    g = oracle.hnsw_build(X, 8, 40, 11)
    r, trace = oracle.select_rank(X, g, 12)
    assert r == 8 and len(trace) == 1
    assert trace[0][1] == pytest.approx(1.0, abs=1e-6)


def test_rank_rule_unreachable_threshold_ends_at_full_rank(small):
    """A threshold above 1 is never met: the rule walks 8, 16, ... up to m and
    stops there, where the basis is complete and corr = 1."""
    X, Q, g = small
    m = X.shape[1]
    r, trace = oracle.select_rank(X, g, 4001, threshold=1.5)
    assert r == m
    assert [t[0] for t in trace] == list(range(8, m + 1, 8))
    assert trace[-1][1] == pytest.approx(1.0, abs=1e-9)
    # every candidate's correlation equals the one of a table build at that rank
    for rr, c in trace[:3]:
        fp, _ = oracle.build_tables(X, g, rr, 4001)
        assert fp.corr == pytest.approx(c, abs=1e-9)
