"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself: a
hand-worked example, a closed form, a published test vector, an algorithmic
reduction (FINGER with skipping off is Algorithm 1; full rank makes the
estimate exact), or brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _stats(mu=0.0, sigma=1.0, muh=0.0, sigmah=1.0, eps=0.0, P=None):
    return oracle.FingerParams(P, mu, sigma, muh, sigmah, eps)


def _graph_from_rows(rows, deg0, M=4):
    n = len(rows)
    adj0 = np.full((n, deg0), -1, np.int32)
    for i, r in enumerate(rows):
        adj0[i, : len(r)] = r
    return oracle.Graph(adj0, np.zeros(n, np.int32), np.full(n, -1, np.int64),
                        np.zeros((0, M), np.int32), 0, 0, M)


@pytest.fixture(scope="module")
def small():
    """2,000 points of the 16-cluster Gaussian mixture, oracle HNSW (M=8)."""
    X = workloads.base_vectors(1, 2000)
    Q = workloads.query_vectors(1, 60)
    g = oracle.hnsw_build(X, 8, 60, 3001)
    return X, Q, g


# ------------------------------------------------------------ generators


def test_splitmix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if l[0] != "#"]
    for inp, out in rows:
        assert oracle.splitmix64(int(inp, 16)) == int(out, 16)


def test_levels_geometric():
    n, M = 200_000, 16
    lv = oracle.levels(n, M, 3001)
    # P(level >= l) = M^-l for the draw floor(-ln U / ln M)
    for l in (1, 2, 3):
        p = M ** -l
        cnt = int((lv >= l).sum())
        assert abs(cnt - n * p) < 6 * math.sqrt(n * p * (1 - p)) + 1


# --------------------------------------------------------- Algorithm 3


def test_estimate_hand_example():
    # c = e1, q = (1,1,0), d = (2,0,1): a = 1, b = 2, q_res = e2, d_res = e3,
    # ||q_proj - d_proj||^2 = 1, ||q_res||^2 = ||d_res||^2 = 1, q_res^T d_res = 0.
    c = np.array([1.0, 0, 0])
    q = np.array([1.0, 1, 0])
    d = np.array([2.0, 0, 1])
    assert oracle.estimate(q, c, d, _stats(P=np.eye(3))) == pytest.approx(3.0, abs=1e-14)
    s = 1 / math.sqrt(2)
    st = dict(mu=0.1, sigma=2.0, muh=0.3, sigmah=4.0, eps=0.05)
    # P = (0,1,1)/sqrt2: P q_res = P d_res = 1/sqrt2 -> t_hat = 1,
    # t = (1 - 0.3) * 2/4 + 0.1 + 0.05 = 0.5, est = 1 + 1 + 1 - 2 * 0.5 = 2
    assert oracle.estimate(q, c, d, _stats(P=np.array([[0, s, s]]), **st)) == pytest.approx(2.0, abs=1e-14)
    # P = (0,1,-1)/sqrt2: t_hat = -1 -> t = -0.5, est = 4
    assert oracle.estimate(q, c, d, _stats(P=np.array([[0, s, -s]]), **st)) == pytest.approx(4.0, abs=1e-14)
    # P = e3: P q_res = 0 -> t_hat = 0 by convention, t = 0, est = 3
    assert oracle.estimate(q, c, d, _stats(P=np.array([[0, 0, 1.0]]), **st)) == pytest.approx(3.0, abs=1e-14)


def test_half_codes_round_to_nearest_even_from_fp64():
    """The binary16 rounding of the stored codes: IEEE round to nearest, ties to
    even, in one step from FP64 (numpy's float64 -> float16 conversion)."""
    cases = {1 + 2 ** -11: 1.0,                       # tie -> even
             1 + 2 ** -11 + 2 ** -40: 1 + 2 ** -10,   # just above the tie (FP32 first would tie)
             1 + 3 * 2 ** -11: 1 + 2 ** -9,           # tie -> even
             0.6: 1229 * 2 ** -11, 0.8: 1638 * 2 ** -11,
             2 ** -25: 0.0, 2 ** -25 + 2 ** -60: 2 ** -24}   # subnormal spacing 2^-24
    for x, want in cases.items():
        assert oracle.half_round(x) == want and oracle.half_round(-x) == -want
    x = np.random.default_rng(5).uniform(-1, 1, 20000) * 10.0 ** np.random.default_rng(6).uniform(-8, 0, 20000)
    assert all(oracle.half_round(v) == float(np.float16(v)) for v in x)


def test_estimate_half_codes_hand_example():
    """Algorithm 3 with the edge's unit residual projection stored as binary16.
    c = e3, P = [e1; e2] (r = 2), d = (3,4,5): b = 5, d_res = (3,4,0), u_d =
    (0.6, 0.8), stored as (1229, 1638) * 2^-11; q = (2,0,1): a = 1, q_res =
    (2,0,0), u_q = (1, 0).  t_hat = 0.60009765625 instead of 0.6, so with the
    identity matching the estimate 45 - 20 t is 32.998046875 instead of the
    exact 33."""
    P = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    q, c, d = np.array([2.0, 0, 1]), np.array([0, 0, 1.0]), np.array([3.0, 4, 5])
    assert oracle.estimate(q, c, d, _stats(P=P)) == 33.0
    fp = _stats(P=P)
    fp.codes = 16
    assert oracle.estimate(q, c, d, fp) == 32.998046875


def test_fp8_codes_round_to_nearest_even_from_fp64():
    """The FP8 E4M3 rounding of the stored codes (4 exponent bits, bias 7, 3
    fraction bits, no infinities, largest finite 448): ties to even, subnormal
    spacing 2^-9, saturation at +-448 as a satfinite conversion does."""
    cases = {1.0: 1.0, 1.0625: 1.0,                 # tie between 1 and 1.125 -> even
             1.1875: 1.25,                          # tie between 1.125 and 1.25 -> even
             1.07: 1.125, 153.6: 160.0, 204.8: 208.0,   # spacing 16 in [128, 256)
             2.0 ** -6: 2.0 ** -6,                  # smallest normal
             2.0 ** -10: 0.0, 3 * 2.0 ** -10: 2.0 ** -8,  # subnormal ties -> even
             5 * 2.0 ** -11: 2.0 ** -9,
             448.0: 448.0, 464.0: 448.0, 500.0: 448.0, 1e6: 448.0}
    for x, want in cases.items():
        assert oracle.e4m3_round(x) == want and oracle.e4m3_round(-x) == -want, x
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no FP8 dtype in this torch")
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, 20000) * 2.0 ** rng.uniform(-12, 8.7, 20000)   # |x| < 416
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert all(oracle.e4m3_round(v) == w for v, w in zip(x, ref))


def test_estimate_fp8_codes_hand_example():
    """Algorithm 3 with the edge's unit residual projection stored as FP8 E4M3
    codes of 256 u.  Same triple as the binary16 example: u_d = (0.6, 0.8), so
    the codes are e4m3(153.6) = 160 and e4m3(204.8) = 208, u_d is read back as
    (0.625, 0.8125), t_hat = 0.625 against u_q = (1, 0), and the estimate
    45 - 20 t is 32.5 instead of 33."""
    P = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    q, c, d = np.array([2.0, 0, 1]), np.array([0, 0, 1.0]), np.array([3.0, 4, 5])
    fp = _stats(P=P)
    fp.codes = 8
    assert oracle.estimate(q, c, d, fp) == 32.5


def test_estimate_fp8_codes_query_split_hand_example():
    """With FP8 codes 256 u_q enters the product as its E4M3 rounding h plus
    the E4M3 rounding of the remainder.  c = e3, P = [e1; e2], d = (3,4,5),
    q = (6,8,2): b = 5, a = 2, u_d = u_q = (0.6, 0.8), so the exact t is 1 and
    the estimate 134 - 100 t is ||q - d||^2 = 34.  256 u = (153.6, 204.8): the
    codes and h are (160, 208), the remainders (-6.4, -3.2) round to (-6.5,
    -3.25), so t_hat = (160 * 153.5 + 208 * 204.75) / 65536 = 1.02459716796875
    and the estimate is 31.540283203125."""
    P = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    q, c, d = np.array([6.0, 8, 2]), np.array([0, 0, 1.0]), np.array([3.0, 4, 5])
    assert oracle.estimate(q, c, d, _stats(P=P)) == pytest.approx(34.0, abs=1e-12)
    fp = _stats(P=P)
    fp.codes = 8
    assert oracle.estimate(q, c, d, fp) == 31.540283203125


def test_estimate_fp8_codes_exact_query_hand_example():
    """codes = 9: the FP8 codes (160, 208) / 256 against u_q = (0.6, 0.8)
    itself: t_hat = (0.6 * 160 + 0.8 * 208) / 256 = 1.025, estimate 31.5."""
    P = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    q, c, d = np.array([6.0, 8, 2]), np.array([0, 0, 1.0]), np.array([3.0, 4, 5])
    fp = _stats(P=P)
    fp.codes = 9
    assert oracle.estimate(q, c, d, fp) == pytest.approx(31.5, abs=1e-12)


def test_estimate_full_rank_is_exact_distance():
    """Eq. (2): with an orthogonal P (r = m) and identity matching the estimate
    is ||q - d||^2 exactly (the cross term q_proj^T q_res vanishes)."""
    rng = np.random.default_rng(0)
    m = 20
    P, _ = np.linalg.qr(rng.standard_normal((m, m)))
    for _ in range(50):
        q, c, d = rng.standard_normal((3, m)) * rng.uniform(0.1, 10)
        est = oracle.estimate(q, c, d, _stats(P=P.T))
        assert est == pytest.approx(float(((q - d) ** 2).sum()), rel=1e-11)


def test_estimate_zero_centre():
    # c = 0: projections vanish, q_res = q, d_res = d
    q, d = np.array([3.0, 0]), np.array([0, 4.0])
    est = oracle.estimate(q, np.zeros(2), d, _stats(P=np.eye(2)))
    assert est == pytest.approx(25.0)


# ------------------------------------------------------------ brute force


def test_bruteforce_hand_example_and_ties():
    X = np.array([[0.0], [1.0], [1.0], [2.0], [5.0]])
    ids, d = oracle.bruteforce(X, np.array([[1.0], [3.4]]), 4)
    assert ids[0].tolist() == [1, 2, 0, 3]          # ties broken by id
    assert d[0].tolist() == [0.0, 0.0, 1.0, 1.0]
    # q = 3.4: (3.4-2)^2 = 1.96, (3.4-5)^2 = 2.56, (3.4-1)^2 = 5.76 twice
    assert ids[1].tolist() == [3, 4, 1, 2]
    np.testing.assert_allclose(d[1], [1.96, 2.56, 5.76, 5.76], rtol=1e-14)


def test_bruteforce_pads_when_k_exceeds_n():
    ids, d = oracle.bruteforce(np.zeros((2, 3)), np.zeros((1, 3)), 4)
    assert ids[0].tolist() == [0, 1, -1, -1]
    assert np.isinf(d[0, 2:]).all()


# --------------------------------------------------------- Algorithm 1


def test_greedy_path_graph_hand_trace():
    """Points x_i = i on a line, path graph, query 7.2, ef = 1, entry 0.
    Hand trace: expansions 0..7 each admit the right neighbour; expanding 7
    evaluates 8 (0.64 > 0.04) and rejects it; no unexpanded entry is left."""
    X = np.arange(10, dtype=np.float64)[:, None]
    rows = [[1]] + [[i - 1, i + 1] for i in range(1, 9)] + [[8]]
    g = _graph_from_rows(rows, 2)
    ids, d, c = oracle.search(g, X, np.array([[7.2]]), 1, 1)
    assert ids[0, 0] == 7 and d[0, 0] == pytest.approx(0.04)
    cnt = dict(zip(oracle.CNT_NAMES, c[0]))
    assert cnt["expansions"] == 8 and cnt["examined"] == 8 and cnt["exact"] == 8
    assert cnt["admitted"] == 7 and cnt["estimates"] == 0 and cnt["upper"] == 1
    ids, d, _ = oracle.search(g, X, np.array([[7.2]]), 3, 3)
    assert ids[0].tolist() == [7, 8, 6]


def _alg4_case():
    import json
    t = json.load(open(os.path.join(GOLDEN, "alg4_hand_trace.json")))
    names = sorted(t["ids"], key=t["ids"].get)
    X = np.array([t["points"][k] for k in names], np.float64)
    rows = [[t["ids"][v] for v in t["adjacency"][k]] for k in names]
    g = _graph_from_rows(rows, 2, M=1)
    g.entry = t["ids"][t["entry"]]
    s = t["stats"]
    fp = oracle.FingerParams(np.array(t["P"], np.float64), s["mu"], s["sigma"], s["mu_hat"],
                             s["sigma_hat"], s["eps"])
    return t, X, g, fp


def test_finger_hand_trace_warmup_and_gate():
    """Algorithm 4 traced by hand (tests/golden/alg4_hand_trace.json).

    Points A=(0,2), B=(0,4), C=(0,-8), D=(-6,-1); path graph A-B-C-D; entry A;
    q = (-1,-4); ef = K = 2; P = [1, 0] (r = 1); mu = 1/4, sigma = 1,
    mu_hat = 1/2, sigma_hat = 2, eps = 1/4, so t = (t_hat - 1/2)/2 + 1/4 + 1/4
    = t_hat/2 + 1/4.  Every quantity below is exact in binary floating point.

    d(q,A) = 1 + 36 = 37.  T = [A 37].
    Expansion 1 (c = A, warm-up): B is new, exact d = 1 + 64 = 65, |T| < ef:
      admitted.  T = [A* 37, B 65].
    Expansion 2 (c = B = (0,4), ||c||^2 = 16): C is new and |T| = ef.
      With warm-up 1 it is estimated: a = q.c/16 = -1, b = c.C/16 = -2,
      q_res = (-1,0), C_res = (0,0), so t_hat = 0 (zero norm) and
      est = (a-b)^2 16 + 1 + 0 - 0 = 17 < ub = 65: not skipped.
      With warm-up 2 it is exact without an estimate.  Exact d = 1 + 16 = 17,
      admitted; A is visited.  T = [C 17, A* 37].
    Expansion 3 (c = C = (0,-8), ||c||^2 = 64): D is new, |T| = ef, estimated
      (both warm-ups): a = 32/64 = 1/2, b = 8/64 = 1/8, q_res = (-1,0),
      D_res = (-6,0), P q_res = -1, P D_res = -6, t_hat = 1, t = 3/4;
      est = (3/8)^2 64 + 1 + 36 - 2*1*6*3/4 = 9 + 37 - 9 = 37 = ub (A).
      Algorithm 4 skips only an estimate above ub: D gets its exact distance
      25 + 9 = 34 < 37 and is admitted.  T = [C* 17, D 34].
      (A gate that also skipped est = ub would drop D and end with [C, A].)
    Expansion 4 (c = D): C is visited.  No unexpanded entry remains.
    Counters: expansions 4, examined 3 (B, C, D), estimates 2 (warm-up 1) or
    1 (warm-up 2), skipped 0, exact 3, admitted 3.

    A warm-up counted one expansion late or early, or a gate that skips on
    equality, changes these counters."""
    t, X, g, fp = _alg4_case()
    q = np.array([t["query"]], np.float64)
    names = {v: k for k, v in t["ids"].items()}
    for key, warmup in (("warmup1_strict", 1), ("warmup2_strict", 2)):
        exp = t["expected"][key]
        ids, d, c = oracle.search(g, X, q, t["K"], t["ef"], fp, warmup=warmup)
        assert [names[i] for i in ids[0]] == exp["ids"], key
        assert d[0].tolist() == exp["dists"], key
        cnt = dict(zip(oracle.CNT_NAMES, c[0]))
        for k in ("expansions", "examined", "estimates", "skipped", "exact", "admitted"):
            assert cnt[k] == exp[k], (key, k, cnt[k], exp[k])
    # the estimate that meets ub exactly, from Algorithm 3 alone
    assert oracle.estimate(q[0], X[2], X[3], fp) == 37.0
    assert oracle.estimate(q[0], X[1], X[2], fp) == 17.0
    # the exact-distance branch for D is what makes the two gate readings differ
    nonstrict = t["expected"]["warmup1_nonstrict"]
    assert nonstrict["ids"] != t["expected"]["warmup1_strict"]["ids"]


def test_greedy_complete_graph_is_bruteforce():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((60, 5))
    Q = rng.standard_normal((20, 5))
    rows = [[j for j in range(60) if j != i] for i in range(60)]
    g = _graph_from_rows(rows, 64)
    gt, gd = oracle.bruteforce(X, Q, 10)
    ids, d, _ = oracle.search(g, X, Q, 10, 10)
    assert (ids == gt).all()
    np.testing.assert_allclose(d, gd, rtol=1e-15)


def test_greedy_exhaustive_ef_is_bruteforce(small):
    """ef = n on a connected graph admits every node, so T holds all of D."""
    X, Q, _ = small
    Xs = X[:300]
    gs = oracle.hnsw_build(Xs, 8, 60, 7)
    seen, stack = {gs.entry}, [gs.entry]
    while stack:
        for u in gs.adj0[stack.pop()]:
            if u >= 0 and u not in seen:
                seen.add(int(u))
                stack.append(int(u))
    assert len(seen) == 300                # precondition: layer 0 is connected
    gt, _ = oracle.bruteforce(Xs, Q, 10)
    ids, _, c = oracle.search(gs, Xs, Q, 10, 300)
    assert (ids == gt).all()
    assert (c[:, 0] == 300).all()          # every node expanded


# ------------------------------------------------------------ HNSW build


def test_hnsw_invariants(small):
    X, Q, g = small
    n = X.shape[0]
    M = g.M
    assert g.adj0.shape == (n, 2 * M)
    for v in range(n):
        row = g.adj0[v]
        valid = row[row >= 0]
        assert (row[len(valid):] == -1).all()            # packed
        assert len(set(valid.tolist())) == len(valid)     # no duplicates
        assert v not in valid
    assert g.level[g.entry] == g.maxlevel == g.level.max()
    assert g.entry == int(np.flatnonzero(g.level == g.maxlevel)[0])
    for v in np.flatnonzero(g.level > 0):
        for l in range(1, g.level[v] + 1):
            row = g.up_adj[g.up_off[v] + l - 1]
            valid = row[row >= 0]
            assert (g.level[valid] >= l).all()
            assert v not in valid
    # layer 0 is connected from the entry point
    seen = np.zeros(n, bool)
    stack = [g.entry]
    seen[g.entry] = True
    while stack:
        v = stack.pop()
        for u in g.adj0[v]:
            if u >= 0 and not seen[u]:
                seen[u] = True
                stack.append(u)
    assert seen.mean() > 0.99          # HNSW does not guarantee full reachability
    gt, _ = oracle.bruteforce(X, Q, 10)
    ids, _, _ = oracle.search(g, X, Q, 10, 60)
    assert oracle.recall(ids, gt, 10) > 0.97


# --------------------------------------------------------- Algorithm 4


def test_finger_without_skipping_is_plain(small):
    X, Q, g = small
    fp, _ = oracle.build_tables(X, g, 8, 4001)
    for ef in (10, 40):
        i1, d1, c1 = oracle.search(g, X, Q, 10, ef)
        i2, d2, c2 = oracle.search(g, X, Q, 10, ef, fp, warmup=10 ** 9)
        assert (i1 == i2).all() and (d1 == d2).all() and (c1 == c2).all()


def test_finger_full_rank_is_plain(small):
    X, Q, g = small
    fp, _ = oracle.build_tables(X, g, X.shape[1], 4001)
    assert fp.mu == pytest.approx(fp.mu_hat, abs=1e-12)
    assert fp.sigma == pytest.approx(fp.sigma_hat, abs=1e-12)
    assert fp.eps < 1e-12
    for ef in (10, 40):
        i1, d1, c1 = oracle.search(g, X, Q, 10, ef)
        i2, d2, c2 = oracle.search(g, X, Q, 10, ef, fp)
        assert (i1 == i2).all() and (d1 == d2).all()
        assert (c2[:, 2] > 0).any()               # estimates were made ...
        assert (c1[:, 0] == c2[:, 0]).all()        # ... and the traversal is the same


def test_finger_low_rank_skips(small):
    X, Q, g = small
    fp, _ = oracle.build_tables(X, g, 8, 4001)
    gt, _ = oracle.bruteforce(X, Q, 10)
    i1, _, c1 = oracle.search(g, X, Q, 10, 40)
    i2, _, c2 = oracle.search(g, X, Q, 10, 40, fp)
    assert c2[:, 3].sum() > 0.2 * c2[:, 2].sum()           # the gate skips
    assert c2[:, 4].sum() < c1[:, 4].sum()                 # fewer exact distances
    assert oracle.recall(i2, gt, 10) > oracle.recall(i1, gt, 10) - 0.05


# ---------------------------------------------------- Algorithm 2 pieces


def test_sample_pairs_properties(small):
    X, _, g = small
    S = oracle.sample_pairs(g.adj0, 4001)
    deg = (g.adj0 >= 0).sum(1)
    assert len(S) == int((deg >= 2).sum())
    for c, d, d2 in S:
        row = set(g.adj0[c][g.adj0[c] >= 0].tolist())
        assert d != d2 and d in row and d2 in row
    # the draw for one node, from the rule i = h1 mod deg, j = h2 mod (deg-1), j += (j >= i)
    c = int(S[5, 0])
    h1 = oracle.splitmix64(4001 ^ c)
    h2 = oracle.splitmix64(h1)
    valid = g.adj0[c][g.adj0[c] >= 0]
    i = h1 % len(valid)
    j = h2 % (len(valid) - 1)
    j += j >= i
    assert (S[5, 1], S[5, 2]) == (valid[i], valid[j])
    assert (oracle.sample_pairs(g.adj0, 4001) == S).all()


def test_residuals_orthogonal_to_centre():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((50, 7))
    R = oracle.residuals(X, np.arange(25), np.arange(25, 50))
    np.testing.assert_allclose(np.einsum("ij,ij->i", X[:25], R), 0, atol=1e-12)
    Rz = oracle.residuals(np.vstack([np.zeros(7), X[1:]]), np.array([0]), np.array([3]))
    np.testing.assert_allclose(Rz[0], X[3])        # c = 0 leaves d as its own residual


def test_basis_proposition1():
    """U_{1:r} maximises the captured energy ||P D_res||_F^2 over orthonormal P,
    which is the minimiser of the objective in the proof of Proposition 1."""
    rng = np.random.default_rng(3)
    m, r = 12, 4
    A = rng.standard_normal((m, m)) * np.linspace(3, 0.2, m)
    D = rng.standard_normal((800, m)) @ A.T
    P = oracle.basis(D, r, "svd")
    np.testing.assert_allclose(P @ P.T, np.eye(r), atol=1e-12)
    e_opt = np.linalg.norm(D @ P.T) ** 2
    s = np.linalg.svd(D, compute_uv=False)
    assert e_opt == pytest.approx((s[:r] ** 2).sum(), rel=1e-12)
    for _ in range(200):
        Qr, _ = np.linalg.qr(rng.standard_normal((m, r)))
        assert np.linalg.norm(D @ Qr) ** 2 <= e_opt * (1 + 1e-12)
    P2 = oracle.basis(D, r, "eigh")
    np.testing.assert_allclose(P2.T @ P2, P.T @ P, atol=1e-10)


def test_matching_stats_closed_forms():
    mu, sigma, muh, sigmah, eps = oracle.matching_stats(np.array([1.0, 2, 3, 4]),
                                                        np.array([1.0, 2, 3, 4]))
    assert (mu, muh) == (2.5, 2.5)
    assert sigma == pytest.approx(math.sqrt(1.25)) and eps == 0.0
    rng = np.random.default_rng(4)
    X = rng.standard_normal(10_000) * 0.2 + 0.3
    Y = 2.5 * X - 0.7                       # an affine image is matched exactly
    mu, sigma, muh, sigmah, eps = oracle.matching_stats(X, Y)
    assert muh == pytest.approx(2.5 * mu - 0.7) and sigmah == pytest.approx(2.5 * sigma)
    assert eps < 1e-12
    Xg = rng.normal(0.4, 0.1, 400_000)
    Yg = rng.normal(-0.2, 0.3, 400_000)
    mu, sigma, muh, sigmah, _ = oracle.matching_stats(Xg, Yg)
    assert abs(mu - 0.4) < 1e-3 and abs(sigma - 0.1) < 1e-3
    assert abs(muh + 0.2) < 3e-3 and abs(sigmah - 0.3) < 3e-3


def test_full_rank_cosines_match(small):
    X, _, g = small
    S = oracle.sample_pairs(g.adj0, 4001)
    Xc, Yc = oracle.pair_cosines(X, S, np.eye(X.shape[1]))
    np.testing.assert_allclose(Xc, Yc, atol=1e-12)
    assert np.abs(Xc).max() <= 1 + 1e-12


def test_edge_tables_definitions(small):
    X, _, g = small
    P = oracle.basis(oracle.residuals(X, np.arange(500), g.adj0[:500, 0]), 8)
    nodes = np.arange(40)
    u, dn, b = oracle.edge_tables(X, g.adj0, P, nodes)
    Xd = X.astype(np.float64)
    for c in nodes:
        for j, d in enumerate(g.adj0[c]):
            if d < 0:
                assert dn[c, j] == 0 and not u[c, j].any()
                continue
            res = Xd[d] - b[c, j] * Xd[c]
            assert abs(Xd[c] @ res) < 1e-9 * (1 + abs(Xd[c] @ Xd[d]))
            assert dn[c, j] == pytest.approx(np.linalg.norm(res), rel=1e-12)
            assert np.linalg.norm(u[c, j]) == pytest.approx(1.0, rel=1e-12)
            np.testing.assert_allclose(u[c, j] * np.linalg.norm(P @ res), P @ res, atol=1e-9)


def test_memory_formula_matches_paper_table():
    """Supplementary F: FINGER adds (r+2) |E| floats; with |E| = n * 2M layer-0
    slots this reproduces the printed extra memory within 10 %."""
    for line in open(os.path.join(GOLDEN, "memory_table.txt")):
        if line.startswith("#") or not line.strip():
            continue
        _, n, M, r, fg, hg = line.split()
        n, M, r, fg, hg = int(n), int(M), int(r), float(fg), float(hg)
        extra = (r + 2) * n * 2 * M * 4 / 1e9
        assert abs(extra - (fg - hg)) / (fg - hg) < 0.10


def test_flat_graph_is_single_layer_and_searchable():
    """The single-layer option: every node on level 0, entry node 0, the layer-0
    caps and invariants of the hierarchical build, and exhaustive search
    (ef = n) finds the brute-force answer."""
    X = workloads.base_vectors(1, 800)
    Q = workloads.query_vectors(1, 20)
    g = oracle.hnsw_build(X, 8, 40, 1, flat=True)
    assert (g.level == 0).all() and g.maxlevel == 0 and g.entry == 0
    assert g.up_adj.shape[0] == 0
    for v in range(0, 800, 13):
        row = g.adj0[v]
        valid = row[row >= 0]
        assert (row[len(valid):] == -1).all() and v not in valid
        assert len(set(valid.tolist())) == len(valid)
    ids, d, _ = oracle.search(g, X, Q, 5, 800)
    gt, gd = oracle.bruteforce(X, Q, 5)
    assert (ids == gt).all()
    np.testing.assert_allclose(d, gd, rtol=1e-12)


def test_merge_of_exact_part_knn_is_exact_knn():
    """The K nearest of a database are the K smallest keys of its parts' K
    nearest: merging the exact kNN of three uneven parts (one smaller than K,
    so its lists are padded) gives the exact kNN of the whole, ties included
    (integer data produce equal distances, broken by global id)."""
    rng = np.random.default_rng(11)
    X = rng.integers(0, 4, size=(700, 6)).astype(np.float32)
    Q = rng.integers(0, 4, size=(25, 6)).astype(np.float32)
    K = 12
    cuts = [0, 5, 300, 700]
    ids_l, d_l = [], []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        i, d = oracle.bruteforce(X[lo:hi], Q, K)
        ids_l.append(i)
        d_l.append(d)
    assert (ids_l[0][:, 5:] == -1).all()            # the 5-row part pads its lists
    mi, md = oracle.merge_topk(ids_l, d_l, cuts[:-1], K)
    gi, gd = oracle.bruteforce(X, Q, K)
    assert (mi == gi).all()
    assert (md == gd).all()
    # more results asked than the parts hold in total: padded
    i1, d1 = oracle.bruteforce(X[:3], Q, 4)
    i2, d2 = oracle.bruteforce(X[3:5], Q, 4)
    mi, md = oracle.merge_topk([i1, i2], [d1, d2], [0, 3], 6)
    gi, gd = oracle.bruteforce(X[:5], Q, 6)
    assert (mi == gi).all() and (mi[:, 5] == -1).all() and np.isinf(md[:, 5]).all()
