"""FP64 CPU oracle for FINGER (arXiv 2206.11408).

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path and never takes an input that the CUDA path produced.

The C part (``oracle.c``, built with plain gcc) holds the loops: brute-force
kNN, HNSW construction, greedy search (Algorithm 1) and FINGER search
(Algorithm 4 with Algorithm 3).  This module holds the FINGER construction of
Algorithm 2 in numpy FP64: residuals of sampled neighbour pairs, the SVD basis
(Proposition 1), the matching statistics (Sec. 3.3) and, for table parity,
the per-edge quantities of Supplementary G written out from their definitions.

Readings of passages the paper leaves open are listed where they are used:
  * ties: keys are the pair (distance, id) everywhere;
  * sigma, sigma_hat are standard deviations (Algorithm 2 prints the variance
    formula but Sec. 3.3 uses sigma/sigma_hat as a scale of N(mu, sigma));
  * Algorithm 2 takes cos(d, d') of the *residual* vectors w.r.t. the sampling
    centre c (Sec. 3.2 and Fig. 3 model residual angles);
  * cos(x, y) = 0 when ||x|| ||y|| = 0; a = b = 0 when c^T c = 0.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None

CNT_NAMES = ("expansions", "examined", "estimates", "skipped", "exact", "admitted", "upper")


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
        L.orc_splitmix64.argtypes = [u64]
        L.orc_splitmix64.restype = u64
        L.orc_levels.argtypes = [i64, i32, u64, P]
        L.orc_bruteforce.argtypes = [P, i64, i32, P, i64, i32, P, P, i32]
        L.orc_hnsw_build.argtypes = [P, i64, i32, i32, i32, P, P, i64, P, P, P, P]
        L.orc_hnsw_build.restype = i32
        L.orc_search.argtypes = [P, i64, i32, P, i32, P, P, i32, i32, i32, P, i64, i32, i32, P,
                                 i32, P, i32, i32, P, P, P, i32, P, ctypes.c_double, i32,
                                 ctypes.c_double]
        L.orc_search.restype = i32
        L.orc_sample_pairs.argtypes = [P, i64, i32, u64, i32, P]
        L.orc_estimate.argtypes = [P, P, P, i32, P, i32, P, i32]
        L.orc_half_round.argtypes = [ctypes.c_double]
        L.orc_half_round.restype = ctypes.c_double
        L.orc_e4m3_round.argtypes = [ctypes.c_double]
        L.orc_e4m3_round.restype = ctypes.c_double
        L.orc_estimate.restype = ctypes.c_double
        L.orc_estimate_mlp.argtypes = [P, P, P, i32, P, i32, P, P, ctypes.c_double, P, P]
        L.orc_estimate_mlp.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------- graph


@dataclasses.dataclass
class Graph:
    """An HNSW graph in flat arrays.

    adj0    (n, 2M) int32   layer-0 neighbour lists, valid entries first, -1 pad
    level   (n,)   int32    top level of each node
    up_off  (n,)   int64    row of (node, level 1); rows of levels 1..level[v]
                            are up_off[v] .. up_off[v]+level[v]-1; -1 if level 0
    up_adj  (R, M) int32    upper-level neighbour lists, -1 pad
    entry, maxlevel         global entry point and its level
    """
    adj0: np.ndarray
    level: np.ndarray
    up_off: np.ndarray
    up_adj: np.ndarray
    entry: int
    maxlevel: int
    M: int


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def levels(n: int, M: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    lib().orc_levels(n, M, seed, _p(out))
    return out


def upper_offsets(level: np.ndarray):
    lv = level.astype(np.int64)
    ends = np.cumsum(lv)
    off = np.where(lv > 0, ends - lv, -1).astype(np.int64)
    return off, int(ends[-1]) if len(lv) else 0


def hnsw_build(X, M: int, ef_construction: int, seed: int, flat: bool = False) -> Graph:
    """Incremental HNSW in FP64, nodes inserted in id order (serial, deterministic).

    ``flat=True`` puts every node on level 0: the same incremental insertion and
    heuristic selection on a single layer (a navigable small-world graph without
    the hierarchy), searched from node 0 -- a non-HNSW graph for FINGER, which
    the paper builds on top of a given graph (Sec. 3.3)."""
    X = _f64(X)
    n, m = X.shape
    lv = np.zeros(n, np.int32) if flat else levels(n, M, seed)
    up_off, R = upper_offsets(lv)
    adj0 = np.empty((n, 2 * M), dtype=np.int32)
    up_adj = np.empty((max(R, 1), M), dtype=np.int32)
    entry = np.zeros(1, dtype=np.int32)
    maxl = np.zeros(1, dtype=np.int32)
    lib().orc_hnsw_build(_p(X), n, m, M, ef_construction, _p(lv), _p(up_off), R, _p(adj0),
                         _p(up_adj), _p(entry), _p(maxl))
    return Graph(adj0, lv, up_off, up_adj[:R] if R else up_adj[:0], int(entry[0]), int(maxl[0]), M)


# ------------------------------------------------------------- brute force


def bruteforce(X, Q, K: int, threads: int = 0):
    """Exact K nearest neighbours by squared L2, ordered by (distance, id)."""
    X, Q = _f64(X), _f64(Q)
    nq = Q.shape[0]
    ids = np.empty((nq, K), dtype=np.int64)
    d = np.empty((nq, K), dtype=np.float64)
    lib().orc_bruteforce(_p(X), X.shape[0], X.shape[1], _p(Q), nq, K, _p(ids), _p(d), threads)
    return ids, d


def merge_topk(ids_list, dists_list, offsets, K: int):
    """K nearest over a partitioned database: the K smallest (distance, global
    id) keys of the union of the parts' lists (the kNN problem of Sec. 1 over
    the union).  ids_list / dists_list: one nq x K pair per part with local
    ids (-1 = empty); offsets: each part's first global id.  Distances keep
    their dtype; missing results are -1 / +inf."""
    nq = ids_list[0].shape[0]
    out_i = np.full((nq, K), -1, dtype=np.int64)
    out_d = np.full((nq, K), np.inf, dtype=np.asarray(dists_list[0]).dtype)
    for q in range(nq):
        cand = []
        for ids, d, off in zip(ids_list, dists_list, offsets):
            for i, x in zip(ids[q], d[q]):
                if i >= 0:
                    cand.append((x, int(i) + int(off)))
        cand.sort()
        for k, (x, g) in enumerate(cand[:K]):
            out_i[q, k] = g
            out_d[q, k] = x
    return out_i, out_d


# ---------------------------------------------------------------- search


@dataclasses.dataclass
class FingerParams:
    """Projection P (r x m) and the statistics mu, sigma, mu_hat, sigma_hat, eps."""
    P: np.ndarray
    mu: float
    sigma: float
    mu_hat: float
    sigma_hat: float
    eps: float
    corr: float = float("nan")      # Pearson correlation of X and Y over S (Supp. E)
    codes: int = 0                  # 16: the per-edge unit P d_res stored as binary16 codes;
                                    # 8: 256 times it stored as FP8 E4M3 codes, 256 u_q as
                                    # its E4M3 rounding plus that of the remainder;
                                    # 9: the same codes against u_q itself

    def stats(self):
        return np.array([self.mu, self.sigma, self.mu_hat, self.sigma_hat, self.eps], np.float64)


def search(g: Graph, X, Q, K: int, ef: int, finger: FingerParams | None = None, warmup: int = 5,
           threads: int = 0, mlp_weights=None, mlp_eps: float = 0.0, mlp_delta: float = -1.0):
    """Descent on levels >= 1, then Algorithm 1 (finger=None) or Algorithm 4.
    With mlp_weights (flat, see oracle.mlp) the learned predictor replaces the
    distribution matching in Algorithm 3 (extension, not in the paper): on
    every estimate when mlp_delta < 0, else only where the matched estimate
    lies within mlp_delta * ub of the ub at the start of the centre's expansion
    (with the result list full then).

    Returns ids (nq, K) int64, dists (nq, K) float64 and per-query counters
    (nq, 8) int64 in the order of CNT_NAMES.
    """
    X, Q = _f64(X), _f64(Q)
    n, m = X.shape
    nq = Q.shape[0]
    ids = np.empty((nq, K), dtype=np.int64)
    d = np.empty((nq, K), dtype=np.float64)
    cnt = np.empty((nq, 8), dtype=np.int64)
    if finger is None:
        P = np.zeros((1, m), np.float64)
        r, st, fl, codes = 1, np.zeros(5, np.float64), 0, 0
    else:
        P = _f64(finger.P)
        r, st, fl, codes = P.shape[0], finger.stats(), 1, int(finger.codes)
    adj0 = np.ascontiguousarray(g.adj0, dtype=np.int32)
    up_adj = np.ascontiguousarray(g.up_adj if len(g.up_adj) else np.full((1, g.M), -1, np.int32),
                                  dtype=np.int32)
    up_off = np.ascontiguousarray(g.up_off, dtype=np.int64)
    mw = None if mlp_weights is None else _f64(mlp_weights)
    rc = lib().orc_search(_p(X), n, m, _p(adj0), adj0.shape[1], _p(up_off), _p(up_adj), g.M,
                          g.entry, g.maxlevel, _p(Q), nq, K, ef, _p(P), r, _p(st), warmup, fl,
                          _p(ids), _p(d), _p(cnt), threads, _p(mw) if mw is not None else None,
                          float(mlp_eps), codes, float(mlp_delta))
    if rc != 0:
        raise ValueError("orc_search rejected its arguments")
    return ids, d, cnt


def estimate(q, c, d, fp: FingerParams) -> float:
    """Algorithm 3 on one triple: the distance estimate of ||q - d||^2 from the
    projection onto centre c, the residual norms and the matched angle."""
    q, c, d, P = _f64(q), _f64(c), _f64(d), _f64(fp.P)
    st = fp.stats()
    return float(lib().orc_estimate(_p(q), _p(c), _p(d), q.shape[0], _p(P), P.shape[0], _p(st),
                                    int(fp.codes)))


def half_round(x: float) -> float:
    """The oracle's rounding of a code to the nearest binary16 value (ties to
    even), as FINGER_F16 stores the per-edge unit residual projections."""
    return float(lib().orc_half_round(float(x)))


def e4m3_round(x: float) -> float:
    """The oracle's rounding to the nearest FP8 E4M3 value (ties to even,
    saturating at +-448), as FINGER_F8 stores 256 times each unit residual
    projection."""
    return float(lib().orc_e4m3_round(float(x)))


def estimate_mlp(q, c, d, fp: FingerParams, mlp_weights, mlp_eps: float = 0.0):
    """Algorithm 3 on one triple with the learned predictor in place of
    distribution matching (extension), as the oracle's search applies it.
    Returns (estimate, features (r + 4), raw prediction)."""
    q, c, d, P = _f64(q), _f64(c), _f64(d), _f64(fp.P)
    st = fp.stats()
    w = _f64(mlp_weights)
    r = P.shape[0]
    f = np.zeros(r + 4, np.float64)
    y = np.zeros(1, np.float64)
    e = lib().orc_estimate_mlp(_p(q), _p(c), _p(d), q.shape[0], _p(P), r, _p(st), _p(w),
                               float(mlp_eps), _p(f), _p(y))
    return float(e), f, float(y[0])


# --------------------------------------------------- Algorithm 2 (FINGER build)


def sample_pairs(adj0, seed: int, samples_per_node: int = 1) -> np.ndarray:
    """Rows (c, d, d') of the pair set S; nodes with fewer than two neighbours
    are dropped.  The draw is the counter-based rule documented in oracle.c."""
    adj0 = np.ascontiguousarray(adj0, dtype=np.int32)
    n, deg0 = adj0.shape
    out = np.empty((n * samples_per_node, 3), dtype=np.int32)
    lib().orc_sample_pairs(_p(adj0), n, deg0, seed, samples_per_node, _p(out))
    return out[out[:, 0] >= 0]


def residuals(X, c_ids, d_ids) -> np.ndarray:
    """d_res = d - (c^T d / c^T c) c for each (c, d), Eq. (1) applied to d."""
    X = np.asarray(X)
    C = X[c_ids].astype(np.float64)
    D = X[d_ids].astype(np.float64)
    cc = np.einsum("ij,ij->i", C, C)
    cd = np.einsum("ij,ij->i", C, D)
    b = np.divide(cd, cc, out=np.zeros_like(cd), where=cc > 0)
    return D - b[:, None] * C


def basis(D_res: np.ndarray, r: int, method: str = "auto") -> np.ndarray:
    """P = U_{1:r}^T from the SVD of D_res (rows are samples: D_res^T in the
    paper's m x N notation).  Proposition 1.  'eigh' uses the Gram matrix, whose
    eigenvectors are the same left singular vectors."""
    N, m = D_res.shape
    if method == "auto":
        method = "svd" if N * m <= 10 ** 8 else "eigh"
    if method == "svd":
        U, s, _ = np.linalg.svd(D_res.T, full_matrices=False)
        return np.ascontiguousarray(U[:, :r].T)
    G = D_res.T @ D_res
    w, V = np.linalg.eigh(G)
    order = np.argsort(-w, kind="stable")
    return np.ascontiguousarray(V[:, order[:r]].T)


def _cos_rows(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    num = np.einsum("ij,ij->i", A, B)
    den = np.linalg.norm(A, axis=1) * np.linalg.norm(B, axis=1)
    return np.divide(num, den, out=np.zeros_like(num), where=den > 0)


def pair_cosines(X, pairs: np.ndarray, P: np.ndarray, chunk: int = 1 << 16):
    """X_i = cos(d_res, d'_res) and Y_i = cos(P d_res, P d'_res) over S."""
    P = _f64(P)
    xs, ys = [], []
    for lo in range(0, len(pairs), chunk):
        p = pairs[lo:lo + chunk]
        R1 = residuals(X, p[:, 0], p[:, 1])
        R2 = residuals(X, p[:, 0], p[:, 2])
        xs.append(_cos_rows(R1, R2))
        ys.append(_cos_rows(R1 @ P.T, R2 @ P.T))
    return np.concatenate(xs), np.concatenate(ys)


def matching_stats(Xc: np.ndarray, Yc: np.ndarray, matching: bool = True, use_eps: bool = True):
    """mu, sigma (std), mu_hat, sigma_hat, eps of Algorithm 2 (population 1/N).

    Ablations of Sec. 4.3: ``matching=False`` keeps the low-rank cosine as it
    is (the map becomes t = t_hat + eps, returned as mu = mu_hat = 0,
    sigma = sigma_hat = 1) and eps is then the mean |Y - X|;
    ``use_eps=False`` drops the error-correction term (eps = 0)."""
    if matching:
        mu, muh = float(np.mean(Xc)), float(np.mean(Yc))
        sigma = float(np.sqrt(np.mean((Xc - mu) ** 2)))
        sigmah = float(np.sqrt(np.mean((Yc - muh) ** 2)))
    else:
        mu, sigma, muh, sigmah = 0.0, 1.0, 0.0, 1.0
    ratio = sigma / sigmah if sigmah > 0 else 0.0
    eps = float(np.mean(np.abs((Yc - muh) * ratio + mu - Xc))) if use_eps else 0.0
    return mu, sigma, muh, sigmah, eps


def correlation(Xc: np.ndarray, Yc: np.ndarray) -> float:
    """Pearson correlation of the true and the low-rank residual cosines over
    the sampled pairs, the quantity of the rank rule (Supplementary E):
    population covariance over the product of the population standard
    deviations; 0 when either is 0."""
    dx, dy = Xc - np.mean(Xc), Yc - np.mean(Yc)
    den = np.sqrt(np.mean(dx * dx) * np.mean(dy * dy))
    return float(np.mean(dx * dy) / den) if den > 0 else 0.0


def _sorted_eigvecs(X, pairs, m, method, chunk):
    """Left singular vectors of D_res ordered by singular value (columns)."""
    if method == "svd":
        D_res = residuals(X, pairs[:, 0], pairs[:, 1])
        U, _, _ = np.linalg.svd(D_res.T, full_matrices=False)
        return U
    G = np.zeros((m, m), np.float64)
    for lo in range(0, len(pairs), chunk):
        p = pairs[lo:lo + chunk]
        R = residuals(X, p[:, 0], p[:, 1])
        G += R.T @ R
    w, V = np.linalg.eigh(G)
    return V[:, np.argsort(-w, kind="stable")]


def build_tables(X, g: Graph, r: int, seed: int, samples_per_node: int = 1,
                 method: str = "auto", chunk: int = 1 << 16, basis: np.ndarray | None = None,
                 matching: bool = True, use_eps: bool = True):
    """Algorithm 2: sample S, D_res, SVD -> P, then the matching statistics.

    ``basis`` (r x m) replaces the SVD basis (the RPLSH comparison of Sec. 4.3
    passes a random Gaussian matrix); ``matching`` / ``use_eps`` are the
    ablations of :func:`matching_stats`."""
    pairs = sample_pairs(g.adj0, seed, samples_per_node)
    m = np.asarray(X).shape[1]
    if method == "auto":
        method = "svd" if len(pairs) * m <= 10 ** 8 else "eigh"
    if basis is not None:
        P = np.ascontiguousarray(_f64(basis)[:r])
    else:
        P = np.ascontiguousarray(_sorted_eigvecs(X, pairs, m, method, chunk)[:, :r].T)
    Xc, Yc = pair_cosines(X, pairs, P, chunk)
    mu, sigma, muh, sigmah, eps = matching_stats(Xc, Yc, matching, use_eps)
    return FingerParams(P, mu, sigma, muh, sigmah, eps, correlation(Xc, Yc)), pairs


def select_rank(X, g: Graph, seed: int, threshold: float = 0.7, r_start: int = 8,
                r_step: int = 8, r_max: int = 64, samples_per_node: int = 1,
                method: str = "auto", chunk: int = 1 << 16):
    """Rank rule of Supplementary E: start at r = 8 and add 8 while the
    correlation of X and Y (Algorithm 2's true and low-rank residual cosines)
    is below the threshold (0.7); stop at r_max.  The basis of every rank is
    the top-r prefix of the same singular vectors.  Returns (r, [(r, corr)])."""
    pairs = sample_pairs(g.adj0, seed, samples_per_node)
    m = np.asarray(X).shape[1]
    if method == "auto":
        method = "svd" if len(pairs) * m <= 10 ** 8 else "eigh"
    U = _sorted_eigvecs(X, pairs, m, method, chunk)
    trace = []
    r = r_start
    while True:
        rr = min(r, m, r_max)
        Xc, Yc = pair_cosines(X, pairs, np.ascontiguousarray(U[:, :rr].T), chunk)
        c = correlation(Xc, Yc)
        trace.append((rr, c))
        if c >= threshold or rr >= min(m, r_max):
            return rr, trace
        r += r_step


def gram(X, pairs: np.ndarray, chunk: int = 1 << 16) -> np.ndarray:
    """sum over S of d_res d_res^T (m x m), the matrix whose top eigenvectors are P^T."""
    m = np.asarray(X).shape[1]
    G = np.zeros((m, m), np.float64)
    for lo in range(0, len(pairs), chunk):
        p = pairs[lo:lo + chunk]
        R = residuals(X, p[:, 0], p[:, 1])
        G += R.T @ R
    return G


def edge_tables(X, adj0, P, nodes=None):
    """Per-edge quantities of Supplementary G from their definitions, FP64.

    For edge (c, d) in row c of adj0: b = c^T d / c^T c, ||d_res|| and
    u = P d_res / ||P d_res|| (0 when the norm is 0).  Returns (u, dres_norm, b)
    with shapes (k, deg0, r), (k, deg0), (k, deg0) for the chosen ``nodes``
    (default all); entries of -1 neighbours are 0.
    """
    X = np.asarray(X)
    adj0 = np.asarray(adj0)
    P = _f64(P)
    if nodes is None:
        nodes = np.arange(adj0.shape[0])
    rows = adj0[nodes]
    k, deg0 = rows.shape
    c = np.repeat(nodes, deg0)
    d = rows.reshape(-1)
    ok = d >= 0
    dres = residuals(X, c[ok], d[ok])
    Pd = dres @ P.T
    nPd = np.linalg.norm(Pd, axis=1)
    u = np.zeros((k * deg0, P.shape[0]))
    u[ok] = np.divide(Pd, nPd[:, None], out=np.zeros_like(Pd), where=nPd[:, None] > 0)
    dn = np.zeros(k * deg0)
    dn[ok] = np.linalg.norm(dres, axis=1)
    C = X[c[ok]].astype(np.float64)
    D = X[d[ok]].astype(np.float64)
    cc = np.einsum("ij,ij->i", C, C)
    bb = np.zeros(k * deg0)
    bb[ok] = np.divide(np.einsum("ij,ij->i", C, D), cc, out=np.zeros(ok.sum()), where=cc > 0)
    return u.reshape(k, deg0, -1), dn.reshape(k, deg0), bb.reshape(k, deg0)


def recall(ids: np.ndarray, gt: np.ndarray, K: int) -> float:
    """recall@K = |T intersect A| / K averaged over queries (Sec. 1)."""
    hit = 0
    for a, b in zip(ids[:, :K], gt[:, :K]):
        hit += len(set(a.tolist()) & set(b.tolist()))
    return hit / (K * len(ids))
