"""Deterministic generators for the five synthetic workloads.

The paper measures on ANN-benchmarks datasets (SIFT, GloVe, DEEP, GIST, ...,
Sec. 4.1).  None of them is used here; each configuration below is a seeded
stand-in with the shape of one of them:

    1  n=10k,  m=64,  16-component isotropic Gaussian mixture (sigma 0.3), L2
    2  n=1M,   m=128, integers 0..255, per-dim gamma, 64 clusters (SIFT-like), L2
    3  n=1.2M, m=100, unit-normalised, 256 clusters, power-law sizes (GloVe-like)
    4  n=1M,   m=96,  unit-normalised, 128-cluster Gaussian mixture (DEEP-like)
    5  n=1M,   m=960, per-dim lognormal magnitudes, 32 clusters (GIST-like), L2

Configurations 3-5 give the within-cluster variation the decaying spectrum of
real embedding and descriptor sets: one covariance shared by all clusters,
R diag(lambda) R^T with a seeded random orthonormal frame R and a Zipf
spectrum lambda_i proportional to 1/i, scaled so that the total variance is
sigma^2 m (for configuration 5 this is the covariance of the log-magnitudes,
so every coordinate stays lognormal).  Isotropic noise would make every
residual direction equally likely, a structure no real embedding set has.

Seeds: mixture parameters and base rows derive from 1000+cfg, queries from
2000+cfg.  Rows are drawn in chunks of 65536 with their own child seed, so a
smaller ``n`` gives a prefix of the full-size dataset and chunks can be drawn
on several threads.  Queries are fresh draws from the same mixture, never base
points.  All arrays are float32, C-contiguous.
"""
from __future__ import annotations

import dataclasses
from concurrent.futures import ThreadPoolExecutor

import numpy as np

CHUNK = 1 << 16


@dataclasses.dataclass(frozen=True)
class WorkloadConfig:
    cfg: int
    name: str
    n: int
    m: int
    M: int            # HNSW degree cap on levels >= 1 (layer 0 allows 2M)
    ef_construction: int
    r: int            # FINGER rank
    nq: int
    K: int
    ef_grid: tuple
    unit_norm: bool
    precision: str    # "fp32" | "lp" (bf16 rows + fp8 codes)


CONFIGS = {
    1: WorkloadConfig(1, "gauss-mixture-10k-64", 10_000, 64, 16, 100, 16, 200, 10,
                      (10, 20, 50, 100), False, "fp32"),
    2: WorkloadConfig(2, "gamma-int-1M-128", 1_000_000, 128, 16, 200, 64, 10_000, 10,
                      tuple(range(10, 401, 10)), False, "fp32"),
    3: WorkloadConfig(3, "powerlaw-unit-1.2M-100", 1_200_000, 100, 24, 200, 32, 10_000, 10,
                      tuple(range(10, 401, 10)), True, "lp"),
    4: WorkloadConfig(4, "gauss-unit-1M-96", 1_000_000, 96, 16, 200, 24, 10_000, 10,
                      tuple(range(10, 401, 10)), True, "fp32"),
    5: WorkloadConfig(5, "lognormal-1M-960", 1_000_000, 960, 32, 256, 64, 50_000, 10,
                      tuple(range(10, 401, 10)) + tuple(range(450, 1001, 50)), False, "fp32"),
}


def config(cfg: int) -> WorkloadConfig:
    return CONFIGS[cfg]


def _zipf_frame(rng: np.random.Generator, m: int, sigma: float):
    """Random orthonormal frame (m x m) and per-axis standard deviations whose
    variances follow 1/i with total sigma^2 m."""
    R = np.linalg.qr(rng.standard_normal((m, m)))[0]
    lam = 1.0 / np.arange(1, m + 1, dtype=np.float64)
    lam *= sigma ** 2 * m / lam.sum()
    return R, np.sqrt(lam)


def _mixture(cfg: int):
    """Mixture parameters of configuration ``cfg`` (drawn from seed 1000+cfg)."""
    c = CONFIGS[cfg]
    rng = np.random.default_rng(1000 + cfg)
    if cfg == 1:
        centres = rng.standard_normal((16, c.m))
        return dict(kind="gauss", centres=centres, weights=np.full(16, 1 / 16), sigma=0.3)
    if cfg == 2:
        shape = rng.uniform(0.5, 2.0, size=(64, c.m))
        scale = rng.uniform(5.0, 40.0, size=(64, c.m))
        return dict(kind="gamma_int", shape=shape, scale=scale, weights=np.full(64, 1 / 64))
    if cfg == 3:
        centres = rng.standard_normal((256, c.m))
        w = np.arange(1, 257, dtype=np.float64) ** -1.5
        R, sd = _zipf_frame(rng, c.m, 1.0)
        return dict(kind="gauss_unit", centres=centres, weights=w / w.sum(), frame=R, sd=sd)
    if cfg == 4:
        centres = rng.standard_normal((128, c.m))
        R, sd = _zipf_frame(rng, c.m, 0.5)
        return dict(kind="gauss_unit", centres=centres, weights=np.full(128, 1 / 128), frame=R,
                    sd=sd)
    if cfg == 5:
        mu = rng.normal(-2.0, 0.5, size=(32, c.m))
        R, sd = _zipf_frame(rng, c.m, 0.5)
        return dict(kind="lognormal", mu=mu, weights=np.full(32, 1 / 32), frame=R, sd=sd)
    raise KeyError(cfg)


def _draw(mix, m: int, rows: int, rng: np.random.Generator) -> np.ndarray:
    k = rng.choice(len(mix["weights"]), size=rows, p=mix["weights"])
    kind = mix["kind"]
    if kind == "gauss":
        x = mix["centres"][k] + mix["sigma"] * rng.standard_normal((rows, m))
    elif kind == "gauss_unit":
        x = mix["centres"][k] + (rng.standard_normal((rows, m)) * mix["sd"]) @ mix["frame"].T
        x /= np.linalg.norm(x, axis=1, keepdims=True)
    elif kind == "gamma_int":
        x = np.minimum(255.0, np.round(rng.gamma(mix["shape"][k], mix["scale"][k])))
    elif kind == "lognormal":
        x = np.exp(mix["mu"][k] + (rng.standard_normal((rows, m)) * mix["sd"]) @ mix["frame"].T)
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(x, dtype=np.float32)


def _rows(cfg: int, n: int, stream: int, base_seed: int, threads: int) -> np.ndarray:
    c = CONFIGS[cfg]
    mix = _mixture(cfg)
    out = np.empty((n, c.m), dtype=np.float32)
    nchunks = (n + CHUNK - 1) // CHUNK

    def work(i):
        lo, hi = i * CHUNK, min(n, (i + 1) * CHUNK)
        rng = np.random.default_rng([base_seed, stream, i])
        block = _draw(mix, c.m, CHUNK, rng)       # always a full chunk: prefix-stable
        out[lo:hi] = block[: hi - lo]

    if threads > 1 and nchunks > 1:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, range(nchunks)))
    else:
        for i in range(nchunks):
            work(i)
    return out


def base_vectors(cfg: int, n: int | None = None, threads: int = 8) -> np.ndarray:
    """Base rows of configuration ``cfg`` (first ``n`` rows; default: full size)."""
    c = CONFIGS[cfg]
    return _rows(cfg, c.n if n is None else int(n), 1, 1000 + cfg, threads)


def query_vectors(cfg: int, nq: int | None = None, threads: int = 8) -> np.ndarray:
    """Queries of configuration ``cfg``: fresh draws from the same mixture."""
    c = CONFIGS[cfg]
    return _rows(cfg, c.nq if nq is None else int(nq), 2, 2000 + cfg, threads)


def training_queries(cfg: int, nq: int, threads: int = 8) -> np.ndarray:
    """Queries for harvesting predictor training data: fresh draws from the same
    mixture with seed 5000+cfg, disjoint from the test queries (2000+cfg)."""
    return _rows(cfg, nq, 3, 5000 + cfg, threads)


def uneven_batches(total: int = 50_000, seed: int = 2005):
    """Batch plan of the uneven query stream (configuration 5).

    Returns a list of (start, size, K array, ef array): batch sizes
    ceil(2**U(0,12)) until ``total`` queries are used, K uniform in {1,10,100},
    ef uniform in [max(K,10), 400].
    """
    rng = np.random.default_rng([seed, 7])
    plan, start = [], 0
    while start < total:
        size = int(min(total - start, np.ceil(2.0 ** rng.uniform(0, 12))))
        K = rng.choice(np.array([1, 10, 100], dtype=np.int32), size=size)
        lo = np.maximum(K, 10)
        ef = (lo + np.floor(rng.uniform(size=size) * (401 - lo))).astype(np.int32)
        plan.append((start, size, K.astype(np.int32), ef))
        start += size
    return plan
