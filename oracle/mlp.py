"""FP64 oracle of the learned angle predictor (an extension of FINGER; the paper
has no learned predictor).  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The predictor replaces the distribution-matching step of Algorithm 3: instead
of t = (t_hat - mu_hat) sigma / sigma_hat + mu it predicts cos(q_res, d_res)
from r + 4 features of one (q, c, d) triple:
    f = [u_q * u_d (r values, their sum is t_hat), t_hat,
         ||q_res|| / ||q||, ||d_res|| / ||d||, a / (|a| + |b| + 1e-6)]
with u_q = P q_res / ||P q_res||, u_d = P d_res / ||P d_res||, a = c^T q / c^T c,
b = c^T d / c^T c.  Network: r+4 -> 64 -> 64 -> 1 with ReLU, BF16 weights,
FP32 accumulation; the inputs of the two hidden layers are rounded to BF16
(round to nearest even) as a tensor-core operand would be; biases are FP32;
the last layer takes the FP32 second hidden layer.  The estimate then uses
t = prediction + eps', eps' = mean |prediction - target| on held-out triples.

Weights are a flat FP32 vector in the order W1 (64 x nf, row j = hidden unit
j), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1).
"""
from __future__ import annotations

import numpy as np

H = 64


def n_weights(nf: int) -> int:
    return H * nf + H + H * H + H + H + 1


def unpack(w: np.ndarray, nf: int):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    W1 = w[o:o + H * nf].reshape(H, nf); o += H * nf
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    w3 = w[o:o + H]; o += H
    b3 = w[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via FP32, returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def quantize_weights(w: np.ndarray, nf: int) -> np.ndarray:
    """The stored model: BF16 W1, W2, w3; FP32 biases."""
    W1, b1, W2, b2, w3, b3 = unpack(w, nf)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731
    return pack(bf16(W1), f32(b1), bf16(W2), f32(b2), bf16(w3), float(np.float32(b3)))


def init(nf: int, seed: int) -> np.ndarray:
    """He-uniform initial weights (FP32 values), zero biases."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (H, nf)) * np.sqrt(6.0 / nf)
    W2 = rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / H)
    w3 = rng.uniform(-1, 1, H) * np.sqrt(6.0 / H)
    w = pack(W1, np.zeros(H), W2, np.zeros(H), w3, 0.0)
    return np.asarray(w, np.float32).astype(np.float64)


def forward(w: np.ndarray, X: np.ndarray, nf: int, round_act: bool = True):
    """Returns (y, cache).  round_act rounds the hidden layers' inputs to BF16."""
    W1, b1, W2, b2, w3, b3 = unpack(w, nf)
    X = np.asarray(X, np.float64)
    x = bf16(X) if round_act else X
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    h1q = bf16(h1) if round_act else h1
    z2 = h1q @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, (x, z1, h1q, z2, h2)


def loss_and_grad(w: np.ndarray, X: np.ndarray, t: np.ndarray, nf: int, round_act: bool = True):
    """Mean squared error and its gradient w.r.t. the flat weights.  Rounding
    of activations is treated as the identity in the backward pass."""
    W1, b1, W2, b2, w3, b3 = unpack(w, nf)
    y, (x, z1, h1q, z2, h2) = forward(w, X, nf, round_act)
    n = len(y)
    r = y - np.asarray(t, np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    dw3 = h2.T @ dy
    db3 = dy.sum()
    dz2 = np.outer(dy, w3) * (z2 > 0)
    dW2 = dz2.T @ h1q
    db2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    dW1 = dz1.T @ x
    db1 = dz1.sum(0)
    return loss, pack(dW1, db1, dW2, db2, dw3, db3)


def features(q, c, d, P) -> tuple[np.ndarray, float]:
    """Features and target cos(q_res, d_res) of one triple from explicit FP64
    vectors (Eq. 1 applied to q and d)."""
    q, c, d, P = (np.asarray(v, np.float64) for v in (q, c, d, P))
    cc = c @ c
    a = (c @ q) / cc if cc > 0 else 0.0
    b = (c @ d) / cc if cc > 0 else 0.0
    qr = q - a * c
    dr = d - b * c
    pq, pd = P @ qr, P @ dr
    npq, npd = np.linalg.norm(pq), np.linalg.norm(pd)
    uq = pq / npq if npq > 0 else np.zeros_like(pq)
    ud = pd / npd if npd > 0 else np.zeros_like(pd)
    prod = uq * ud
    that = prod.sum()
    nq_, nqr, nd_, ndr = (np.linalg.norm(v) for v in (q, qr, d, dr))
    f = np.concatenate([prod, [that, nqr / nq_ if nq_ > 0 else 0.0,
                               ndr / nd_ if nd_ > 0 else 0.0, a / (abs(a) + abs(b) + 1e-6)]])
    den = nqr * ndr
    target = float(qr @ dr / den) if den > 0 else 0.0
    return f, target
