"""Shared comparison of CUDA search results with the FP64 oracle (imported by
the GPU parity tests; holds no method arithmetic).

Bars (Algorithm 1 / Algorithm 4 results): result lists identical to the
oracle's on >= 99 % of queries (ties ordered by FP32 distance then id, the
kernel's precision), per-pair distances within 1e-5 relative of FP64, recall@K
within 0.002 of the oracle's.  Traversal counters must be equal on >= 97 % of
the queries whose lists match: an estimate that lies within FP32 rounding of
ub can take the other side of the gate than in FP64 without changing the
list, which changes that query's skipped/exact counters (a reading of the
gate's strict comparison at the kernel's precision).  The measured fraction
is printed so every run records it.
"""
import numpy as np

import oracle

REL = 1e-5


def gpu_search(ix, q, K, ef, mode, warmup=5):
    import torch
    ix.set_mode(mode, warmup)
    cnt = torch.zeros((q.shape[0], 8), dtype=torch.int32, device="cuda")
    ix.set_counters(cnt)
    ids, d = ix.search(q, K, ef)
    torch.cuda.synchronize()
    ix.sync()
    ix.set_counters(None)
    return ids.cpu().numpy(), d.cpu().numpy(), cnt.cpu().numpy()


def fp32_canonical(oi, od):
    """The oracle's lists reordered by (FP32 distance, id): the kernel computes
    distances in FP32 and breaks exact ties by id, so two entries whose FP64
    distances differ below FP32 resolution are a tie at the kernel's precision
    (their order is not unique; the set and the traversal still are)."""
    d32 = od.astype(np.float32)
    out = oi.copy()
    for qi in range(oi.shape[0]):
        valid = oi[qi] >= 0
        order = np.lexsort((oi[qi][valid], d32[qi][valid]))
        out[qi, :valid.sum()] = oi[qi][valid][order]
    return out


def compare(gi, gd, gc, oi, od, oc, gt, K, what, min_lists=0.99, min_counters=0.97):
    """Assert the parity bars; returns the measured fractions."""
    oi = fp32_canonical(oi, od)
    od = np.sort(od, axis=1)
    match = (gi == oi).all(axis=1)
    assert match.mean() >= min_lists, f"{what}: {match.mean():.4f} of lists identical"
    ok = oi[match] >= 0
    rel = np.abs(gd[match][ok] - od[match][ok]) / np.maximum(od[match][ok], 1e-30)
    assert rel.max() < REL, f"{what}: max rel distance error {rel.max():.2e}"
    same = np.ones(int(match.sum()), bool)
    if gc is not None and oc is not None:
        same = (gc[match][:, :7] == oc[match][:, :7]).all(axis=1)
        diff = np.abs(gc[match][~same][:, :7].astype(np.int64) - oc[match][~same][:, :7]).sum(0)
        print(f"{what}: lists identical {match.mean():.4f}, counters equal on "
              f"{same.mean():.4f} of those (counter differences summed: {diff.tolist()})")
        assert same.mean() >= min_counters, f"{what}: counters equal on {same.mean():.4f}; diff {diff}"
    r_g, r_o = oracle.recall(gi, gt, K), oracle.recall(oi, gt, K)
    assert abs(r_g - r_o) <= 0.002, f"{what}: recall {r_g} vs oracle {r_o}"
    return float(match.mean()), float(same.mean())
