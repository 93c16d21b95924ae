"""Full-size checks on the SIFT-like workload (1,000,000 x 128, the benchmark's
configuration: GPU HNSW graph with 200 exact candidates, r = 64, 10,000
queries, K = 10, FINGER at ef = 140 and plain at ef = 130).

The oracle cannot search the GPU-built graph (no oracle input may come from
the CUDA path), so at this size the checks are what the oracle computes one
by one and properties that hold at any size:
* exact kNN on the tensor cores = FP64 brute force on sampled queries;
* every returned distance is the FP64 distance of the returned id (within the
  1e-5 relative bar); lists are sorted by (distance, id), ids unique and valid;
* FINGER with skipping disabled is plain search, exactly;
* the batched and the allocation-free entry points return what finger_search
  returns;
* recall@10 of the benchmark's settings against FP64 brute force.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_11408_gb300 as fg  # noqa: E402

NQ, K, EF_F, EF_P = 10000, 10, 140, 130
SAMPLE = 48


@pytest.fixture(scope="module")
def sift():
    c = workloads.config(2)
    X = workloads.base_vectors(2)
    Q = workloads.query_vectors(2, NQ)
    ix = fg.Index(X)
    ix.build_graph(c.M, candidates=c.ef_construction, level_seed=3002)
    ix.build_tables(c.r, 4002)
    q = torch.from_numpy(Q).cuda()
    sel = np.random.default_rng(17).choice(NQ, SAMPLE, replace=False)
    gt, gd = oracle.bruteforce(X, Q[sel], K)
    yield dict(X=X, Q=Q, q=q, ix=ix, sel=sel, gt=gt, gd=gd)
    ix.close()


def _check_lists(X, Q, ids, d, sel):
    assert ((ids >= 0) & (ids < X.shape[0])).all()
    for row in ids:
        assert len(set(row.tolist())) == len(row)
    keys_sorted = (d[:, 1:] > d[:, :-1]) | ((d[:, 1:] == d[:, :-1]) & (ids[:, 1:] > ids[:, :-1]))
    assert keys_sorted.all()
    Xd = X.astype(np.float64)
    for i in sel:
        exact = ((Xd[ids[i]] - Q[i].astype(np.float64)) ** 2).sum(1)
        np.testing.assert_allclose(d[i], exact, rtol=1e-5)


def test_tensor_core_ground_truth_is_exact(sift):
    ids, d = sift["ix"].knn(sift["q"][sift["sel"]], K)
    torch.cuda.synchronize()
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    assert (ids == sift["gt"]).mean() > 0.999
    np.testing.assert_allclose(d, sift["gd"], rtol=1e-5)


@pytest.mark.parametrize("mode,ef", [(fg.MODE_FINGER, EF_F), (fg.MODE_PLAIN, EF_P)])
def test_results_are_exact_sorted_and_accurate(sift, mode, ef):
    ix = sift["ix"]
    ix.set_mode(mode, 5)
    ids, d = ix.search(sift["q"], K, ef)
    ix.sync()
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    _check_lists(sift["X"], sift["Q"], ids, d, sift["sel"])
    rec = oracle.recall(ids[sift["sel"]], sift["gt"], K)
    assert rec >= 0.9, rec


def test_finger_without_skipping_is_plain_at_full_size(sift):
    ix = sift["ix"]
    ix.set_mode(fg.MODE_PLAIN, 5)
    i0, d0 = ix.search(sift["q"], K, EF_F)
    ix.set_mode(fg.MODE_FINGER, 10 ** 9)
    i1, d1 = ix.search(sift["q"], K, EF_F)
    ix.sync()
    assert torch.equal(i0, i1) and torch.equal(d0, d1)


def test_batch_and_noalloc_equal_search_at_full_size(sift):
    ix = sift["ix"]
    ix.set_mode(fg.MODE_FINGER, 5)
    q = sift["q"][:4096]
    ids, d = ix.search(q, K, EF_F)
    Kt = torch.full((q.shape[0],), K, dtype=torch.int32, device="cuda")
    eft = torch.full((q.shape[0],), EF_F, dtype=torch.int32, device="cuda")
    bi, bd, off = ix.search_batch(q, Kt, eft)
    ni = torch.empty_like(ids)
    nd = torch.empty_like(d)
    ix.search_noalloc(q, K, EF_F, ni, nd)
    ix.sync()
    assert torch.equal(bi.view(-1, K), ids) and torch.equal(bd.view(-1, K), d)
    assert torch.equal(ni, ids) and torch.equal(nd, d)
