"""finger_search_noalloc, the search entry point that allocates nothing.

Some callers cannot allocate device memory while they run queries: serving
processes that reserve their memory budget at start-up, and loops for which a
cudaMalloc/cudaFree (possible device synchronisation, unbounded latency) is not
allowed on the query path.  For them the library offers finger_search_noalloc,
whose scratch is a fixed device array inside the library.  This test calls it
through the C ABI twice in a row (the second call sees the array as the first
left it) and checks both results against finger_search.  It lives in its own
file, collected last, and builds its own indexes so that it runs the same
alone in a fresh process and after the other tests.

The array holds a fixed number of per-warp visited bitmaps and spill lists, so
for a large index and a large batch the entry point runs fewer warps than
finger_search (about 233 at 200,000 rows against 2,000 for 2,000 queries);
the second test makes sure that path, with its visited sets spilling to the
bitmaps (ef 200), gives finger_search's results, and that alternating a small
and a large index (whose bitmap regions lie over each other's spill lists)
still starts every call from zeroed bitmaps.  A block smaller than four warps
is only needed above about 1.3e8 rows and is not exercised here.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_11408_gb300 as fg  # noqa: E402


@pytest.fixture(scope="module")
def index():
    X = workloads.base_vectors(1, 5000)
    ix = fg.Index(X)
    ix.build_graph(16, 64, 3001)
    ix.build_tables(16, 4001)
    yield ix
    ix.close()


@pytest.mark.parametrize("mode", [fg.MODE_PLAIN, fg.MODE_FINGER])
def test_noalloc_matches_search_on_two_calls(index, mode):
    ix = index
    nq, K, ef = 300, 10, 64
    q = torch.from_numpy(workloads.query_vectors(1, nq)).cuda()
    ix.set_mode(mode, 5)
    ref_ids, ref_d = ix.search(q, K, ef)
    torch.cuda.synchronize()
    for call in range(2):
        ids = torch.full((nq, K), -7, dtype=torch.int64, device="cuda")
        d = torch.full((nq, K), -1.0, dtype=torch.float32, device="cuda")
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
        ix.search_noalloc(q, K, ef, ids, d)
        torch.cuda.synchronize()
        ix.sync()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] >= free_before - (2 << 20)
        assert torch.equal(ids, ref_ids), f"call {call}: ids differ"
        torch.testing.assert_close(d, ref_d, rtol=1e-5, atol=0.0)


def test_noalloc_rejects_bad_arguments(index):
    q = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    ids = torch.empty((4, 10), dtype=torch.int64, device="cuda")
    d = torch.empty((4, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(fg.FingerError):
        index.search_noalloc(q, 10, 5, ids, d)          # K > ef
    with pytest.raises(fg.FingerError):
        index.search_noalloc(q, 10, 5000, ids, d)       # ef above the 1024 capacity


@pytest.fixture(scope="module")
def large():
    X = workloads.base_vectors(2, 200_000)
    ix = fg.Index(X)
    ix.build_graph(16, 64, 3002)
    ix.build_tables(16, 4002)
    yield ix
    ix.close()


def _noalloc(ix, q, K, ef):
    ids = torch.full((q.shape[0], K), -7, dtype=torch.int64, device="cuda")
    d = torch.full((q.shape[0], K), -1.0, dtype=torch.float32, device="cuda")
    ix.search_noalloc(q, K, ef, ids, d)
    torch.cuda.synchronize()
    ix.sync()          # raises on a latched kernel status (e.g. FINGER_ERR_LIMIT)
    return ids, d


@pytest.mark.parametrize("mode", [fg.MODE_PLAIN, fg.MODE_FINGER])
def test_noalloc_fewer_warps_and_alternating_indexes(index, large, mode):
    K, ef = 10, 200
    qs = torch.from_numpy(workloads.query_vectors(1, 300)).cuda()
    ql = torch.from_numpy(workloads.query_vectors(2, 2000)).cuda()
    refs = {}
    for name, ix, q in (("small", index, qs), ("large", large, ql)):
        ix.set_mode(mode, 5)
        refs[name] = ix.search(q, K, ef)
        torch.cuda.synchronize()
        ix.sync()          # raises on a latched kernel status (e.g. FINGER_ERR_LIMIT)
    # small, large, large, small, large: the large index's bitmaps cover the
    # small index's spill lists and the other way round
    for name in ("small", "large", "large", "small", "large"):
        ix, q = (index, qs) if name == "small" else (large, ql)
        ids, d = _noalloc(ix, q, K, ef)
        ref_ids, ref_d = refs[name]
        assert torch.equal(ids, ref_ids), f"{name}: ids differ"
        torch.testing.assert_close(d, ref_d, rtol=1e-5, atol=0.0)
