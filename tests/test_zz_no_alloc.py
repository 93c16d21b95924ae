"""finger_search_noalloc, the search entry point that allocates nothing.

Some callers cannot allocate device memory while they run queries: serving
processes that reserve their memory budget at start-up, and loops for which a
cudaMalloc/cudaFree (possible device synchronisation, unbounded latency) is not
allowed on the query path.  For them the library offers finger_search_noalloc,
whose scratch is a fixed device array inside the library.  This test calls it
through the C ABI twice in a row (the second call sees the array as the first
left it) and checks both results against finger_search.  It lives in its own
file, collected last, and builds its own index so that it runs the same alone
in a fresh process and after the other tests.
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
