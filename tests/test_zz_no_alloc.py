"""knn_exact_noalloc: the exhaustive k-NN entry point that allocates no device memory (for
callers that cannot allocate while they run, e.g. a process whose device memory is reserved by
another allocator, or a loop that cannot take cudaMalloc's implicit synchronisation). It must
return what knn_exact returns, call after call, although every call reuses the same static
scratch array. This file sorts last so a stop-at-first-failure run has run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2307_10479_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(lib, base, q, k):
    ids = torch.empty((q.shape[0], k), dtype=torch.int32, device="cuda")
    d = torch.empty((q.shape[0], k), dtype=torch.float32, device="cuda")
    st = lib.knn_exact_noalloc(ctypes.c_void_p(base.data_ptr()), base.shape[0], ctypes.c_void_p(q.data_ptr()),
                               q.shape[0], base.shape[1], k, ctypes.c_void_p(ids.data_ptr()),
                               ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, ids, d


def test_noalloc_knn_matches_knn_exact_on_consecutive_calls():
    import paper_2307_10479_gb300 as deg
    lib = deg.lib()
    # 20,000 rows -> 419 queries per scratch chunk, so 1,000 queries take three chunks
    base = torch.from_numpy(synth.uniform(20_000, 32, 0)).cuda()
    q = torch.from_numpy(synth.uniform(1_000, 32, 1)).cuda()
    ref_ids, ref_d = deg.knn_exact(base, q, 10)
    for _ in range(2):
        st, ids, d = _noalloc(lib, base, q, 10)
        assert st == deg.DEG_OK, lib.deg_last_error()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids)
        np.testing.assert_allclose(d.cpu().numpy(), ref_d.cpu().numpy(), rtol=1e-5)
    # a different shape right after reuses the same scratch
    q2 = torch.from_numpy(synth.uniform(37, 32, 2)).cuda()
    st, ids, d = _noalloc(lib, base, q2, 100)
    r_ids, r_d = deg.knn_exact(base, q2, 100)
    torch.cuda.synchronize()
    assert st == deg.DEG_OK and torch.equal(ids, r_ids)


@pytest.mark.parametrize("n,nq", [(8 << 20, 3), (2, 65535 * 64 + 70)])
def test_noalloc_at_the_chunking_extremes(n, nq):
    # n = 8,388,608 rows fills the scratch with one query per chunk; n = 2 rows with more than
    # 65,535 * 64 queries needs a second chunk because one launch takes at most 65,535 * 64 queries
    import paper_2307_10479_gb300 as deg
    lib = deg.lib()
    g = torch.Generator(device="cuda").manual_seed(5)
    base = torch.rand((n, 4), generator=g, device="cuda")
    q = torch.rand((nq, 4), generator=g, device="cuda")
    ref_ids, ref_d = deg.knn_exact(base, q, 1)
    for _ in range(2):
        st, ids, d = _noalloc(lib, base, q, 1)
        assert st == deg.DEG_OK, lib.deg_last_error()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids)
        assert torch.allclose(d, ref_d, rtol=1e-5, atol=0)


def test_noalloc_rejects_a_base_larger_than_its_scratch():
    import paper_2307_10479_gb300 as deg
    lib = deg.lib()
    base = torch.zeros((64, 4), dtype=torch.float32, device="cuda")
    q = torch.zeros((2, 4), dtype=torch.float32, device="cuda")
    ids = torch.empty((2, 1), dtype=torch.int32, device="cuda")
    d = torch.empty((2, 1), dtype=torch.float32, device="cuda")
    # n above 8,388,608 rows is refused before any launch (only the size is looked at)
    st = lib.knn_exact_noalloc(ctypes.c_void_p(base.data_ptr()), (8 << 20) + 1, ctypes.c_void_p(q.data_ptr()), 2, 4, 1,
                               ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d.data_ptr()), None)
    assert st == deg.DEG_EINVAL and b"static scratch" in lib.deg_last_error()
