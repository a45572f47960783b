"""GPU parity of knn_exact (Eq. 1) against the FP64 oracle's exhaustive search."""
import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth
from parity import compare_lists

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [1, 10, 100, 256])
def test_knn_exact_float_data(k):
    import paper_2307_10479_gb300 as deg
    base = synth.uniform(10_000, 32, 0)
    q = synth.uniform(200, 32, 1)
    ids, d = deg.knn_exact(torch.from_numpy(base).cuda(), torch.from_numpy(q).cuda(), k)
    o_ids, o_d = oracle.knn_bruteforce(base, q, k)
    # float32 vs FP64 distances: a swap is allowed only between distances within 1e-5.
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d, min_identical=0.95 if k > 10 else 0.99)


def test_knn_exact_integer_data_is_bit_exact():
    # SIFT-like integer rows: squared distances <= 128 * 255^2 < 2^24 are exact in float32, so
    # ids (ties broken by id) and distances match the oracle exactly.
    import paper_2307_10479_gb300 as deg
    w = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 30_000, 100)
    base, q = w.base(), w.queries()
    ids, d = deg.knn_exact(torch.from_numpy(base).cuda(), torch.from_numpy(q).cuda(), 100)
    o_ids, o_d = oracle.knn_bruteforce(base, q, 100)
    assert np.array_equal(ids.cpu().numpy(), o_ids)
    assert np.array_equal(d.cpu().numpy().astype(np.float64), o_d.astype(np.float32).astype(np.float64))


def test_knn_exact_ragged_and_chunked_shapes():
    import paper_2307_10479_gb300 as deg
    base = synth.uniform(1_001, 7, 5)                  # odd n, dim not a multiple of 4
    q = synth.uniform(67, 7, 6)
    ids, d = deg.knn_exact(torch.from_numpy(base).cuda(), torch.from_numpy(q).cuda(), 5)
    o_ids, o_d = oracle.knn_bruteforce(base, q, 5)
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d, min_identical=0.98)
    e_ids, _ = deg.knn_exact(torch.from_numpy(base).cuda(), torch.from_numpy(q[:0]).cuda(), 5)
    assert e_ids.shape == (0, 5)
    with pytest.raises(deg.DegError):
        deg.knn_exact(torch.from_numpy(base[:3]).cuda(), torch.from_numpy(q).cuda(), 5)


# ---- the tensor-core path against the CUDA-core path ---------------------------------------
# knn_exact computes distances with tcgen05 (bfloat16 operands, float32 accumulators), keeps every
# row within a proven error bound of the k-th approximate distance and re-ranks those in float32;
# knn_exact_noalloc computes every float32 distance on the CUDA cores. Both sum
# fmaf(q_d - x_d, q_d - x_d, .) in dimension order and order ties by id, so they agree bit for bit.

def _cuda_core(base, q, k):
    import ctypes
    import paper_2307_10479_gb300 as deg
    ids = torch.empty((q.shape[0], k), dtype=torch.int32, device="cuda")
    d = torch.empty((q.shape[0], k), dtype=torch.float32, device="cuda")
    st = deg.lib().knn_exact_noalloc(ctypes.c_void_p(base.data_ptr()), base.shape[0], ctypes.c_void_p(q.data_ptr()),
                                     q.shape[0], base.shape[1], k, ctypes.c_void_p(ids.data_ptr()),
                                     ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == deg.DEG_OK, deg.lib().deg_last_error()
    torch.cuda.synchronize()
    return ids, d


def _both(base, q, k):
    import paper_2307_10479_gb300 as deg
    b, qq = torch.from_numpy(np.ascontiguousarray(base)).cuda(), torch.from_numpy(np.ascontiguousarray(q)).cuda()
    t_ids, t_d = deg.knn_exact(b, qq, k)
    s_ids, s_d = _cuda_core(b, qq, k)
    return t_ids.cpu().numpy(), t_d.cpu().numpy(), s_ids.cpu().numpy(), s_d.cpu().numpy()


@pytest.mark.parametrize("n,dim,nq,k", [
    (10_000, 32, 200, 1), (10_000, 32, 200, 10), (10_000, 32, 300, 100), (10_000, 32, 129, 256),
    (1_001, 7, 67, 5),            # ragged everything; K padded from 7 to 64
    (5_000, 65, 130, 10),         # K padded to 128: two chunks of 64
    (3_000, 300, 50, 10),         # K = 320 > 256: the query tile is staged per chunk
    (1, 16, 3, 1),                # a single row
    (300, 24, 1, 300 // 2),       # n below one 256-row tile
])
def test_tensor_core_path_equals_cuda_core_path_on_float_data(n, dim, nq, k):
    base = synth.uniform(n, dim, 11)
    q = synth.uniform(nq, dim, 12)
    t_ids, t_d, s_ids, s_d = _both(base, q, k)
    assert np.array_equal(t_ids, s_ids)
    assert np.array_equal(t_d.view(np.uint32), s_d.view(np.uint32))


def test_tensor_core_path_signed_and_scaled_data():
    # zero-mean data of large magnitude: approximate distances cancel |q|^2 + |x|^2 against 2 q.x
    rng = np.random.default_rng(4)
    base = (rng.standard_normal((8_000, 48)) * 1e3).astype(np.float32)
    q = (rng.standard_normal((150, 48)) * 1e3).astype(np.float32)
    t_ids, t_d, s_ids, s_d = _both(base, q, 10)
    assert np.array_equal(t_ids, s_ids) and np.array_equal(t_d.view(np.uint32), s_d.view(np.uint32))


def test_tensor_core_path_sampled_threshold_on_integer_rows():
    # 100,000 SIFT-like rows: the threshold comes from every 4th row (32,768-row sample limit)
    w = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 100_000, 257)
    base, q = w.base(), w.queries()
    t_ids, t_d, s_ids, s_d = _both(base, q, 10)
    assert np.array_equal(t_ids, s_ids) and np.array_equal(t_d.view(np.uint32), s_d.view(np.uint32))
    o_ids, o_d = oracle.knn_bruteforce(base, q[:40], 10)
    assert np.array_equal(t_ids[:40], o_ids)


def test_tensor_core_path_all_ties_falls_back_exactly():
    # 20,000 equal rows: every row is a candidate (more than the per-query buffer), so the query
    # is recomputed on the CUDA cores; the answer is the k smallest ids.
    base = np.tile(synth.uniform(1, 32, 3), (20_000, 1))
    base[7] += 0.5                                      # one row farther away
    q = synth.uniform(5, 32, 4)
    t_ids, t_d, s_ids, s_d = _both(base, q, 20)
    assert np.array_equal(t_ids, s_ids) and np.array_equal(t_d.view(np.uint32), s_d.view(np.uint32))
    for row in t_ids:                                   # equal distances: the smallest ids
        assert set(row.tolist()) <= set(range(21))


# ---- nearest of a small row set (the pivot routing's search) ------------------------------

@pytest.mark.parametrize("n,dim", [(39, 32), (781, 128), (4096, 128), (5, 7)])
def test_nearest_rows_matches_exhaustive_search(n, dim):
    import paper_2307_10479_gb300 as deg
    rows = synth.uniform(n, dim, 21)
    q = synth.uniform(1000, dim, 22)
    r, qq = torch.from_numpy(rows).cuda(), torch.from_numpy(q).cuda()
    ids, d = deg.nearest_rows(r, qq)
    s_ids, s_d = _cuda_core(r, qq, 1)                   # float32 CUDA-core exhaustive search
    assert np.array_equal(ids.cpu().numpy(), s_ids.cpu().numpy()[:, 0])
    assert np.array_equal(d.cpu().numpy().view(np.uint32), s_d.cpu().numpy()[:, 0].view(np.uint32))
    o_ids, _ = oracle.knn_bruteforce(rows, q[:100], 1)
    assert (ids.cpu().numpy()[:100] == o_ids[:, 0]).mean() >= 0.99


def test_nearest_rows_overflow_scores_every_row():
    # cap 1: any query with a second row inside the rounding bound is scored against all rows;
    # duplicated rows make every query do that. The answer must not change.
    import paper_2307_10479_gb300 as deg
    base = synth.uniform(600, 16, 23)
    rows = np.concatenate([base, base, base[:100]])       # every row appears at least twice
    q = synth.uniform(300, 16, 24)
    r, qq = torch.from_numpy(rows).cuda(), torch.from_numpy(q).cuda()
    a_ids, a_d = deg.nearest_rows(r, qq, cap=256)
    b_ids, b_d = deg.nearest_rows(r, qq, cap=1)
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)
    assert (a_ids.cpu().numpy() < 600).all()                    # ties go to the lower index
    s_ids, _ = _cuda_core(r, qq, 1)
    assert np.array_equal(a_ids.cpu().numpy(), s_ids.cpu().numpy()[:, 0])
    with pytest.raises(deg.DegError):
        deg.nearest_rows(r, qq, cap=3)
    with pytest.raises(deg.DegError):
        deg.nearest_rows(torch.zeros((4097, 16), device="cuda"), qq)


def test_knn_exact_up_to_k_1024_integer_data_is_bit_exact():
    # k above 256 (the ground truth of k = 1,000 exploration) on integer rows: exact, ties by id
    import paper_2307_10479_gb300 as deg
    w = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 20_000, 40)
    base, q = w.base(), w.queries()
    for k in (257, 1000, 1024):
        ids, d = deg.knn_exact(torch.from_numpy(base).cuda(), torch.from_numpy(q).cuda(), k)
        o_ids, o_d = oracle.knn_bruteforce(base, q, k)
        assert np.array_equal(ids.cpu().numpy(), o_ids)
        assert np.array_equal(d.cpu().numpy().astype(np.float64), o_d.astype(np.float32).astype(np.float64))
    with pytest.raises(deg.DegError):
        deg.knn_exact(torch.from_numpy(base).cuda(), torch.from_numpy(q).cuda(), 1025)
