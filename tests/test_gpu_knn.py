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
