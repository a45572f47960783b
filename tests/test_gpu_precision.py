"""Reduced-precision storage (BF16, FP8 E4M3 with per-row scales) with a float32 re-rank:
the device's codes are bit-identical to the oracle's quantizers, and the search over them
matches the oracle's search over the decoded rows followed by the same re-rank."""
import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth
from parity import compare_lists, recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2307_10479_gb300 as deg
    w = synth.scaled(synth.WORKLOADS["mix-1m-d960"], 4_000, 300)
    base, q = w.base(), w.queries()
    # a small 960-d graph: the precision workload's dimension with the Enron row's parameters
    adj = oracle.build_graph(base, 16, 32, 0.3, 16, 0.001, 5)
    idx = deg.Index.from_arrays(base, adj)
    idx.upload(("f32", "bf16", "fp8"))
    gt, _ = oracle.knn_bruteforce(base, q, 10)
    return dict(deg=deg, base=base, q=q, adj=adj, idx=idx, gt=gt, qd=torch.from_numpy(q).cuda(),
                entry=oracle.median_vertex(base))


def test_device_codes_match_oracle_quantizers(setup):
    idx, base = setup["idx"], setup["base"]
    assert np.array_equal(idx.export_codes("bf16"), oracle.quantize_bf16(base))
    c, s = idx.export_codes("fp8")
    oc, os_ = oracle.quantize_fp8(base)
    assert np.array_equal(s, os_) and np.array_equal(c, oc)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("keep", [10, 64])
def test_reduced_precision_search_parity(setup, precision, keep):
    idx, base, adj, q = setup["idx"], setup["base"], setup["adj"], setup["q"]
    codes = oracle.quantize_bf16(base) if precision == "bf16" else oracle.quantize_fp8(base)
    dec = oracle.decode(precision, *(codes if precision == "fp8" else (codes,)))
    eps = 0.1
    ids, d = idx.search(setup["qd"], k=10, eps=eps, precision=precision, rerank=keep)
    o_ids, o_d = oracle.range_search_decoded(dec, base, adj, q, np.full(len(q), setup["entry"], np.int32), 10, eps,
                                             keep=keep)
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d, min_identical=0.99)
    # the re-ranked distances are the float32-row distances of the returned ids
    ids_np = ids.cpu().numpy()
    true = np.sqrt(((base[ids_np].astype(np.float64) - q[:, None, :]) ** 2).sum(-1))
    np.testing.assert_allclose(d.cpu().numpy(), true, rtol=1e-5)


def test_reduced_precision_distance_error_and_recall(setup):
    # Report-style bounds: BF16 keeps 8 mantissa bits (|err| <= 2^-9 relative per element),
    # FP8 3 bits; with a 64-wide re-rank the recall loss against float32 stays small.
    idx, gt = setup["idx"], setup["gt"]
    f_ids, _ = idx.search(setup["qd"], k=10, eps=0.1)
    r32 = recall(f_ids.cpu().numpy(), gt)
    for precision in ("bf16", "fp8"):
        ids, _ = idx.search(setup["qd"], k=10, eps=0.1, precision=precision, rerank=64)
        assert recall(ids.cpu().numpy(), gt) >= r32 - 0.05
