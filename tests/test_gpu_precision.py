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
    # The distances the kernel computes on the stored codes (rerank=-1: no re-rank) against FP64
    # on the float32 rows, pair by pair, within the bound the formats and float32 give:
    #   |d_kernel - delta| <= |x - s decode(x)|                  (storage, triangle inequality)
    #                        + float32 accumulation of the kernel's sum,
    # and the storage term within the mantissa widths: 2^-9 |x| for bf16 (8 significant bits,
    # round to nearest), 2^-4 |x| + 2^-10 s sqrt(dim) for E4M3 (4 significant bits, subnormal
    # spacing 2^-9 s). The accumulation term: bf16 sums (q - x)^2 directly, relative error at most
    # (dim + 8) 2^-24 of the distance; FP8 expands |q|^2 - 2 s q.x + s^2 |x|^2, absolute error of
    # the square at most (dim + 8) 2^-24 (|q| + s |x|)^2, so of the distance at most its root.
    idx, gt, base, q = setup["idx"], setup["gt"], setup["base"], setup["q"]
    dim = base.shape[1]
    u = 2.0 ** -24 * (dim + 8)
    qs = q.astype(np.float64)
    f_ids, _ = idx.search(setup["qd"], k=10, eps=0.1)
    r32 = recall(f_ids.cpu().numpy(), gt)
    for precision in ("bf16", "fp8"):
        ids, d = idx.search(setup["qd"], k=10, eps=0.1, precision=precision, rerank=-1)
        ids, d = ids.cpu().numpy(), d.cpu().numpy().astype(np.float64)
        if precision == "bf16":
            xs = oracle.decode("bf16", oracle.quantize_bf16(base)).astype(np.float64)
            s = np.ones(len(base))
        else:
            codes, sc = oracle.quantize_fp8(base)
            xs = oracle.decode("fp8", codes, sc).astype(np.float64)          # s * decode(x)
            s = sc.astype(np.float64)
        x = base[ids].astype(np.float64)
        xq = xs[ids]
        exact = np.sqrt(((x - qs[:, None, :]) ** 2).sum(-1))
        stored = np.sqrt(((xq - qs[:, None, :]) ** 2).sum(-1))
        store_err = np.sqrt(((x - xq) ** 2).sum(-1))
        xn = np.sqrt((x ** 2).sum(-1))
        fmt = 2.0 ** -9 * xn if precision == "bf16" else 2.0 ** -4 * xn + 2.0 ** -10 * s[ids] * np.sqrt(dim)
        assert (store_err <= fmt * (1 + 1e-9)).all()
        if precision == "bf16":
            arith = u * stored
        else:
            qn = np.sqrt((qs ** 2).sum(-1))[:, None]
            arith = np.sqrt(u) * (qn + np.sqrt((xq ** 2).sum(-1)))
        err = np.abs(d - exact)
        assert (err <= store_err + arith + 1e-6 * exact).all(), precision
        rel = err / exact
        print(f"{precision}: max relative distance error vs FP64 {rel.max():.3e} (mean {rel.mean():.3e}) "
              f"over {rel.size} pairs")
        r_ids, _ = idx.search(setup["qd"], k=10, eps=0.1, precision=precision, rerank=64)
        assert recall(r_ids.cpu().numpy(), gt) >= r32 - 0.05
