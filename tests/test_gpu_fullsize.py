"""Full-size parity: the 1M x 128 workload the benchmark times, in the benchmark's calls and launch
configuration (all 10,000 queries in one launch), checked on 200 sampled queries that the FP64
oracle searches one by one from the same graph file.

The rows are integers (the mixture's coordinates are rounded to 0..255), so float32 squared
distances are exact (at most 128 * 255^2 < 2^24). Both sides break exact distance ties by the
caller's id, and the kernel's admission test r^2 (1 + eps)^2 is exact to about 2^-46, so the plain
float32 form must match the oracle's results, hops and evaluations on every sampled query (the
oracle gets the float32 eps the library searched with). The FP8 form computes in
float32 on decoded codes (rounding differs from the oracle's FP64), so it is held to identical
lists on most sampled queries, the same recall, and re-ranked distances equal to the float32
rows'."""
import os

import numpy as np
import pytest

import bench
import oracle
from paper_2307_10479_gb300 import graphs, synth
from parity import compare_lists, eps32, recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["sift-1m-d128"]
SAMPLE = np.arange(0, W.nq, 50)                     # 200 of the 10,000 queries


@pytest.fixture(scope="module")
def full():
    # the host-built graph file when present (40 min to build on one core), else the device
    # builder's graph (about 4 min on a GB300, saved beside it); parity holds on either graph
    base, q = W.base(), W.queries()
    idx = graphs.load_or_build(W, base, builder="device")
    path = graphs.graph_path(W) if os.path.exists(graphs.graph_path(W)) else graphs.graph_path(W, "device")
    idx.upload(("f32", "fp8"))
    adj = bench.read_adjacency(path)                 # the graph, read independently of the library
    qs = q[SAMPLE]
    gt, _ = oracle.knn_bruteforce(base, qs, 10)
    return dict(base=base, q=q, qs=qs, idx=idx, adj=adj, gt=gt, entry=oracle.median_vertex(base),
                qd=torch.from_numpy(q).cuda())


def test_entry_vertex_at_full_size(full):
    assert full["idx"].entry_vertex == full["entry"]


def test_plain_float32_form_matches_the_oracle_exactly(full):
    idx, base, adj, qs = full["idx"], full["base"], full["adj"], full["qs"]
    eps = 0.08                                        # the plain form's operating point (recall 0.957)
    ids, d, st, tr = idx.search(full["qd"], k=10, eps=eps, with_status=True, with_trace=True)
    torch.cuda.synchronize()
    ids, d, st, tr = ids.cpu().numpy(), d.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy()
    assert (st == 0).all()
    o_ids, o_d, o_tr = oracle.range_search(base, adj, qs, np.full(len(qs), full["entry"], np.int32), 10, eps32(eps))
    # 1% of these sampled queries have an exact tie between their 10th and 11th neighbour: both
    # sides keep the lower caller id
    frac, diff = compare_lists(ids[SAMPLE], d[SAMPLE], o_ids, o_d, min_identical=0.999)
    same = np.ones(len(qs), bool)
    same[diff] = False
    assert np.mean(tr[SAMPLE][same, 0] == o_tr[same, 0]) >= 0.999     # hops H
    assert np.mean(tr[SAMPLE][same, 1] == o_tr[same, 1]) >= 0.999     # evaluations E


def test_headline_fp8_form_against_the_oracle(full):
    idx, base, adj, qs, gt = full["idx"], full["base"], full["adj"], full["qs"], full["gt"]
    eps = 0.003                                       # the sampled-pivot fp8 form's operating point (recall 0.950)
    ids, d, st = idx.search(full["qd"], k=10, eps=eps, precision="fp8", rerank=32, entry="pivot",
                            with_status=True)
    torch.cuda.synchronize()
    ids, d, st = ids.cpu().numpy()[SAMPLE], d.cpu().numpy()[SAMPLE], st.cpu().numpy()
    assert (st == 0).all()
    # the oracle's seeds: the nearest pivot p * (n // P), P = min(4096, n // 256), by FP64 brute force
    n = len(base)
    npv = min(4096, n // 256)
    piv = (np.arange(npv) * (n // npv)).astype(np.int32)
    lab, _ = oracle.knn_bruteforce(base[piv], qs, 1)
    codes, scales = oracle.quantize_fp8(base)
    dec = oracle.decode("fp8", codes, scales)
    o_ids, o_d = oracle.range_search_decoded(dec, base, adj, qs, piv[lab[:, 0]], 10, eps32(eps), keep=32)
    del dec
    same = np.all(ids == o_ids, axis=1)
    assert same.mean() >= 0.95, f"{same.mean():.3f} of the sampled lists identical"
    assert abs(recall(ids, gt) - recall(o_ids, gt)) <= 0.01
    np.testing.assert_allclose(d[same], o_d[same], rtol=1e-5)
    # re-ranked: the returned distances are the float32 rows' distances of the returned ids
    true = np.sqrt(((base[ids].astype(np.float64) - qs[:, None, :]) ** 2).sum(-1))
    np.testing.assert_allclose(d, true, rtol=1e-5)


def test_headline_fp8_learned_entry_form_against_the_oracle(full):
    # the bench's headline: fp8 + re-rank 32 from the learned entry points, eps 0.001; the oracle
    # starts each sampled query at the nearest learned entry point (FP64 brute force over them)
    idx, base, adj, qs, gt = full["idx"], full["base"], full["adj"], full["qs"], full["gt"]
    idx.train_entry(len(idx.pivots()), 10)
    piv = idx.pivots(learned=True)
    eps = 0.001
    ids, d, st = idx.search(full["qd"], k=10, eps=eps, precision="fp8", rerank=32, entry="learned", with_status=True)
    torch.cuda.synchronize()
    ids, d, st = ids.cpu().numpy()[SAMPLE], d.cpu().numpy()[SAMPLE], st.cpu().numpy()
    assert (st == 0).all()
    lab, _ = oracle.knn_bruteforce(base[piv], qs, 1)
    codes, scales = oracle.quantize_fp8(base)
    dec = oracle.decode("fp8", codes, scales)
    o_ids, o_d = oracle.range_search_decoded(dec, base, adj, qs, piv[lab[:, 0]], 10, eps32(eps), keep=32)
    del dec
    same = np.all(ids == o_ids, axis=1)
    assert same.mean() >= 0.95, f"{same.mean():.3f} of the sampled lists identical"
    assert abs(recall(ids, gt) - recall(o_ids, gt)) <= 0.01
    true = np.sqrt(((base[ids].astype(np.float64) - qs[:, None, :]) ** 2).sum(-1))
    np.testing.assert_allclose(d, true, rtol=1e-5)
