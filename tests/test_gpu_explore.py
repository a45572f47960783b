"""Exploration queries at the paper's size (Sec. 6.7: indexed queries seeded at their own vertex,
k = 1,000, recall@1000) and at the other k of the 1M x 128 configuration, on integer-valued rows
where float32 distances are exact: the library's results must equal the FP64 oracle's on the same
graph, ties broken by id on both sides.

The graph is built by the library's device builder (a valid DEG is all Alg. 1 needs); the ground
truth of an exploration query is the exact k-NN of x_v over V without v, which knn_exact gives
with k + 1 results minus v."""
import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth
from parity import compare_lists, eps32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 20_000, 64)


@pytest.fixture(scope="module")
def g():
    import paper_2307_10479_gb300 as deg
    base = W.base()
    idx = deg.Index.build_device(base, W.degree, W.k_ext, W.eps_ext)
    adj = idx.adjacency()
    idx.upload(("f32", "bf16"))
    return dict(deg=deg, base=base, idx=idx, adj=adj, v=W.explore_ids(64))


def explore_truth(deg, base, v, k):
    ids, d = deg.knn_exact(torch.from_numpy(base).cuda(), torch.from_numpy(base[v]).cuda(), k + 1)
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    out = np.empty((len(v), k), np.int32)
    for i, (row, vi) in enumerate(zip(ids, v)):
        out[i] = row[row != vi][:k]
    return out


@pytest.mark.parametrize("k", [1, 100, 1000])
def test_exploration_parity_and_recall(g, k):
    idx, base, adj, v = g["idx"], g["base"], g["adj"], g["v"]
    eps = 0.1
    ids, d, st, tr = idx.search(seeds=torch.from_numpy(v).cuda(), explore=True, k=k, eps=eps, with_status=True,
                                with_trace=True)
    ids, d, st, tr = ids.cpu().numpy(), d.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy()
    assert (st == 0).all()
    o_ids, o_d, o_tr = oracle.range_search(base, adj, None, v, k, eps32(eps), explore=True)
    frac, diff = compare_lists(ids, d, o_ids, o_d)
    same = np.ones(len(v), bool)
    same[diff] = False
    assert np.array_equal(tr[same, :2], o_tr[same, :2])                    # hops and evaluations
    assert not np.any(ids == v[:, None])
    truth = explore_truth(g["deg"], base, v, k)
    rec = np.mean([len(set(a) & set(b)) / k for a, b in zip(ids, truth)])
    o_rec = np.mean([len(set(a) & set(b)) / k for a, b in zip(o_ids, truth)])
    assert abs(rec - o_rec) <= 0.001 and rec > 0.5, (rec, o_rec)


@pytest.mark.parametrize("k", [1, 100])
def test_vector_queries_at_k_1_and_100(g, k):
    idx, base, adj = g["idx"], g["base"], g["adj"]
    q = W.queries()
    ids, d, tr = idx.search(torch.from_numpy(q).cuda(), k=k, eps=0.1, with_trace=True)
    o_ids, o_d, o_tr = oracle.range_search(base, adj, q, np.full(len(q), oracle.median_vertex(base), np.int32), k,
                                           eps32(0.1))
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)
    assert np.array_equal(tr.cpu().numpy()[:, :2], o_tr[:, :2])


def test_bf16_exploration_at_k_1000_re_ranks_exactly(g):
    # bf16 holds these integer rows exactly, so the bf16 form with a re-rank equals float32
    idx, v = g["idx"], g["v"]
    a_ids, a_d = idx.search(seeds=torch.from_numpy(v).cuda(), explore=True, k=1000, eps=0.1)
    b_ids, b_d = idx.search(seeds=torch.from_numpy(v).cuda(), explore=True, k=1000, eps=0.1, precision="bf16",
                            rerank=1000)
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)
