"""Graph construction on the device (batched ExtendGraph, Alg. 3 scheme C with RNG checks).

The device builder makes a different graph than the sequential oracle (batches, claims, no edge
optimisation), so it is held to what both must satisfy and to search quality:
- the structural invariants of the paper's graphs, checked by the oracle: every vertex has
  exactly d neighbours, the adjacency is symmetric, no loops or duplicates, BFS-connected (on a
  small graph also bridge-free, App. B's 2-edge connectivity);
- Alg. 1 on the device-built graph reaches the recall of Alg. 1 on the oracle's graph within a
  stated margin at the same eps (both searched by the oracle, FP64);
- the library's search on the device-built graph is the oracle's search on it (parity)."""
import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth
from parity import compare_lists, eps32, recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["uniform-10k-d32"]


@pytest.fixture(scope="module")
def built():
    import paper_2307_10479_gb300 as deg
    base, q = W.base(), W.queries()
    idx = deg.Index.build_device(base, W.degree, W.k_ext, W.eps_ext)
    adj = idx.adjacency()
    gt, _ = oracle.knn_bruteforce(base, q, 10)
    return dict(deg=deg, base=base, q=q, idx=idx, adj=adj, gt=gt)


def test_device_graph_invariants(built):
    adj = built["adj"]
    assert adj.shape == (W.n, W.degree)
    assert oracle.check_graph(adj) == 0


def test_device_graph_search_quality_against_the_oracle_graph(built):
    base, q, gt = built["base"], built["q"], built["gt"]
    # the sequential oracle's construction-only graph (i_opt = 0: the optional optimizeEdge of
    # Alg. 3 never changes an edge), the same algorithm the device runs in batches
    o_adj = oracle.build_graph(base, W.degree, W.k_ext, W.eps_ext, W.k_opt, W.eps_opt, 0)
    entry = np.full(len(q), oracle.median_vertex(base), np.int32)
    for eps in (0.1, 0.2):
        g_ids, _, g_tr = oracle.range_search(base, built["adj"], q, entry, 10, eps)
        o_ids, _, o_tr = oracle.range_search(base, o_adj, q, entry, 10, eps)
        print(f"eps {eps}: device {recall(g_ids, gt):.4f} ({g_tr[:, 1].mean():.0f} evals), "
              f"sequential {recall(o_ids, gt):.4f} ({o_tr[:, 1].mean():.0f} evals)")
        assert recall(g_ids, gt) >= recall(o_ids, gt) - 0.02, (eps, recall(g_ids, gt), recall(o_ids, gt))


def test_search_parity_on_the_device_graph(built):
    idx, base, q, adj = built["idx"], built["base"], built["q"], built["adj"]
    idx.upload()
    ids, d = idx.search(torch.from_numpy(q).cuda(), k=10, eps=0.1)
    o_ids, o_d, _ = oracle.range_search(base, adj, q, np.full(len(q), oracle.median_vertex(base), np.int32), 10,
                                        eps32(0.1))
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)


@pytest.mark.parametrize("degree,batch_div", [(30, 256), (30, 2), (8, 1)])
def test_invariants_under_heavy_contention(degree, batch_div):
    # batch_div 1-2: a batch as large as half the graph, so new vertices compete for the same old
    # vertices and some run out of candidates and are inserted again later
    import paper_2307_10479_gb300 as deg
    w = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 6_000, 10)
    base = w.base()
    idx = deg.Index.build_device(base, degree, 2 * degree, 0.2, batch_div=batch_div)
    adj = idx.adjacency()
    assert oracle.check_graph(adj, bridge_max_n=6_000 if degree == 8 else 0) == 0


def test_smallest_graphs_and_bad_arguments():
    import paper_2307_10479_gb300 as deg
    base = synth.uniform(10, 4, 3)
    adj = deg.Index.build_device(base[:9], 8, 8, 0.2).adjacency()       # K_9 itself
    assert oracle.check_graph(adj) == 0
    assert all(set(adj[u]) == set(range(9)) - {u} for u in range(9))
    assert oracle.check_graph(deg.Index.build_device(base, 8, 8, 0.2).adjacency()) == 0
    for kw in (dict(degree=7, k_ext=8), dict(degree=8, k_ext=4), dict(degree=130, k_ext=130)):
        with pytest.raises(deg.DegError):
            deg.Index.build_device(synth.uniform(200, 4, 3), eps_ext=0.2, **kw)
    with pytest.raises(deg.DegError):
        deg.Index.build_device(base, 8, 8, 0.2, batch_div=0)
