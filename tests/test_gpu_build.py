"""Graph construction on the device: batched ExtendGraph (Alg. 3, scheme C with RNG checks),
batched optimizeEdge (Alg. 4) for the new edges, and batched dynamicEdgeOptimization (Alg. 5).

The device builder makes a different graph than the sequential oracle (batches, claims, the order
the warps run in), so it is held to what both must satisfy and to search quality:
- the structural invariants of the paper's graphs, checked by the oracle: every vertex has
  exactly d neighbours, the adjacency is symmetric, no loops or duplicates, BFS-connected (on the
  smallest graphs also bridge-free, App. B's 2-edge connectivity);
- Alg. 1 on the device-built graph reaches the recall of Alg. 1 on the sequential oracle's graph
  within 0.02 at the same eps (both searched by the oracle, FP64), with and without optimizeEdge;
- Alg. 5 lowers the average neighbour distance it minimises (Sec. 5.3) and keeps the invariants;
- the library's search on the device-built graph is the oracle's search on it (parity)."""
import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth
from parity import compare_lists, eps32, recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["uniform-10k-d32"]


def _params(i_opt):
    return dict(k_opt=W.k_opt, eps_opt=W.eps_opt, i_opt=i_opt)


@pytest.fixture(scope="module")
def built():
    import paper_2307_10479_gb300 as deg
    base, q = W.base(), W.queries()
    full = deg.Index.build_device(base, W.degree, W.k_ext, W.eps_ext, **_params(W.i_opt))
    plain = deg.Index.build_device(base, W.degree, W.k_ext, W.eps_ext, **_params(0))
    gt, _ = oracle.knn_bruteforce(base, q, 10)
    return dict(deg=deg, base=base, q=q, idx=full, adj=full.adjacency(), adj0=plain.adjacency(), gt=gt)


def test_device_graph_invariants(built):
    for adj in (built["adj"], built["adj0"]):
        assert adj.shape == (W.n, W.degree)
        assert oracle.check_graph(adj) == 0


@pytest.mark.parametrize("i_opt", [0, 5])
def test_device_graph_search_quality_against_the_oracle_graph(built, i_opt):
    # the sequential oracle's graph with the same parameters; i_opt = 0 leaves out the optional
    # optimizeEdge of Alg. 3 on both sides (the paper's construction-only graph)
    base, q, gt = built["base"], built["q"], built["gt"]
    g_adj = built["adj"] if i_opt else built["adj0"]
    o_adj = oracle.build_graph(base, W.degree, W.k_ext, W.eps_ext, W.k_opt, W.eps_opt, i_opt)
    entry = np.full(len(q), oracle.median_vertex(base), np.int32)
    for eps in (0.1, 0.2):
        g_ids, _, g_tr = oracle.range_search(base, g_adj, q, entry, 10, eps)
        o_ids, _, o_tr = oracle.range_search(base, o_adj, q, entry, 10, eps)
        print(f"i_opt {i_opt} eps {eps}: device {recall(g_ids, gt):.4f} ({g_tr[:, 1].mean():.0f} evals), "
              f"sequential {recall(o_ids, gt):.4f} ({o_tr[:, 1].mean():.0f} evals)")
        assert recall(g_ids, gt) >= recall(o_ids, gt) - 0.02, (eps, recall(g_ids, gt), recall(o_ids, gt))


def test_search_parity_on_the_device_graph(built):
    idx, base, q, adj = built["idx"], built["base"], built["q"], built["adj"]
    idx.upload()
    ids, d = idx.search(torch.from_numpy(q).cuda(), k=10, eps=0.1)
    o_ids, o_d, _ = oracle.range_search(base, adj, q, np.full(len(q), oracle.median_vertex(base), np.int32), 10,
                                        eps32(0.1))
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)


def test_refinement_lowers_the_average_neighbour_distance(built):
    deg, base = built["deg"], built["base"]
    idx = deg.Index.from_arrays(base, built["adj0"])
    before = oracle.average_neighbor_distance(base, built["adj0"])
    improved = idx.refine_device(20_000, W.k_opt, W.eps_opt, W.i_opt, seed=11)
    adj = idx.adjacency()
    after = oracle.average_neighbor_distance(base, adj)
    print(f"Alg. 5, 20,000 rounds: {improved} edges improved, AND {before:.5f} -> {after:.5f}")
    assert oracle.check_graph(adj) == 0
    assert improved > 0 and after < before
    idx.upload()                                              # the refined graph searches as usual
    ids, _ = idx.search(torch.from_numpy(built["q"][:64]).cuda(), k=10, eps=0.1)
    assert (ids.cpu().numpy() >= 0).all()


@pytest.mark.parametrize("degree,batch_div,i_opt", [(30, 256, 5), (30, 2, 5), (8, 1, 5), (8, 1, 0)])
def test_invariants_under_heavy_contention(degree, batch_div, i_opt):
    # batch_div 1-2: a batch as large as half the graph, so new vertices compete for the same old
    # vertices and some run out of candidates and are inserted again later; their optimisations
    # compete too and some are undone and repeated
    import paper_2307_10479_gb300 as deg
    w = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 6_000, 10)
    base = w.base()
    idx = deg.Index.build_device(base, degree, 2 * degree, 0.2, k_opt=degree, eps_opt=0.001, i_opt=i_opt,
                                 batch_div=batch_div)
    adj = idx.adjacency()
    assert oracle.check_graph(adj, bridge_max_n=6_000 if degree == 8 else 0) == 0


def test_smallest_graphs_and_bad_arguments():
    import paper_2307_10479_gb300 as deg
    base = synth.uniform(10, 4, 3)
    adj = deg.Index.build_device(base[:9], 8, 8, 0.2).adjacency()       # K_9 itself
    assert oracle.check_graph(adj) == 0
    assert all(set(adj[u]) == set(range(9)) - {u} for u in range(9))
    assert oracle.check_graph(deg.Index.build_device(base, 8, 8, 0.2, i_opt=5, k_opt=8).adjacency()) == 0
    for kw in (dict(degree=7, k_ext=8), dict(degree=8, k_ext=4), dict(degree=130, k_ext=130),
               dict(degree=8, k_ext=8, i_opt=7), dict(degree=8, k_ext=8, refine_rounds=5)):
        with pytest.raises(deg.DegError):
            deg.Index.build_device(synth.uniform(200, 4, 3), eps_ext=0.2, **kw)
    with pytest.raises(deg.DegError):
        deg.Index.build_device(base, 8, 8, 0.2, batch_div=0)


def test_insert_grows_a_graph_like_a_build():
    # a graph over the first 6,000 rows, then the last 2,000 inserted by deg_insert_device: the
    # invariants hold over all 8,000, and Alg. 1 finds the new vertices as well as the old
    import paper_2307_10479_gb300 as deg
    w = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 8_000, 200)
    base, q = w.base(), w.queries()
    idx = deg.Index.build_device(base[:6000], 30, 60, 0.2, k_opt=30, i_opt=5)
    idx.insert_device(base[6000:], 60, 0.2, k_opt=30, i_opt=5)
    n, dim, degree = idx.info()
    adj = idx.adjacency()
    assert (n, degree) == (8000, 30) and oracle.check_graph(adj) == 0
    full = deg.Index.build_device(base, 30, 60, 0.2, k_opt=30, i_opt=5).adjacency()
    gt, _ = oracle.knn_bruteforce(base, q, 10)
    entry = np.full(len(q), oracle.median_vertex(base), np.int32)
    r_ins = recall(oracle.range_search(base, adj, q, entry, 10, 0.1)[0], gt)
    r_full = recall(oracle.range_search(base, full, q, entry, 10, 0.1)[0], gt)
    assert r_ins >= r_full - 0.02, (r_ins, r_full)
    idx.upload()
    ids, _ = idx.search(torch.from_numpy(base[6000:6100]).cuda(), k=1, eps=0.1)
    assert np.mean(ids.cpu().numpy()[:, 0] == np.arange(6000, 6100)) >= 0.99   # new rows find themselves
    with pytest.raises(deg.DegError):
        idx.insert_device(base[:10], 4, 0.2)                 # k_ext below the degree


def test_removal_then_insertion_keeps_search_quality():
    # 8,000 rows built on the device; 2,000 random vertices removed (deg_remove, each re-pairing its
    # neighbours and moving the last vertex into its id); the graph keeps its invariants, Alg. 1 on
    # it reaches the recall of a fresh build over the 6,000 rows left, the library's search on it is
    # the oracle's; the removed rows inserted again find themselves
    import paper_2307_10479_gb300 as deg
    w = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 8_000, 200)
    base, q = w.base(), w.queries()
    idx = deg.Index.build_device(base, 30, 60, 0.2, k_opt=30, i_opt=5)
    rows = np.arange(8000)                         # id -> row of base
    rng = np.random.default_rng(11)
    for _ in range(2000):
        v = int(rng.integers(len(rows)))
        moved = idx.remove(v)
        if moved >= 0:
            rows[v] = rows[moved]
        rows = rows[:-1]
    n, _, degree = idx.info()
    adj = idx.adjacency()
    assert (n, degree) == (6000, 30) and oracle.check_graph(adj) == 0
    left = base[rows]
    fresh = deg.Index.build_device(left, 30, 60, 0.2, k_opt=30, i_opt=5).adjacency()
    gt, _ = oracle.knn_bruteforce(left, q, 10)
    entry = np.full(len(q), oracle.median_vertex(left), np.int32)
    r_rem = recall(oracle.range_search(left, adj, q, entry, 10, 0.1)[0], gt)
    r_new = recall(oracle.range_search(left, fresh, q, entry, 10, 0.1)[0], gt)
    assert r_rem >= r_new - 0.02, (r_rem, r_new)
    idx.upload()
    ids, d = idx.search(torch.from_numpy(q).cuda(), k=10, eps=0.1)
    o_ids, o_d, _ = oracle.range_search(left, adj, q, entry, 10, eps32(0.1))
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)
    gone = np.setdiff1d(np.arange(8000), rows)
    idx.insert_device(base[gone], 60, 0.2, k_opt=30, i_opt=5)
    assert idx.info()[0] == 8000 and oracle.check_graph(idx.adjacency()) == 0
    idx.upload()
    ids, _ = idx.search(torch.from_numpy(base[gone[:100]]).cuda(), k=1, eps=0.1)
    assert np.mean(ids.cpu().numpy()[:, 0] == np.arange(6000, 6100)) >= 0.99
