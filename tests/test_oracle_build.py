"""Pins for the CPU oracle's construction side (Sec. 5, Alg. 2-5, Eq. 3-4, App. B): structural
invariants the paper proves for every DEG, hand-built geometry for the MRNG lune test, closed
forms for AND and GQ, and the bit-exact revert of a failed edge optimisation."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth


def _sym_edges(adj):
    return {(min(u, v), max(u, v)) for u in range(adj.shape[0]) for v in adj[u]}


@pytest.fixture(scope="module", params=[(4, 60), (8, 400), (6, 150)])
def built(request):
    d, n = request.param
    base = synth.uniform(n, 6, 21 + d)
    adj, w = oracle.build_graph(base, d, 2 * d, 0.2, d, 0.001, 5, with_weights=True)
    return base, adj, w, d


def test_build_structural_invariants(built):
    # Sec. 5.1: even-regular, undirected, no loops; |E| = |V| d / 2; connected (Euler) and
    # bridge-free (2-edge-connected).
    base, adj, _, d = built
    n = adj.shape[0]
    assert oracle.check_graph(adj, bridge_max_n=400) == 0
    assert len(_sym_edges(adj)) == n * d // 2
    deg_in = np.bincount(adj.ravel(), minlength=n)
    assert deg_in.min() == d and deg_in.max() == d      # Table 8 DEG rows: min/max in = d, 0 sources


def test_build_weights_are_distances(built):
    base, adj, w, _ = built
    true = np.sqrt(((base[adj].astype(np.float64) - base[:, None, :].astype(np.float64)) ** 2).sum(-1))
    np.testing.assert_allclose(w, true, rtol=1e-14)


def test_build_cut_set_lower_bound(built):
    # App. B: any vertex set S with |S| <= d has a cut-set of size
    # |B| = 2(|S| d / 2 - |L|) >= |S|(d+1) - |S|^2 >= d.
    base, adj, _, d = built
    n = adj.shape[0]
    if n > 80:
        pytest.skip("subset enumeration only on the smallest graph")
    nbr = [set(r) for r in adj.tolist()]
    for size in range(1, d + 1):
        for S in itertools.combinations(range(n), size):
            Sset = set(S)
            L = sum(1 for u in S for v in nbr[u] if v in Sset) // 2
            B = sum(1 for u in S for v in nbr[u] if v not in Sset)
            assert B == 2 * (size * d // 2 - L)
            assert B >= size * (d + 1) - size * size >= d


def test_first_graph_is_complete():
    # The smallest DEG_d is K_{d+1} (Sec. 5.1).
    base = synth.uniform(7, 3, 30)
    adj = oracle.build_graph(base, 6, 12, 0.2, 6, 0.001, 5)
    for u in range(7):
        assert sorted(adj[u].tolist()) == [v for v in range(7) if v != u]


def test_check_graph_flags_plants():
    base = synth.uniform(40, 4, 31)
    adj = oracle.build_graph(base, 4, 8, 0.2, 4, 0.001, 5)
    assert oracle.check_graph(adj, 40) == 0
    bad = adj.copy(); bad[0, 0] = 0
    assert oracle.check_graph(bad) & 2
    bad = adj.copy(); bad[0, 1] = bad[0, 0]
    assert oracle.check_graph(bad) & 4
    bad = adj.copy(); u, v = 0, adj[0, 0]; bad[0, 0] = [x for x in range(40) if x not in adj[0] and x != 0][0]
    assert oracle.check_graph(bad) & 8
    # two disjoint K5 blocks: regular and symmetric but disconnected
    k5 = np.array([[j for j in range(5) if j != i] for i in range(5)], np.int32)
    two = np.vstack([k5, k5 + 5])
    assert oracle.check_graph(two) == 16


def test_check_graph_detects_bridge():
    # An even-regular graph can have no bridge (Sec. 5.1, Euler), so plant one in a 3-regular
    # graph: two copies of K4 with edge (a,b) subdivided by e, the two e's joined by a bridge.
    one = [[2, 3, 4], [2, 3, 4], [0, 1, 3], [0, 1, 2], [0, 1, 9]]
    two = [[r + 5 if r != 9 else 4 for r in row] for row in one]
    two[4] = [5, 6, 4]
    adj = np.array(one + two, np.int32)
    assert oracle.check_graph(adj, 100) == 32 | 64           # odd degree and a bridge
    assert oracle.check_graph(adj, 0) == 32                  # bridge test skipped above the limit


def test_check_mrng_hand_geometry():
    # Alg. 2: the edge (v1, v2) fails when a common neighbour u has
    # delta(v1, v2) > max(w(v1, u), w(v2, u)), i.e. u lies in the lune of v1 and v2.
    # K5 on: v1 = (0,0), v2 = (2,0), u = (1, 0.1) [inside the lune], a = (1, 5), b = (1, -5).
    base = np.array([[0, 0], [2, 0], [1, 0.1], [1, 5], [1, -5]], np.float32)
    k5 = np.array([[j for j in range(5) if j != i] for i in range(5)], np.int32)
    assert oracle.check_mrng(base, k5, 0, 1) is False          # 2 > max(1.005, 1.005)
    # (v1, a): delta = sqrt(26) = 5.10; u is also inside that lune (1.005 and 4.90 < 5.10).
    assert oracle.check_mrng(base, k5, 0, 3) is False
    # (u, a) = (2, 3): delta 4.90; common neighbours v1 (max 5.10), v2 (5.10), b (10.0) -> passes.
    assert oracle.check_mrng(base, k5, 2, 3) is True
    # Move u out of the lune (to (1, 3)): delta(v1,v2) = 2 < 3.16 -> passes.
    base2 = base.copy(); base2[2] = [1, 3]
    assert oracle.check_mrng(base2, k5, 0, 1) is True


def test_optimize_edge_never_increases_and_and_reverts_bit_exact():
    # Alg. 4 either lowers AND (Eq. 4) -- a positive total gain -- or reverts every change.
    base = synth.uniform(300, 5, 32)
    adj = oracle.build_graph(base, 6, 12, 0.2, 6, 0.001, 0)     # i_opt = 0: no optimisation
    a0 = oracle.average_neighbor_distance(base, adj)
    changed_any = reverted_any = False
    for v1 in range(0, 300, 7):
        for v2 in adj[v1][:2]:
            ch, new = oracle.optimize_edge(base, adj, int(v1), int(v2), 5, 6, 0.001)
            assert oracle.check_graph(new) == 0
            if ch:
                changed_any = True
                assert oracle.average_neighbor_distance(base, new) < a0
            else:
                reverted_any = True
                assert np.array_equal(new, adj)                 # bit-identical, slot order included
    assert changed_any and reverted_any


def test_edge_optimisation_lowers_average_neighbor_distance():
    base = synth.uniform(400, 5, 33)
    a_plain = oracle.average_neighbor_distance(base, oracle.build_graph(base, 6, 12, 0.2, 6, 0.001, 0))
    a_opt = oracle.average_neighbor_distance(base, oracle.build_graph(base, 6, 12, 0.2, 6, 0.001, 5))
    a_ref = oracle.average_neighbor_distance(
        base, oracle.build_graph(base, 6, 12, 0.2, 6, 0.001, 5, refine_rounds=300, seed=9))
    assert a_opt < a_plain and a_ref <= a_opt


def test_and_closed_form_on_simplex():
    # K5 on the 5 standard basis vectors of R^5: every edge has length sqrt(2) -> AND = sqrt(2).
    base = np.eye(5, dtype=np.float32)
    k5 = np.array([[j for j in range(5) if j != i] for i in range(5)], np.int32)
    assert oracle.average_neighbor_distance(base, k5) == pytest.approx(np.sqrt(2.0), rel=1e-15)


def test_graph_quality_complete_graph_is_one():
    # Sec. 5.1: a complete graph has GQ = 1 (every vertex is adjacent to its d nearest).
    base = synth.uniform(5, 3, 34)
    k5 = np.array([[j for j in range(5) if j != i] for i in range(5)], np.int32)
    knn, _ = oracle.knn_bruteforce(base, base, 4, exclude=np.arange(5, dtype=np.int32))
    assert oracle.graph_quality(k5, knn) == 1.0
    # Cycle on 6 points of a regular hexagon with d=2: each vertex's 2-NN are its polygon
    # neighbours, so GQ = 1; a "skip-one" cycle shares none of them: GQ = 0.
    t = np.arange(6) * np.pi / 3
    hexa = np.stack([np.cos(t), np.sin(t)], 1).astype(np.float32)
    ring = np.array([[(i + 1) % 6, (i - 1) % 6] for i in range(6)], np.int32)
    skip = np.array([[(i + 2) % 6, (i - 2) % 6] for i in range(6)], np.int32)
    knn, _ = oracle.knn_bruteforce(hexa, hexa, 2, exclude=np.arange(6, dtype=np.int32))
    assert oracle.graph_quality(ring, knn) == 1.0
    assert oracle.graph_quality(skip, knn) == 0.0


def test_build_is_deterministic():
    base = synth.uniform(200, 4, 35)
    a = oracle.build_graph(base, 6, 12, 0.2, 6, 0.001, 5, refine_rounds=20, seed=3)
    b = oracle.build_graph(base, 6, 12, 0.2, 6, 0.001, 5, refine_rounds=20, seed=3)
    assert np.array_equal(a, b)


def test_build_rejects_bad_degree():
    base = synth.uniform(50, 4, 36)
    for d in (3, 2, 5):
        with pytest.raises(ValueError):
            oracle.build_graph(base, d, 12, 0.2, 6, 0.001, 5)
