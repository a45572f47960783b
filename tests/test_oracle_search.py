"""Pins for the CPU oracle's search side: Eq. 1 (exact kNN), Alg. 1 (RangeSearch) and the
fixed entry vertex -- each checked against something other than the oracle itself: traces of
Alg. 1 worked by hand, closed forms, brute force on tiny inputs and independent numpy routines."""
import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth


def _cycle(n):
    """Cycle graph 0-1-...-(n-1)-0 as a degree-2 adjacency (row i = [i+1, i-1])."""
    return np.array([[(i + 1) % n, (i - 1) % n] for i in range(n)], np.int32)


# ----------------------------------------------------------------------------------------------
# Eq. 1: exact kNN
# ----------------------------------------------------------------------------------------------

def test_knn_bruteforce_matches_numpy_sort():
    rng = np.random.default_rng(5)
    base = rng.random((300, 7), dtype=np.float32)
    q = rng.random((20, 7), dtype=np.float32)
    ids, d = oracle.knn_bruteforce(base, q, 9)
    dd = np.sqrt(((q[:, None, :].astype(np.float64) - base[None].astype(np.float64)) ** 2).sum(-1))
    for i in range(20):
        order = np.lexsort((np.arange(300), dd[i]))[:9]
        assert np.array_equal(ids[i], order)
        np.testing.assert_allclose(d[i], dd[i][order], rtol=1e-14)


def test_knn_bruteforce_ties_lower_id_and_exclude():
    # Points on a line at -1, +1, -1, +1 around q = 0: all four tie; lower ids first.
    base = np.array([[-1.0], [1.0], [-1.0], [1.0], [5.0]], np.float32)
    ids, d = oracle.knn_bruteforce(base, np.zeros((1, 1), np.float32), 3)
    assert ids.tolist() == [[0, 1, 2]] and d.tolist() == [[1.0, 1.0, 1.0]]
    ids, _ = oracle.knn_bruteforce(base, np.zeros((1, 1), np.float32), 3, exclude=np.array([1]))
    assert ids.tolist() == [[0, 2, 3]]
    # k > n pads with -1 / +inf
    ids, d = oracle.knn_bruteforce(base, np.zeros((1, 1), np.float32), 7)
    assert ids[0, 5:].tolist() == [-1, -1] and np.isinf(d[0, 5:]).all()


def test_knn_distance_is_euclidean_not_squared():
    # 3-4-5 triangle: delta((0,0),(3,4)) = 5 exactly.
    ids, d = oracle.knn_bruteforce(np.array([[3.0, 4.0]], np.float32), np.zeros((1, 2), np.float32), 1)
    assert d[0, 0] == 5.0


# ----------------------------------------------------------------------------------------------
# Alg. 1: traces worked by hand
# ----------------------------------------------------------------------------------------------
# Five points on a line, a cycle graph 0-1-2-3-4-0, query q = 0, seed 0, k = 1.
#   positions: v0 = 5, v1 = 3, v2 = 6, v3 = 1, v4 = 7  ->  delta to q: 5, 3, 6, 1, 7.
POS = np.array([[5.0], [3.0], [6.0], [1.0], [7.0]], np.float32)
CYC5 = _cycle(5)
Q0 = np.zeros((1, 1), np.float32)


def test_alg1_hand_trace_eps0_stops_at_barrier():
    # eps = 0:  pop v0 (5 <= inf): N = {v1, v4}; v1: 3 <= inf -> S, R = {v1, v0} -> trim v0,
    #   r = 3; v4: 7 > 3 -> rejected.  pop v1 (3 <= 3): N \ C = {v2}: 6 > 3 -> rejected.
    #   S empty -> R = {v1 @ 3}; hops 2, evaluations 4 (v0, v1, v4, v2).
    ids, d, tr = oracle.range_search(POS, CYC5, Q0, [0], 1, 0.0)
    assert ids.tolist() == [[1]] and d.tolist() == [[3.0]]
    assert tr[0, 0] == 2 and tr[0, 1] == 4 and tr[0, 3] == 4


def test_alg1_hand_trace_eps1_boundary_is_inclusive():
    # eps = 1 -> admission radius r(1+eps) = 6 once r = 3.
    #   pop v0: v1 -> R = {v1}, r = 3; v4: 7 > 6 rejected.
    #   pop v1 (3 <= 6): v2: 6 <= 6 admitted to S (boundary, Alg. 1 uses <=), 6 > 3 not in R.
    #   pop v2 (6 > 6 is false -> continue): v3: 1 <= 6 -> S, 1 <= 3 -> R = {v3, v1} -> trim v1,
    #   r = 1.  pop v3 (1 <= 2): N all checked.  S empty -> R = {v3 @ 1}; hops 4, evals 5.
    ids, d, tr = oracle.range_search(POS, CYC5, Q0, [0], 1, 1.0)
    assert ids.tolist() == [[3]] and d.tolist() == [[1.0]]
    assert tr[0, 0] == 4 and tr[0, 1] == 5


def test_alg1_hand_trace_eps_half_rejects():
    # eps = 0.5 -> radius 4.5: v2 (6) is never admitted, so the result equals eps = 0's.
    ids, _, tr = oracle.range_search(POS, CYC5, Q0, [0], 1, 0.5)
    assert ids.tolist() == [[1]] and tr[0, 0] == 2


def test_alg1_hand_trace_k2_radius_infinite_until_first_trim():
    # k = 2, eps = 0:  pop v0: v1 (3) -> R = {v1, v0}, |R| = 2 = k so r stays inf;
    #   v4 (7 <= inf) -> S and R = {v1, v0, v4} -> trim v4, r = 5.   S = {v1, v4}.
    #   pop v1 (3 <= 5): v2 (6 > 5) rejected.  pop v4 (7 > 5) -> return {v1, v0}.
    #   max |S| = 2 (v1 and v4 were both admitted while r was still infinite).
    ids, d, tr = oracle.range_search(POS, CYC5, Q0, [0], 2, 0.0)
    assert ids.tolist() == [[1, 0]] and d.tolist() == [[3.0, 5.0]]
    assert tr[0, 0] == 2 and tr[0, 1] == 4 and tr[0, 2] == 2


@pytest.mark.parametrize("adj", [[[1, 2], [0, 2], [0, 1]], [[2, 1], [2, 0], [1, 0]]])
def test_alg1_ties_keep_lower_id_in_either_visit_order(adj):
    # v1 at -3 and v2 at +3 tie at distance 3 from q = 0; with k = 1 the lower id must win
    # whichever neighbour is evaluated first (argmax over R is taken on (delta, id)).
    base = np.array([[5.0], [-3.0], [3.0]], np.float32)
    ids, d, _ = oracle.range_search(base, np.array(adj, np.int32), Q0, [0], 1, 0.0)
    assert ids.tolist() == [[1]] and d.tolist() == [[3.0]]


def test_alg1_exploration_excludes_the_seed():
    # Exploration from v3 (query = x_v3 = 1): v3 is expanded but never returned.
    #   distances to x_v3: v0 4, v1 2, v2 5, v4 6.  k = 2, eps = 0:
    #   pop v3 (0): N = [v4, v2]: v4 6 -> R = {v4}; v2 5 -> R = {v2, v4} (r still inf).
    #   pop v2 (5 <= inf): v1 2 -> R = {v1, v2, v4} -> trim v4, r = 5.
    #   pop v1 (2): v0 4 <= 5 -> R = {v1, v0, v2} -> trim v2, r = 4.  pop v0 (4 <= 4): nothing.
    #   pop v4 (6 > 4) -> return {v1 @ 2, v0 @ 4}.
    ids, d, tr = oracle.range_search(POS, CYC5, None, [3], 2, 0.0, explore=True)
    assert ids.tolist() == [[1, 0]] and d.tolist() == [[2.0, 4.0]]
    assert tr[0, 0] == 4


# ----------------------------------------------------------------------------------------------
# Alg. 1: special cases that reduce to Eq. 1
# ----------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_deg():
    base = synth.uniform(600, 8, 11)
    adj = oracle.build_graph(base, 8, 16, 0.2, 8, 0.001, 5)
    return base, adj


def test_alg1_large_eps_is_exact_knn(small_deg):
    # A huge eps never stops before S empties; on a connected graph every vertex is checked,
    # so R is the exact k-NN (Eq. 1), ties included.
    base, adj = small_deg
    q = synth.uniform(40, 8, 12)
    ids, d, tr = oracle.range_search(base, adj, q, np.zeros(40, np.int32), 10, 1e9)
    gid, gd = oracle.knn_bruteforce(base, q, 10)
    assert np.array_equal(ids, gid)
    np.testing.assert_allclose(d, gd, rtol=1e-14)
    assert (tr[:, 1] == 600).all() and (tr[:, 3] == 600).all()


def test_alg1_exploration_large_eps_is_knn_without_self(small_deg):
    base, adj = small_deg
    v = np.array([3, 77, 599], np.int32)
    ids, d, _ = oracle.range_search(base, adj, None, v, 5, 1e9, explore=True)
    gid, gd = oracle.knn_bruteforce(base, base[v], 5, exclude=v)
    assert np.array_equal(ids, gid)


def test_alg1_on_complete_graph_is_exact():
    # K_{d+1}: every vertex neighbours the seed, so one hop checks all of them.
    base = synth.uniform(9, 5, 13)
    adj = np.array([[j for j in range(9) if j != i] for i in range(9)], np.int32)
    q = synth.uniform(6, 5, 14)
    for eps in (0.0, 0.3):
        ids, _, tr = oracle.range_search(base, adj, q, np.full(6, 4, np.int32), 3, eps)
        gid, _ = oracle.knn_bruteforce(base, q, 3)
        assert np.array_equal(ids, gid)
        assert (tr[:, 1] == 9).all()


def test_alg1_k_at_least_n_returns_everything_sorted(small_deg):
    base, adj = small_deg
    q = synth.uniform(3, 8, 15)
    ids, d, _ = oracle.range_search(base, adj, q, np.zeros(3, np.int32), 700, 0.0)
    gid, gd = oracle.knn_bruteforce(base, q, 700)
    assert np.array_equal(ids, gid)          # r never becomes finite: all 600 found, 100 pads
    assert (ids[:, 600:] == -1).all()


def test_alg1_result_invariants(small_deg):
    # Every returned distance is the true distance of the returned id, results are sorted by
    # (distance, id), unique, and at most 1 + hops * d vertices are evaluated.
    base, adj = small_deg
    q = synth.uniform(50, 8, 16)
    for eps in (0.0, 0.05, 0.2):
        ids, d, tr = oracle.range_search(base, adj, q, np.zeros(50, np.int32), 10, eps)
        true = np.sqrt(((base[ids].astype(np.float64) - q[:, None, :].astype(np.float64)) ** 2).sum(-1))
        np.testing.assert_allclose(d, true, rtol=1e-14)
        for i in range(50):
            assert len(set(ids[i].tolist())) == 10
            key = list(zip(d[i], ids[i]))
            assert key == sorted(key)
        assert (tr[:, 1] <= 1 + tr[:, 0] * adj.shape[1]).all()
        assert (tr[:, 1] == tr[:, 3]).all()


def test_alg1_recall_grows_with_eps(small_deg):
    base, adj = small_deg
    q = synth.uniform(100, 8, 17)
    gid, _ = oracle.knn_bruteforce(base, q, 10)
    rec, evals = [], []
    for eps in (0.0, 0.1, 0.3):
        ids, _, tr = oracle.range_search(base, adj, q, np.zeros(100, np.int32), 10, eps)
        rec.append(np.mean([len(set(a) & set(b)) for a, b in zip(ids.tolist(), gid.tolist())]) / 10)
        evals.append(tr[:, 1].mean())
    assert evals[0] < evals[1] < evals[2]
    assert rec[2] >= rec[0]


# ----------------------------------------------------------------------------------------------
# Fixed entry vertex (Sec. 5.4 "median vertex"; lower-median reading)
# ----------------------------------------------------------------------------------------------

def test_median_vertex_hand_examples():
    # Coordinates (x, y): lower medians x: sorted [0, 1, 2, 9] -> rank 1 -> 1; y: [0, 0, 3, 4] -> 0.
    # Median vector (1, 0): nearest row is (1, 0) itself = id 2.
    base = np.array([[0, 3], [9, 0], [1, 0], [2, 4]], np.float32)
    assert oracle.median_vertex(base) == 2
    # Odd n, 1-D: median of {5, 1, 3} = 3 -> id 2.
    assert oracle.median_vertex(np.array([[5.0], [1.0], [3.0]], np.float32)) == 2
    # n = 5: sorted [-1, -0.5, 0.5, 1, 7] -> rank 2 -> 0.5 = id 2.
    assert oracle.median_vertex(np.array([[-1.0], [1.0], [0.5], [-0.5], [7.0]], np.float32)) == 2
    # Tie: x and y lower medians are both 1 -> (1, 1), at distance sqrt(2) from (0, 2) = id 0
    # and (2, 0) = id 1; the lower id wins.
    base = np.array([[0, 2], [2, 0], [1, -5], [-5, 1], [3, 3]], np.float32)
    assert oracle.median_vertex(base) == 0
    assert oracle.median_vertex(base[[1, 0, 2, 3, 4]]) == 0


def test_median_vertex_matches_numpy_definition():
    base = synth.uniform(1001, 6, 18)
    med = np.sort(base, axis=0)[(1001 - 1) // 2].astype(np.float64)
    d = np.sqrt(((base.astype(np.float64) - med) ** 2).sum(1))
    assert oracle.median_vertex(base) == int(np.argmin(d))


# ----------------------------------------------------------------------------------------------
# Alg. 1 on reduced-precision rows with a float32 re-rank (the library's bf16/FP8 forms)
# ----------------------------------------------------------------------------------------------

def test_decoded_search_on_exact_rows_is_the_float32_search(small_deg):
    # Rows whose values bf16 holds exactly decode to themselves, so with keep = k the
    # reduced-precision search is Alg. 1 on the float32 rows: same ids, same distances.
    base, adj = small_deg
    exact = np.round(base * 64) / 64                          # 6 fractional bits: exact in bf16
    q = synth.uniform(30, 8, 15)
    dec = oracle.decode("bf16", oracle.quantize_bf16(exact))
    assert np.array_equal(dec, exact.astype(np.float64))
    for eps in (0.0, 0.2):
        seeds = np.zeros(30, np.int32)
        ids, d = oracle.range_search_decoded(dec, exact, adj, q, seeds, 10, eps, keep=10)
        o_ids, o_d, _ = oracle.range_search(exact, adj, q, seeds, 10, eps)
        assert np.array_equal(ids, o_ids)
        np.testing.assert_allclose(d, o_d, rtol=1e-14)


def test_decoded_search_keeping_everything_reranks_to_exact_knn(small_deg):
    # With a huge eps every vertex is checked; keeping all n results and re-ranking them on the
    # float32 rows gives the exact k-NN (Eq. 1) of the float32 rows, although FP8 distances alone
    # would order them differently.
    base, adj = small_deg
    q = synth.uniform(30, 8, 16)
    dec = oracle.decode("fp8", *oracle.quantize_fp8(base))
    ids, d = oracle.range_search_decoded(dec, base, adj, q, np.zeros(30, np.int32), 10, 1e9, keep=len(base))
    gid, gd = oracle.knn_bruteforce(base, q, 10)
    assert np.array_equal(ids, gid)
    np.testing.assert_allclose(d, gd, rtol=1e-14)
    # the FP8 order alone is not the exact one on this data (else the test above proves nothing)
    fid, _ = oracle.knn_bruteforce(dec.astype(np.float32), q, 10)
    assert not np.array_equal(fid, gid)


def test_decoded_search_returns_the_float32_distances_of_the_kept_candidates(small_deg):
    # keep > k: the k returned are the k closest by float32 distance among the keep candidates
    # the decoded search found (with a huge eps these are the decoded rows' keep nearest).
    base, adj = small_deg
    q = synth.uniform(20, 8, 17)
    dec = oracle.decode("fp8", *oracle.quantize_fp8(base))
    keep = 32
    ids, d = oracle.range_search_decoded(dec, base, adj, q, np.zeros(20, np.int32), 10, 1e9, keep=keep)
    cand = np.argsort(((dec[None, :, :] - q[:, None, :].astype(np.float64)) ** 2).sum(-1), axis=1, kind="stable")[:, :keep]
    for i in range(len(q)):
        true = np.sqrt(((base[cand[i]].astype(np.float64) - q[i].astype(np.float64)) ** 2).sum(-1))
        order = np.lexsort((cand[i], true))[:10]
        assert np.array_equal(ids[i], cand[i][order])
        np.testing.assert_allclose(d[i], true[order], rtol=1e-14)
