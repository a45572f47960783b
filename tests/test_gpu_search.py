"""GPU parity of the search path (Alg. 1) against the FP64 oracle, through the C ABI.

Workload: 10,000 x 32 iid U[0,1) base (seed 0), 1,000 queries (seed 1), a degree-8 DEG built by
the oracle; k = 10 and eps in {0, 0.1, 0.2}, plus exploration, explicit seeds, the device-memory
tier, the degenerate cases and the end-to-end host-buffer call."""
import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth
from parity import compare_lists, eps32, recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["uniform-10k-d32"]


@pytest.fixture(scope="module")
def cfg1():
    import paper_2307_10479_gb300 as deg
    base, q = W.base(), W.queries()
    adj = oracle.build_graph(base, W.degree, W.k_ext, W.eps_ext, W.k_opt, W.eps_opt, W.i_opt)
    idx = deg.Index.from_arrays(base, adj)
    idx.upload(("f32", "bf16", "fp8"))
    gt, _ = oracle.knn_bruteforce(base, q, 100)
    return dict(deg=deg, base=base, q=q, adj=adj, idx=idx, gt=gt, entry=oracle.median_vertex(base),
                qd=torch.from_numpy(q).cuda())


def test_entry_vertex_matches_oracle(cfg1):
    assert cfg1["idx"].entry_vertex == cfg1["entry"]


@pytest.mark.parametrize("eps", [0.0, 0.1, 0.2])
def test_search_parity(cfg1, eps):
    idx, q, base, adj = cfg1["idx"], cfg1["q"], cfg1["base"], cfg1["adj"]
    ids, d, st, tr = idx.search(cfg1["qd"], k=10, eps=eps, with_status=True, with_trace=True)
    torch.cuda.synchronize()
    ids, d, st, tr = ids.cpu().numpy(), d.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy()
    o_ids, o_d, o_tr = oracle.range_search(base, adj, q, np.full(len(q), cfg1["entry"], np.int32), 10, eps32(eps))
    assert (st == 0).all()
    frac, diff = compare_lists(ids, d, o_ids, o_d)
    assert abs(recall(ids, cfg1["gt"]) - recall(o_ids, cfg1["gt"])) <= 0.001
    # Exactness of the batched hop: hops H and evaluations E equal the sequential algorithm's.
    same = np.ones(len(q), bool); same[diff] = False
    assert np.mean(tr[same, 0] == o_tr[same, 0]) >= 0.999
    assert np.mean(tr[same, 1] == o_tr[same, 1]) >= 0.999


def test_explore_parity(cfg1):
    idx, base, adj = cfg1["idx"], cfg1["base"], cfg1["adj"]
    v = W.explore_ids(1000)
    ids, d, st = idx.search(seeds=torch.from_numpy(v).cuda(), explore=True, k=10, eps=0.1, with_status=True)
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    o_ids, o_d, _ = oracle.range_search(base, adj, None, v, 10, 0.1, explore=True)
    compare_lists(ids, d, o_ids, o_d)
    assert not np.any(ids == v[:, None])                      # the query vertex is never returned
    assert (st.cpu().numpy() == 0).all()


def test_explicit_seeds_parity(cfg1):
    idx, q, base, adj = cfg1["idx"], cfg1["q"], cfg1["base"], cfg1["adj"]
    seeds = np.random.default_rng(3).integers(0, len(base), len(q)).astype(np.int32)
    ids, d = idx.search(cfg1["qd"], k=10, eps=0.1, seeds=torch.from_numpy(seeds).cuda())
    o_ids, o_d, _ = oracle.range_search(base, adj, q, seeds, 10, 0.1)
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)


def test_second_kernel_is_bit_identical(cfg1):
    # A one-key device-memory pool overflows on every query that needs it; those queries are
    # rerun from scratch by the second kernel (room for all n vertices). Same results, same H, E.
    idx = cfg1["idx"]
    a_ids, a_d, a_tr = idx.search(cfg1["qd"], k=10, eps=0.2, with_trace=True)
    b_ids, b_d, b_tr = idx.search(cfg1["qd"], k=10, eps=0.2, queue_cap=1, with_trace=True)
    torch.cuda.synchronize()
    assert (a_tr[:, 3] == 0).all() and (b_tr[:, 3] == 1).sum() > 100
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)
    assert torch.equal(a_tr[:, :2], b_tr[:, :2])       # the pool peak depends on the capacity


def test_huge_eps_returns_exact_knn(cfg1):
    # eps large: S never stops early, every vertex is checked -> Eq. 1 (exact kNN).
    idx, q, base = cfg1["idx"], cfg1["q"][:64], cfg1["base"]
    ids, d, tr = idx.search(cfg1["qd"][:64], k=10, eps=1e6, with_trace=True)
    g_ids, g_d = oracle.knn_bruteforce(base, q, 10)
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), g_ids, g_d)
    assert (tr[:, 1].cpu() == len(base)).all()


def test_degenerate_and_ragged_cases(cfg1):
    idx, qd, base, adj, deg = cfg1["idx"], cfg1["qd"], cfg1["base"], cfg1["adj"], cfg1["deg"]
    # empty batch is a no-op
    e_ids, e_d = idx.search(qd[:0], k=10, eps=0.1)
    assert e_ids.shape == (0, 10)
    # ragged batch sizes and k = 1
    for nq in (1, 3, 5, 33):
        ids, d = idx.search(qd[:nq], k=1, eps=0.1)
        o_ids, o_d, _ = oracle.range_search(base, adj, cfg1["q"][:nq], np.full(nq, cfg1["entry"], np.int32), 1, 0.1)
        compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)
    # bad seed -> per-query status, other queries unaffected
    seeds = torch.tensor([0, -1, len(base), 5], dtype=torch.int32, device="cuda")
    ids, d, st = idx.search(qd[:4], k=5, eps=0.1, seeds=seeds, with_status=True)
    assert st.cpu().tolist() == [0, deg.DEG_EINVAL, deg.DEG_EINVAL, 0]
    assert (ids[1].cpu() == -1).all() and torch.isinf(d[1]).all()
    # hop cap -> DEG_EHOPLIMIT with H == cap
    ids, d, st, tr = idx.search(qd[:8], k=10, eps=0.2, max_hops=3, with_status=True, with_trace=True)
    assert (st.cpu() == deg.DEG_EHOPLIMIT).all() and (tr[:, 0].cpu() == 3).all()
    # invalid arguments are rejected before launch
    for kw in (dict(k=0), dict(k=1025), dict(k=10, eps=-0.5), dict(k=10, eps=float("nan"))):
        with pytest.raises(deg.DegError):
            idx.search(qd[:4], eps=kw.pop("eps", 0.1), **kw)


def test_k_equals_n_on_small_graph(cfg1):
    import paper_2307_10479_gb300 as deg
    base = synth.uniform(300, 8, 51)
    adj = oracle.build_graph(base, 8, 16, 0.2, 8, 0.001, 5)
    idx = deg.Index.from_arrays(base, adj)
    idx.upload()
    q = synth.uniform(4, 8, 52)
    ids, d = idx.search(torch.from_numpy(q).cuda(), k=300, eps=0.0)
    o_ids, o_d = oracle.knn_bruteforce(base, q, 300)
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)
    v = np.array([0, 299], np.int32)
    ids, d = idx.search(seeds=torch.from_numpy(v).cuda(), explore=True, k=299, eps=0.0)
    o_ids, o_d = oracle.knn_bruteforce(base, base[v], 299, exclude=v)
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)
    with pytest.raises(deg.DegError):
        idx.search(seeds=torch.from_numpy(v).cuda(), explore=True, k=300, eps=0.0)


def test_host_buffer_call_matches_device_call(cfg1):
    idx, q = cfg1["idx"], cfg1["q"]
    ids, d = idx.search(cfg1["qd"], k=10, eps=0.1)
    h_ids, h_d = idx.search_host(q, 10, 0.1)
    assert np.array_equal(h_ids, ids.cpu().numpy()) and np.array_equal(h_d, d.cpu().numpy())
    v = W.explore_ids(100)
    e_ids, e_d = idx.search(seeds=torch.from_numpy(v).cuda(), explore=True, k=10, eps=0.1)
    h_ids, h_d = idx.search_host(None, 10, 0.1, explore_ids=v)
    assert np.array_equal(h_ids, e_ids.cpu().numpy())


def test_stream_ordering_on_a_side_stream(cfg1):
    idx = cfg1["idx"]
    ref_ids, _ = idx.search(cfg1["qd"], k=10, eps=0.1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ids, _ = idx.search(cfg1["qd"], k=10, eps=0.1)
    s.synchronize()
    assert torch.equal(ids, ref_ids)


def test_pivot_entry_parity(cfg1):
    # entry="pivot": each query starts at the nearest of the pivots p * (n // P), P = n // 256
    # (at most 4096). The oracle picks that pivot by FP64 brute force and runs Alg. 1 from it.
    idx, q, base, adj = cfg1["idx"], cfg1["q"], cfg1["base"], cfg1["adj"]
    n = len(base)
    npv = max(1, min(4096, n // 256))
    piv = (np.arange(npv) * (n // npv)).astype(np.int32)
    lab, _ = oracle.knn_bruteforce(base[piv], q, 1)
    seeds = piv[lab[:, 0]]
    ids, d = idx.search(cfg1["qd"], k=10, eps=0.1, entry="pivot")
    o_ids, o_d, _ = oracle.range_search(base, adj, q, seeds, 10, 0.1)
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)
    with pytest.raises(cfg1["deg"].DegError):
        idx.search(cfg1["qd"], k=10, eps=0.1, entry="pivot", seeds=torch.zeros(len(q), dtype=torch.int32, device="cuda"))


def _circulant(n, d, seed):
    """A d-regular undirected graph without loops or duplicates: vertex perm[i] joined to
    perm[i +- 1 .. d/2] (mod n). Alg. 1 needs no DEG property, only a valid graph."""
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    offs = np.concatenate([np.arange(1, d // 2 + 1), -np.arange(1, d // 2 + 1)])
    adj = np.empty((n, d), np.int32)
    for i in range(n):
        adj[perm[i]] = perm[(i + offs) % n]
    return adj


@pytest.mark.parametrize("degree", [64, 128])
def test_degrees_above_one_warp(degree):
    # Degree 64 and 128 (the largest the kernels take) read a neighbour list in several 32-lane
    # chunks and admit a hop's candidates in several batches. With a huge eps every vertex is
    # checked, so R is the exact k-NN and H = E = n on both sides.
    import paper_2307_10479_gb300 as deg
    n = 3000
    base = synth.uniform(n, 16, 62)
    adj = _circulant(n, degree, 7)
    assert oracle.check_graph(adj) == 0
    idx = deg.Index.from_arrays(base, adj)
    idx.upload()
    q = synth.uniform(60, 16, 63)
    ids, d, st, tr = idx.search(torch.from_numpy(q).cuda(), k=10, eps=1e9, with_status=True, with_trace=True)
    o_ids, o_d, o_tr = oracle.range_search(base, adj, q, np.full(len(q), oracle.median_vertex(base), np.int32), 10, 1e9)
    assert (st.cpu().numpy() == 0).all()
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)
    assert np.array_equal(tr.cpu().numpy()[:, 1], o_tr[:, 1]) and (o_tr[:, 1] == n).all()
    assert np.array_equal(tr.cpu().numpy()[:, 0], o_tr[:, 0])


def test_largest_k():
    # k = 1024, the largest the kernels take: a 1024-long R (and re-sorted output) per query.
    import paper_2307_10479_gb300 as deg
    n = 3000
    base = synth.uniform(n, 16, 64)
    adj = _circulant(n, 32, 8)
    idx = deg.Index.from_arrays(base, adj)
    idx.upload()
    q = synth.uniform(20, 16, 65)
    ids, d, st = idx.search(torch.from_numpy(q).cuda(), k=1024, eps=1e9, with_status=True)
    gid, gd = oracle.knn_bruteforce(base, q, 1024)
    assert (st.cpu().numpy() == 0).all()
    # In a 1,024-long list, neighbours closer than float32 rounding (about 10% of these queries
    # in a float32 scan) may come in either order: such lists count as not identical, and
    # compare_lists asserts that they differ only by swaps of equal distances.
    compare_lists(ids.cpu().numpy(), d.cpu().numpy(), gid, gd, min_identical=0.5)
