"""Learned entry points (deg_train_entry): k-means on the device, each centroid replaced by its
nearest vertex, used as a second routing set (entry="learned").

- The search from the learned entry is Alg. 1 from the seed the routing picks: the library's
  results equal the oracle's from the nearest learned pivot (FP64 brute force over those rows).
- The training does what Lloyd's algorithm is for: the rows' mean squared distance to their
  nearest pivot falls below that of the same number of pivots sampled at upload, and the final
  clusters cover every row."""
import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth
from parity import compare_lists, eps32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 20_000, 400)


@pytest.fixture(scope="module")
def g():
    import paper_2307_10479_gb300 as deg
    base, q = W.base(), W.queries()
    idx = deg.Index.build_device(base, W.degree, W.k_ext, W.eps_ext, k_opt=W.k_opt, i_opt=5)
    adj = idx.adjacency()
    idx.upload(("f32", "fp8"))
    sampled = idx.pivots()
    sizes = idx.train_entry(len(sampled), 10)
    return dict(deg=deg, base=base, q=q, idx=idx, adj=adj, sampled=sampled, learned=idx.pivots(learned=True),
                sizes=sizes)


def test_learned_pivots_are_vertices_and_cover_the_rows(g):
    piv, base = g["learned"], g["base"]
    assert len(piv) == len(g["sampled"]) and ((piv >= 0) & (piv < len(base))).all()
    assert g["sizes"].sum() == len(base) and (g["sizes"] >= 0).all()


def test_learned_pivots_quantise_the_rows_better_than_sampled_ones(g):
    base = g["base"]
    _, d_s = oracle.knn_bruteforce(base[g["sampled"]], base, 1)
    _, d_l = oracle.knn_bruteforce(base[g["learned"]], base, 1)
    print(f"mean squared distance to the nearest pivot: sampled {np.mean(d_s ** 2):.1f}, learned {np.mean(d_l ** 2):.1f}")
    assert np.mean(d_l ** 2) < np.mean(d_s ** 2)


def test_learned_entry_search_parity(g):
    idx, base, adj, q = g["idx"], g["base"], g["adj"], g["q"]
    piv = g["learned"]
    lab, _ = oracle.knn_bruteforce(base[piv], q, 1)
    seeds = piv[lab[:, 0]]
    ids, d, tr = idx.search(torch.from_numpy(q).cuda(), k=10, eps=0.05, entry="learned", with_trace=True)
    o_ids, o_d, o_tr = oracle.range_search(base, adj, q, seeds, 10, eps32(0.05))
    frac, diff = compare_lists(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_d)
    same = np.ones(len(q), bool)
    same[diff] = False
    assert np.array_equal(tr.cpu().numpy()[same, :2], o_tr[same, :2])
    # the fp8 form routes the same way
    f_ids, _ = idx.search(torch.from_numpy(q).cuda(), k=10, eps=0.05, entry="learned", precision="fp8", rerank=32)
    assert (f_ids.cpu().numpy() >= 0).all()


def test_learned_entry_needs_training():
    import paper_2307_10479_gb300 as deg
    base = synth.uniform(2000, 8, 4)
    adj = oracle.build_graph(base, 8, 16, 0.2, 8, 0.001, 0)
    idx = deg.Index.from_arrays(base, adj)
    idx.upload()
    with pytest.raises(deg.DegError):
        idx.search(torch.from_numpy(base[:4]).cuda(), k=5, eps=0.1, entry="learned")
    with pytest.raises(deg.DegError):
        idx.train_entry(0, 5)
    assert len(idx.pivots(learned=True)) == 0
