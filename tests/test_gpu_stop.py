"""Learned early stop (library extension): the training kernels against the FP64 oracle, the
stop's semantics on fixed networks, the training traces, and what a trained network gains over
the plain eps rule on the 10k x 32 workload."""
import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth
from parity import recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["uniform-10k-d32"]


def _rand(seed, count):
    rng = np.random.default_rng(seed)
    w = (rng.standard_normal(5122) * 0.3).astype(np.float32)
    x = rng.standard_normal((count, 12)).astype(np.float32)
    y = rng.integers(0, 2, count).astype(np.int32)
    return w, x, y


@pytest.mark.parametrize("count", [1, 127, 1000])
def test_gradient_matches_oracle(count):
    import paper_2307_10479_gb300 as deg
    w, x, y = _rand(count, count)
    loss, grad = deg.mlp_loss_grad(torch.from_numpy(w).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    o_loss, o_grad = oracle.mlp_loss_grad(w.astype(np.float64), x, y)
    assert abs(float(loss.item()) - o_loss) <= 1e-4 * max(1.0, abs(o_loss))
    g = grad.cpu().numpy().astype(np.float64)
    # float32 sums of a few hundred terms: relative error of the gradient vector below 1e-3
    assert np.linalg.norm(g - o_grad) <= 1e-3 * np.linalg.norm(o_grad)


def test_predict_matches_oracle():
    import paper_2307_10479_gb300 as deg
    w, x, _ = _rand(5, 2000)
    p = deg.mlp_predict(torch.from_numpy(w).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_allclose(p, oracle.mlp_predict(w.astype(np.float64), x), atol=1e-5)


def test_adam_training_reduces_the_loss():
    import paper_2307_10479_gb300 as deg
    rng = np.random.default_rng(7)
    x = rng.standard_normal((20000, 12)).astype(np.float32)
    y = (x[:, 0] + 0.5 * x[:, 3] > 0).astype(np.int32)          # a separable rule
    w, hist = deg.train_stop_model(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), epochs=5, batch=1024)
    assert hist[-1] < 0.3 * hist[0] and hist[-1] < 0.1


@pytest.fixture(scope="module")
def small():
    import paper_2307_10479_gb300 as deg
    base, q = W.base(), W.queries()
    adj = oracle.build_graph(base, W.degree, W.k_ext, W.eps_ext, W.k_opt, W.eps_opt, W.i_opt)
    idx = deg.Index.from_arrays(base, adj)
    idx.upload()
    gt, _ = oracle.knn_bruteforce(base, q, 10)
    return dict(deg=deg, idx=idx, q=torch.from_numpy(q).cuda(), gt=gt, base=base)


def _fixed_net(stop):
    w = np.zeros(5122, np.float32)
    w[-2:] = [-10.0, 10.0] if stop else [10.0, -10.0]
    return torch.from_numpy(w).cuda()


def test_never_stop_network_is_the_plain_method(small):
    idx, q = small["idx"], small["q"]
    a_ids, a_d, a_tr = idx.search(q, k=10, eps=0.1, with_trace=True)
    idx.set_stop_model(_fixed_net(False), 0.5)
    b_ids, b_d, b_tr = idx.search(q, k=10, eps=0.1, learned_stop=True, with_trace=True)
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d) and torch.equal(a_tr[:, :2], b_tr[:, :2])


def test_always_stop_network_stops_at_the_first_check(small):
    idx, q = small["idx"], small["q"]
    idx.set_stop_model(_fixed_net(True), 0.5)
    ids, d, tr = idx.search(q, k=10, eps=0.1, learned_stop=True, with_trace=True)
    _, _, tp = idx.search(q, k=10, eps=0.1, with_trace=True)
    h, hp = tr[:, 0].cpu(), tp[:, 0].cpu()
    # the network is consulted every fourth hop once R has not changed for two hops: each query
    # ends at its first such check, or earlier where the eps rule ends it
    assert ((h % 4 == 0) | (h == hp)).all() and (h <= hp).all() and (h < hp).any()
    # the eps rule still bounds it: with eps = 0 no query runs longer than without the network
    _, _, t0 = idx.search(q, k=10, eps=0.0, with_trace=True)
    _, _, t1 = idx.search(q, k=10, eps=0.0, learned_stop=True, with_trace=True)
    assert (t1[:, 0] <= t0[:, 0]).all()


def test_recorded_traces_are_consistent(small):
    idx, q = small["idx"], small["q"]
    _, _, tr = idx.search(q, k=10, eps=0.1, with_trace=True)
    feats, labels, counts = idx.stop_record(q, k=10, eps=0.1, cap=64)
    h = tr[:, 0].cpu().numpy()
    c = counts.cpu().numpy()
    assert np.array_equal(c, np.minimum(h, 64))
    lab = labels.cpu().numpy()
    f = feats.cpu().numpy()
    for i in range(0, len(c), 37):
        row = lab[i, :c[i]]
        assert np.all(np.diff(row) >= 0)                           # 0 ... 0 1 ... 1
        if h[i] <= 64:
            assert row[-1] == 1                                    # R is final after the last hop
        np.testing.assert_allclose(f[i, :c[i], 0], np.arange(1, c[i] + 1) / 64.0, rtol=1e-6)   # hops


def test_trained_network_saves_work_at_small_recall_cost(small):
    # Train on traces of 20,000 held-out queries (seed 3) searched with eps = 0.3, then search the
    # 1,000 test queries with the same eps: the network (stop when P(stop) > 0.6) must cut the
    # evaluations by at least half, keep recall@10 >= 0.94, and need fewer evaluations than the
    # plain eps rule does for the same recall (the smallest eps on a 0.01 grid reaching it).
    deg, idx, q, gt = small["deg"], small["idx"], small["q"], small["gt"]
    eps = 0.3
    train_q = torch.from_numpy(W.training_queries(20000)).cuda()
    feats, labels, counts = idx.stop_record(train_q, k=10, eps=eps, cap=1024)
    mask = torch.arange(1024, device="cuda")[None, :] < counts[:, None]
    w, hist = deg.train_stop_model(feats[mask].contiguous(), labels[mask].contiguous(), epochs=4, batch=4096)
    idx.set_stop_model(w, 0.6)
    p_ids, _, p_tr = idx.search(q, k=10, eps=eps, with_trace=True)
    l_ids, _, l_tr = idx.search(q, k=10, eps=eps, learned_stop=True, with_trace=True)
    r_plain, r_learn = recall(p_ids.cpu().numpy(), gt), recall(l_ids.cpu().numpy(), gt)
    e_plain, e_learn = p_tr[:, 1].float().mean().item(), l_tr[:, 1].float().mean().item()
    matched = None
    for e2 in np.arange(0.15, 0.31, 0.01):
        ids2, _, tr2 = idx.search(q, k=10, eps=float(e2), with_trace=True)
        if recall(ids2.cpu().numpy(), gt) >= r_learn:
            matched = (float(e2), tr2[:, 1].float().mean().item())
            break
    print(f"eps {eps}: plain recall {r_plain:.4f} E {e_plain:.0f}; learned recall {r_learn:.4f} E {e_learn:.0f}; "
          f"plain at matched recall (eps, E) = {matched}; loss {[round(h, 4) for h in hist]}")
    assert e_learn <= 0.5 * e_plain
    assert r_learn >= 0.94
    assert matched is not None and e_learn < matched[1]
