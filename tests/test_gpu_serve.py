"""Serving (library extension): a persistent kernel takes mixed requests from a ring as warps
free up. Each result must equal the same request searched alone; waits are bounded (an idle
server ends with DEG_ETIMEOUT); a full ring rejects a post instead of overwriting."""
import time

import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["uniform-10k-d32"]


@pytest.fixture(scope="module")
def index():
    import paper_2307_10479_gb300 as deg
    base = W.base()
    adj = oracle.build_graph(base, W.degree, W.k_ext, W.eps_ext, W.k_opt, W.eps_opt, W.i_opt)
    idx = deg.Index.from_arrays(base, adj)
    idx.upload(("f32", "bf16"))
    return deg, idx, base


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    q = synth.uniform(n, W.dim, seed)
    ks = rng.choice([1, 10, 100], n).astype(np.int32)
    epss = rng.choice([0.05, 0.1, 0.2], n).astype(np.float32)
    explore = rng.random(n) < 0.2
    vertices = np.where(explore, rng.integers(0, W.n, n), -1).astype(np.int32)
    return q, vertices, ks, epss


@pytest.mark.parametrize("precision,entry", [("f32", "fixed"), ("bf16", "fixed")])
def test_results_in_the_mix_equal_results_alone(index, precision, entry):
    deg, idx, _ = index
    q, vertices, ks, epss = _requests(400, 11)
    srv = deg.Server(idx, capacity=1024, kmax=128, precision=precision, entry=entry, idle_timeout_s=30.0)
    assert srv.slots > 0
    lat, ids, dists, st, dev = srv.run_trace(q, vertices, ks, epss, np.zeros(len(ks)), device_times=True)  # all at once
    srv.stop()
    assert (st == 0).all() and (lat >= 0).all()
    # device time: a warp's time on the request, within the request's whole latency
    assert (dev > 0).all() and (dev <= lat + 1e-3).all()
    for i in range(len(ks)):
        k, eps = int(ks[i]), float(epss[i])
        if vertices[i] >= 0:
            a_ids, a_d = idx.search(seeds=torch.tensor([vertices[i]], dtype=torch.int32, device="cuda"), explore=True,
                                    k=k, eps=eps, precision=precision)
        else:
            a_ids, a_d = idx.search(torch.from_numpy(q[i:i + 1]).cuda(), k=k, eps=eps, precision=precision)
        assert np.array_equal(ids[i, :k], a_ids.cpu().numpy()[0]), i
        assert np.array_equal(dists[i, :k], a_d.cpu().numpy()[0]), i


def test_idle_server_ends_with_timeout(index):
    deg, idx, _ = index
    srv = deg.Server(idx, capacity=16, kmax=16, idle_timeout_s=0.05)
    time.sleep(0.3)
    with pytest.raises(deg.DegError) as e:
        srv.stop()
    assert e.value.status == deg.DEG_ETIMEOUT


def test_full_ring_rejects_a_post(index):
    deg, idx, base = index
    srv = deg.Server(idx, capacity=2, kmax=10, idle_timeout_s=10.0)
    s0 = srv.submit(vec=base[0], k=10, eps=0.1)
    s1 = srv.submit(vertex=5, k=10, eps=0.1)
    with pytest.raises(deg.DegError) as e:
        srv.submit(vec=base[1], k=10, eps=0.1)             # slot of s0 not collected yet
    assert e.value.status == deg.DEG_EOVERFLOW
    t0 = time.time()
    got = {}
    while len(got) < 2 and time.time() - t0 < 5:
        for s in (s0, s1):
            if s not in got:
                r = srv.poll(s, 10)
                if r is not None:
                    got[s] = r
    assert len(got) == 2 and got[s0][0][0] == 0             # base row 0 finds itself first
    assert 5 not in got[s1][0]                              # exploration never returns its vertex
    srv.submit(vec=base[1], k=10, eps=0.1)                  # the ring has room again
    srv.stop()


def test_max_blocks_caps_the_kernel(index):
    # a server limited to 16 blocks keeps 16 x 4 warps and still answers, leaving the rest of the GPU
    deg, idx, _ = index
    q, vertices, ks, epss = _requests(64, 12)
    srv = deg.Server(idx, capacity=256, kmax=128, idle_timeout_s=30.0, max_blocks=16)
    assert srv.slots == 16 * 4
    lat, ids, dists, st = srv.run_trace(q, vertices, ks, epss, np.zeros(len(ks)))
    srv.stop()
    assert (st == 0).all()
    a_ids, a_d = idx.search(torch.from_numpy(q[:1]).cuda(), k=int(ks[0]), eps=float(epss[0])) if vertices[0] < 0 else \
        idx.search(seeds=torch.tensor([vertices[0]], dtype=torch.int32, device="cuda"), explore=True, k=int(ks[0]),
                   eps=float(epss[0]))
    assert np.array_equal(ids[0, :int(ks[0])], a_ids.cpu().numpy()[0])
