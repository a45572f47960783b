"""Continuous refinement while serving (Sec. 5.3: Alg. 5 improves the graph while it is in use).
deg_refine_live runs Alg. 5 on the device while the persistent serving kernel answers requests on
the same index; each batch's changes are published into the serving adjacency in place.

- The serving kernel and the refinement overlap in time (requests complete during the call).
- Every served result is well formed on the changing graph: vertices in range, distinct, with
  their exact distances, in ascending order; recall stays within reach of either graph's.
- Afterwards the refined graph keeps the invariants (oracle checker), has a lower average
  neighbour distance, and the device copy equals it: the batched search on the live copy, never
  uploaded again, equals the oracle's search on the host graph."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2307_10479_gb300 import synth
from parity import compare_lists, eps32, recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_refinement_while_serving():
    import paper_2307_10479_gb300 as deg
    w = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 20_000, 400)
    base, q = w.base(), w.queries()
    # construction only (i_opt = 0): Alg. 5 has edges to improve
    idx = deg.Index.build_device(base, 30, 60, 0.2, i_opt=0)
    idx.upload()
    adj0 = idx.adjacency()
    gt, _ = oracle.knn_bruteforce(base, q, 10)
    qd = torch.from_numpy(q).cuda()
    r_before = recall(idx.search(qd, k=10, eps=0.1)[0].cpu().numpy(), gt)

    # a first call grows the refinement's memory pool and loads its kernels before serving starts
    assert idx.refine_live(64, 30, 0.001, 5, seed=1) >= 0
    adj0 = idx.adjacency()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    srv = deg.Server(idx, capacity=4096, kmax=10, idle_timeout_s=10.0, max_blocks=sms)
    assert 0 < srv.slots <= 8 * sms                   # one block per SM at most: the rest is free
    nreq = 40_000
    reps = np.arange(nreq) % len(q)
    arrival = np.linspace(0.0, 4.0, nreq)
    out = {}

    def serve():
        out["t0"] = time.perf_counter()
        out["trace"] = srv.run_trace(q[reps], np.full(nreq, -1, np.int32), np.full(nreq, 10, np.int32),
                                     np.full(nreq, 0.1, np.float32), arrival, timeout_s=120.0)

    th = threading.Thread(target=serve)
    th.start()
    time.sleep(0.2)
    t_start = time.perf_counter()
    improved = idx.refine_live(40_000, 30, 0.001, 5, seed=3)
    t_end = time.perf_counter()
    th.join()
    srv.stop()
    lat, ids, dists, st = out["trace"]
    assert (st == 0).all()

    # overlap: requests finished while the refinement ran
    done_at = out["t0"] + arrival + lat
    during = int(((done_at > t_start) & (done_at < t_end)).sum())
    assert during > 100, (during, t_end - t_start)

    # every result is well formed: distinct vertices with their exact distances, ascending
    assert ((ids >= 0) & (ids < len(base))).all()
    assert all(len(set(r)) == 10 for r in ids)
    pick = np.arange(0, nreq, 17)
    exact = np.sqrt(((base[ids[pick]].astype(np.float64) - q[reps[pick]][:, None, :]) ** 2).sum(-1))
    np.testing.assert_allclose(dists[pick], exact, rtol=1e-5, atol=1e-3)
    assert (np.diff(dists, axis=1) >= 0).all()

    # the refined graph: invariants, lower average neighbour distance, device copy == host graph
    adj1 = idx.adjacency()
    assert improved > 0 and not np.array_equal(adj0, adj1)
    assert oracle.check_graph(adj1) == 0
    assert oracle.average_neighbor_distance(base, adj1) < oracle.average_neighbor_distance(base, adj0)
    ids1, d1 = idx.search(qd, k=10, eps=0.1)
    entry = np.full(len(q), oracle.median_vertex(base), np.int32)
    o_ids, o_d, _ = oracle.range_search(base, adj1, q, entry, 10, eps32(0.1))
    compare_lists(ids1.cpu().numpy(), d1.cpu().numpy(), o_ids, o_d)

    # served recall within reach of the graphs before and after
    r_after = recall(ids1.cpu().numpy(), gt)
    r_served = recall(ids, gt[reps])
    assert r_served >= min(r_before, r_after) - 0.02, (r_served, r_before, r_after)
