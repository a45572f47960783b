"""Vertex removal (deg_remove) on the host. The paper calls the graph fully dynamic but leaves the
removal procedure open (App. A); the library's removal is checked here against the invariants the
paper fixes for a DEG (Sec. 4: even-regular, undirected, no loops or duplicates, connected; the
oracle's checker), against a plain restatement of its own rule on edge sets, and for its refusals."""
import numpy as np
import pytest

import oracle
import paper_2307_10479_gb300 as deg
from paper_2307_10479_gb300 import _build, synth


@pytest.fixture(scope="module", autouse=True)
def L():
    _build.build()
    return deg.lib()


def _dist(x, a, b):
    return np.float32(np.sqrt(np.sum((x[a].astype(np.float64) - x[b].astype(np.float64)) ** 2)))


def removal_by_rule(x, adj, v):
    """The removal rule written out on edge sets: returns (vectors, adjacency as a set of edges) after
    removing v, or None when the rule refuses."""
    n, d = adj.shape
    nbr = {u: set(int(w) for w in adj[u]) for u in range(n)}
    nb = sorted(nbr[v], key=lambda u: list(adj[v]).index(u))     # v's slot order
    for u in nb:
        nbr[u].discard(v)
    nbr[v] = set()
    pairs = sorted(((float(_dist(x, nb[i], nb[j])), nb[i], nb[j]) for i in range(d) for j in range(i + 1, d)
                    if nb[j] not in nbr[nb[i]]))
    done = set()
    for _, a, b in pairs:
        if a in done or b in done:
            continue
        nbr[a].add(b)
        nbr[b].add(a)
        done |= {a, b}
    left = [u for u in nb if u not in done]
    for a, b in zip(left[0::2], left[1::2]):
        best = None
        for m in nbr[a]:
            for xx in nbr[m]:
                if xx in (a, b) or xx in nbr[a]:
                    continue
                for yy in nbr[xx]:
                    if yy in (a, b) or yy in nbr[b]:
                        continue
                    c = np.float32(np.float32(_dist(x, a, xx) + _dist(x, b, yy)) - _dist(x, xx, yy))
                    if best is None or c < best[0]:
                        best = (c, xx, yy)
        if best is None:
            return None
        _, xx, yy = best
        nbr[xx].discard(yy)
        nbr[yy].discard(xx)
        nbr[a].add(xx)
        nbr[xx].add(a)
        nbr[b].add(yy)
        nbr[yy].add(b)
    # connected exactly when the former neighbours reach one another
    seen, stack = {nb[0]}, [nb[0]]
    while stack:
        for w in nbr[stack.pop()]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    if not set(nb) <= seen:
        return None
    last = n - 1
    x = x.copy()
    if v != last:
        for u in list(nbr[last]):
            nbr[u].discard(last)
            nbr[u].add(v)
        nbr[v] = nbr.pop(last)
        x[v] = x[last]
    else:
        nbr.pop(last)
    return x[:last], {(min(a, b), max(a, b)) for a in nbr for b in nbr[a]}


def edges(adj):
    return {(min(a, int(b)), max(a, int(b))) for a in range(adj.shape[0]) for b in adj[a]}


def test_removals_keep_the_invariants_and_follow_the_rule(tmp_path):
    x = synth.uniform(600, 10, 81)
    idx = deg.Index.build(x, 8, 16, 0.2, 8, 0.001, 5)
    rng = np.random.default_rng(7)
    for step in range(60):
        n = idx.info()[0]
        v = int(rng.integers(n))
        expect = removal_by_rule(x, idx.adjacency(), v)
        assert expect is not None
        moved = idx.remove(v)
        assert moved == (-1 if v == n - 1 else n - 1)
        adj = idx.adjacency()
        assert idx.info() == (n - 1, 10, 8)
        assert oracle.check_graph(adj, bridge_max_n=0) == 0, oracle.GRAPH_FLAGS
        x, expect_edges = expect
        assert edges(adj) == expect_edges, step
    # the vectors moved with their ids: a graph file without vectors loads only with the same rows
    path = str(tmp_path / "g.deg")
    idx.save(path, with_vectors=False)
    assert deg.Index.load(path, x).info() == (540, 10, 8)
    with pytest.raises(deg.DegError):
        deg.Index.load(path, x[::-1].copy())


def test_removal_down_to_few_vertices():
    x = synth.uniform(40, 6, 82)
    idx = deg.Index.build(x, 4, 8, 0.2, 4, 0.001, 5)
    removed = refused = 0
    while idx.info()[0] > 6:
        n = idx.info()[0]
        before = idx.adjacency()
        try:
            idx.remove(n // 2)
            removed += 1
        except deg.DegError as e:
            # a refusal leaves the index as it was
            assert e.status == deg.DEG_EINVAL
            assert (idx.adjacency() == before).all()
            refused += 1
            break
        assert oracle.check_graph(idx.adjacency(), bridge_max_n=0) == 0
    assert removed >= 30


def test_a_cut_vertex_is_refused():
    """v joins two halves (each K5 less one edge); pairing its neighbours closest first would join
    each half to itself and cut the graph, so the removal is refused and nothing changes."""
    d = 4
    pos = np.zeros((11, 3), np.float32)
    pos[1:6, 0] = [0.0, 0.01, 1, 2, 3]                          # A: a1 = 1, a2 = 2 close together
    pos[6:11, 0] = [100.0, 100.01, 101, 102, 103]               # B: b1 = 6, b2 = 7
    pos[0, 0] = 50.0
    adj = [[] for _ in range(11)]
    for lo in (1, 6):
        group = list(range(lo, lo + 5))
        for i in group:
            for j in group:
                if i < j and (i, j) != (lo, lo + 1):
                    adj[i].append(j)
                    adj[j].append(i)
    for u in (1, 2, 6, 7):
        adj[0].append(u)
        adj[u].append(0)
    adj = np.array(adj, np.int32)
    assert adj.shape == (11, d)
    idx = deg.Index.from_arrays(pos, adj)
    assert removal_by_rule(pos, adj, 0) is None
    with pytest.raises(deg.DegError) as e:
        idx.remove(0)
    assert e.value.status == deg.DEG_EINVAL and "disconnect" in str(e.value)
    assert (idx.adjacency() == adj).all()
    # every other vertex can go
    idx.remove(3)
    assert oracle.check_graph(idx.adjacency(), bridge_max_n=0) == 0


def test_remove_argument_checks():
    x = synth.uniform(30, 4, 83)
    idx = deg.Index.build(x, 4, 8, 0.2, 4, 0.001, 0)
    for v in (-1, 30, 1 << 30):
        with pytest.raises(deg.DegError) as e:
            idx.remove(v)
        assert e.value.status == deg.DEG_EINVAL
    small = deg.Index.build(x[:5], 4, 8, 0.2, 4, 0.001, 0)        # the complete graph K5
    with pytest.raises(deg.DegError):
        small.remove(0)
