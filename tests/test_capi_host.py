"""The C-ABI library on the host (no GPU needed): it builds, loads, exports every symbol that
include/deg.h declares, and its host-side calls (construction, graph files, validation) behave
as documented. The library's own builder is checked against the oracle's invariant checker."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2307_10479_gb300 as deg
from paper_2307_10479_gb300 import _build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return deg.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "deg.h")).read()
    return sorted(set(re.findall(r"^DEG_API [^(]*?\b(\w+)\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("deg_search", "deg_explore", "knn_exact", "deg_build", "deg_upload", "deg_free",
                     "deg_last_error", "deg_search_ex", "deg_search_host", "deg_load", "deg_save"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_symbols():
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_build_produces_a_valid_deg(L):
    base = synth.uniform(800, 12, 41)
    idx = deg.Index.build(base, 8, 16, 0.2, 8, 0.001, 5)
    adj = idx.adjacency()
    assert idx.info() == (800, 12, 8)
    assert oracle.check_graph(adj, bridge_max_n=800) == 0
    # edge optimisation lowers the average neighbour distance, as the oracle's builder does
    plain = deg.Index.build(base, 8, 16, 0.2, 8, 0.001, 0).adjacency()
    assert oracle.average_neighbor_distance(base, adj) < oracle.average_neighbor_distance(base, plain)


def test_build_rejects_bad_parameters(L):
    base = synth.uniform(50, 4, 42)
    for d in (3, 5, 2):
        with pytest.raises(deg.DegError) as e:
            deg.Index.build(base, d, 12, 0.2, 6, 0.001, 5)
        assert e.value.status == deg.DEG_EINVAL and "degree" in str(e.value)
    with pytest.raises(deg.DegError):
        deg.Index.build(base[:6], 6, 12, 0.2, 6, 0.001, 5)      # n < d + 1


def test_from_arrays_validates_the_graph(L):
    base = synth.uniform(60, 4, 43)
    adj = oracle.build_graph(base, 4, 8, 0.2, 4, 0.001, 5)
    deg.Index.from_arrays(base, adj)
    bad = adj.copy(); bad[3, 0] = 3
    with pytest.raises(deg.DegError) as e:
        deg.Index.from_arrays(base, bad)
    assert e.value.status == deg.DEG_EGRAPH
    bad = adj.copy(); bad[3, 0] = [v for v in range(60) if v not in adj[3] and v != 3][0]
    with pytest.raises(deg.DegError) as e:
        deg.Index.from_arrays(base, bad)
    assert "asymmetric" in str(e.value)
    bad = adj.copy(); bad[0, 0] = 60
    with pytest.raises(deg.DegError):
        deg.Index.from_arrays(base, bad)


def test_graph_file_round_trip(L, tmp_path):
    base = synth.uniform(300, 6, 44)
    idx = deg.Index.build(base, 6, 12, 0.2, 6, 0.001, 3)
    p1, p2 = str(tmp_path / "a.deg"), str(tmp_path / "b.deg")
    idx.save(p1, with_vectors=True)
    idx.save(p2, with_vectors=False)
    assert np.array_equal(deg.Index.load(p1).adjacency(), idx.adjacency())
    assert np.array_equal(deg.Index.load(p2, base).adjacency(), idx.adjacency())
    with pytest.raises(deg.DegError) as e:
        deg.Index.load(p2, base + 1.0)                      # vectors do not match the checksum
    assert e.value.status == deg.DEG_EIO
    with pytest.raises(deg.DegError):
        deg.Index.load(p2)                                  # no vectors in file, none given
    open(str(tmp_path / "junk.deg"), "wb").write(b"nonsense" * 20)
    with pytest.raises(deg.DegError) as e:
        deg.Index.load(str(tmp_path / "junk.deg"))
    assert e.value.status == deg.DEG_EIO


def test_search_before_upload_is_rejected(L):
    base = synth.uniform(100, 4, 45)
    idx = deg.Index.build(base, 4, 8, 0.2, 4, 0.001, 5)
    p = deg.SearchParams(10, 0.1, 0, 0, 0, 0, 0)
    st = L.deg_search_ex(idx._h, ctypes.byref(p), ctypes.c_void_p(16), None, 0, 4, ctypes.c_void_p(16),
                         ctypes.c_void_p(16), None, None, None)
    assert st == deg.DEG_ENOTREADY
    assert b"upload" in L.deg_last_error()
    assert L.deg_entry_vertex(idx._h) == -1
    assert L.deg_upload(None, 1, None) == deg.DEG_EINVAL


def test_serve_config_layout():
    # the serving configuration's layout as deg.h declares it: max_blocks follows idle_timeout_s
    assert deg.ServeConfig.max_blocks.offset == 32 and ctypes.sizeof(deg.ServeConfig) == 40


def test_knn_exact_argument_checks(L):
    assert L.knn_exact(None, 10, None, 1, 4, 1, None, None, None) == deg.DEG_EINVAL
    assert L.knn_exact(ctypes.c_void_p(16), 10, ctypes.c_void_p(16), 1, 4, 0, ctypes.c_void_p(16),
                       ctypes.c_void_p(16), None) == deg.DEG_EINVAL
    assert b"k must be" in L.deg_last_error()


@pytest.mark.parametrize("n,dim,d,seed", [(300, 8, 8, 5), (500, 6, 4, 6), (400, 12, 10, 7)])
def test_library_builder_equals_the_oracle_on_integer_rows(L, n, dim, d, seed):
    # Two independent implementations of Alg. 2-5 with the same readings: the library's in float32,
    # the oracle's in FP64. On small integer coordinates every squared distance is exact in both and
    # distinct distances stay distinct after the square root, so every decision agrees and the
    # graphs must be identical, edge for edge.
    base = np.random.default_rng(seed).integers(0, 16, (n, dim)).astype(np.float32)
    a = oracle.build_graph(base, d, 2 * d, 0.2, d, 0.001, 5)
    b = deg.Index.build(base, d, 2 * d, 0.2, d, 0.001, 5).adjacency()
    assert np.array_equal(np.sort(a, axis=1), np.sort(b, axis=1))
