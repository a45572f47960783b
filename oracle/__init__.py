"""CPU oracle for the DEG search path -- TEST INFRASTRUCTURE ONLY.

A plain FP64 C++ restatement of the paper's definitions and algorithms (Eq. 1-4, Alg. 1-5),
built with g++ into ``oracle/_build/liboracle.so`` and called through ctypes. Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it; the CUDA library
neither links nor calls it, and it shares no code with that library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["oracle_search.cpp", "oracle_build.cpp", "oracle_quant.cpp", "oracle_mlp.cpp"]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (portable flags only: it must build on x86-64 and aarch64)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    deps = srcs + [os.path.join(_HERE, h) for h in ("deg_oracle.h", "oracle_common.h")]
    if not force and os.path.exists(_LIB_PATH):
        if os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(p) for p in deps):
            return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, *srcs, "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            # DEG_ORACLE_LIB names another build of these sources (the mutation tests load copies
            # with one planted mistake this way)
            L = ctypes.CDLL(os.environ.get("DEG_ORACLE_LIB") or build())
            P, i32, i64, f64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
            L.oracle_knn_bruteforce.argtypes = [P, i64, i32, P, i64, i32, P, P, P, i32]
            L.oracle_knn_bruteforce.restype = ctypes.c_int
            L.oracle_range_search.argtypes = [P, i64, i32, P, i32, P, P, i64, i32, i32, f64, P, P, P, i32]
            L.oracle_range_search.restype = ctypes.c_int
            L.oracle_median_vertex.argtypes = [P, i64, i32]
            L.oracle_median_vertex.restype = i32
            L.deg_build_oracle.argtypes = [P, i64, i32, i32, i32, f64, i32, f64, i32, i32, u64, P, P]
            L.deg_build_oracle.restype = ctypes.c_int
            L.oracle_check_graph.argtypes = [P, i64, i32, i64]
            L.oracle_check_graph.restype = i32
            L.oracle_average_neighbor_distance.argtypes = [P, i64, i32, P, i32]
            L.oracle_average_neighbor_distance.restype = f64
            L.oracle_graph_quality.argtypes = [P, P, i64, i32]
            L.oracle_graph_quality.restype = f64
            L.oracle_check_mrng.argtypes = [P, i64, i32, P, i32, i32, i32]
            L.oracle_check_mrng.restype = i32
            L.oracle_optimize_edge.argtypes = [P, i64, i32, P, i32, i32, i32, i32, i32, f64]
            L.oracle_optimize_edge.restype = i32
            L.oracle_quantize_bf16.argtypes = [P, i64, i32, P]
            L.oracle_quantize_fp8.argtypes = [P, i64, i32, P, P]
            L.oracle_decode.argtypes = [i32, P, P, i64, i32, P]
            L.oracle_range_search_decoded.argtypes = [P, P, i64, i32, P, i32, P, P, i64, i32, i32, i32, f64, P, P, i32]
            L.oracle_range_search_decoded.restype = ctypes.c_int
            L.oracle_mlp_nparams.restype = ctypes.c_int
            L.oracle_mlp_loss_grad.argtypes = [P, P, P, i64, P]
            L.oracle_mlp_loss_grad.restype = f64
            L.oracle_mlp_predict.argtypes = [P, P, i64, P]
            _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def knn_bruteforce(base, queries, k, exclude=None, nthreads=None):
    """Eq. 1 by exhaustive FP64 search -> (ids int32 [nq,k], dists float64 [nq,k])."""
    base, queries = _f32(base), _f32(queries)
    nq = queries.shape[0]
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    ex = None if exclude is None else _i32(exclude)
    rc = lib().oracle_knn_bruteforce(_ptr(base), base.shape[0], base.shape[1], _ptr(queries), nq, k,
                                     _ptr(ex), _ptr(ids), _ptr(dists), nthreads or default_threads())
    if rc:
        raise ValueError("oracle_knn_bruteforce: invalid arguments")
    return ids, dists


def range_search(base, adj, queries, seeds, k, eps, explore=False, nthreads=None):
    """Alg. 1 per query -> (ids [nq,k], dists float64 [nq,k], trace int64 [nq,4] = H, E, max|S|, |C|)."""
    base, adj, seeds = _f32(base), _i32(adj), _i32(seeds)
    nq = seeds.shape[0]
    q = None if explore else _f32(queries)
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    trace = np.empty((nq, 4), np.int64)
    rc = lib().oracle_range_search(_ptr(base), base.shape[0], base.shape[1], _ptr(adj), adj.shape[1],
                                   _ptr(q), _ptr(seeds), nq, 1 if explore else 0, k, float(eps),
                                   _ptr(ids), _ptr(dists), _ptr(trace), nthreads or default_threads())
    if rc:
        raise ValueError("oracle_range_search: invalid arguments")
    return ids, dists, trace


def median_vertex(base) -> int:
    base = _f32(base)
    return int(lib().oracle_median_vertex(_ptr(base), base.shape[0], base.shape[1]))


def build_graph(base, degree, k_ext, eps_ext, k_opt, eps_opt, i_opt, refine_rounds=0, seed=0,
                with_weights=False):
    """DEG construction (Alg. 2-5) in FP64 -> adjacency int32 [n, degree] (+ weights)."""
    base = _f32(base)
    n = base.shape[0]
    adj = np.empty((n, degree), np.int32)
    w = np.empty((n, degree), np.float64) if with_weights else None
    rc = lib().deg_build_oracle(_ptr(base), n, base.shape[1], degree, k_ext, float(eps_ext), k_opt,
                                float(eps_opt), i_opt, refine_rounds, seed, _ptr(adj), _ptr(w))
    if rc:
        raise ValueError(f"deg_build_oracle failed ({rc})")
    return (adj, w) if with_weights else adj


def check_graph(adj, bridge_max_n=0) -> int:
    adj = _i32(adj)
    return int(lib().oracle_check_graph(_ptr(adj), adj.shape[0], adj.shape[1], bridge_max_n))


GRAPH_FLAGS = {1: "slot", 2: "self-loop", 4: "duplicate", 8: "asymmetric", 16: "disconnected",
               32: "degree", 64: "bridge"}


def average_neighbor_distance(base, adj) -> float:
    base, adj = _f32(base), _i32(adj)
    return float(lib().oracle_average_neighbor_distance(_ptr(base), base.shape[0], base.shape[1],
                                                        _ptr(adj), adj.shape[1]))


def graph_quality(adj, knn) -> float:
    adj, knn = _i32(adj), _i32(knn)
    return float(lib().oracle_graph_quality(_ptr(adj), _ptr(knn), adj.shape[0], adj.shape[1]))


def check_mrng(base, adj, v1, v2) -> bool:
    base, adj = _f32(base), _i32(adj)
    return bool(lib().oracle_check_mrng(_ptr(base), base.shape[0], base.shape[1], _ptr(adj),
                                        adj.shape[1], v1, v2))


def optimize_edge(base, adj, v1, v2, i_opt, k_opt, eps_opt):
    """Alg. 4 on a copy of adj -> (changed: bool, new adjacency)."""
    base = _f32(base)
    out = np.array(adj, dtype=np.int32, copy=True, order="C")
    rc = lib().oracle_optimize_edge(_ptr(base), base.shape[0], base.shape[1], _ptr(out), out.shape[1],
                                    v1, v2, i_opt, k_opt, float(eps_opt))
    if rc < 0:
        raise ValueError(f"oracle_optimize_edge failed ({rc})")
    return rc == 1, out


def quantize_bf16(x):
    """bfloat16 bit patterns (uint16) of float32 x, round to nearest even."""
    x = _f32(x)
    out = np.empty(x.shape, np.uint16)
    lib().oracle_quantize_bf16(_ptr(x), x.shape[0], x.shape[1], _ptr(out))
    return out


def quantize_fp8(x):
    """Per-row scaled FP8 E4M3 codes (uint8) and float32 scales of float32 x."""
    x = _f32(x)
    codes = np.empty(x.shape, np.uint8)
    scales = np.empty(x.shape[0], np.float32)
    lib().oracle_quantize_fp8(_ptr(x), x.shape[0], x.shape[1], _ptr(codes), _ptr(scales))
    return codes, scales


def decode(precision, codes, scales=None):
    """Exact FP64 values of bf16 (precision 'bf16') or scaled fp8 ('fp8') codes."""
    codes = np.ascontiguousarray(codes)
    sc = None if scales is None else np.ascontiguousarray(scales, np.float32)
    out = np.empty(codes.shape, np.float64)
    lib().oracle_decode(1 if precision == "bf16" else 2, _ptr(codes), _ptr(sc), codes.shape[0], codes.shape[1], _ptr(out))
    return out


def range_search_decoded(decoded, base, adj, queries, seeds, k, eps, keep=None, explore=False, nthreads=None):
    """Alg. 1 on decoded reduced-precision rows keeping `keep` (>= k) results, re-ranked on the
    float32 rows -> (ids, dists)."""
    decoded = np.ascontiguousarray(decoded, np.float64)
    base, adj, seeds = _f32(base), _i32(adj), _i32(seeds)
    nq = seeds.shape[0]
    q = None if explore else _f32(queries)
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    rc = lib().oracle_range_search_decoded(_ptr(decoded), _ptr(base), base.shape[0], base.shape[1], _ptr(adj),
                                           adj.shape[1], _ptr(q), _ptr(seeds), nq, 1 if explore else 0,
                                           keep or k, k, float(eps), _ptr(ids), _ptr(dists),
                                           nthreads or default_threads())
    if rc:
        raise ValueError("oracle_range_search_decoded: invalid arguments")
    return ids, dists


MLP_SHAPES = [("W1", (64, 12)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (2, 64)), ("b3", (2,))]


def mlp_nparams() -> int:
    return int(lib().oracle_mlp_nparams())


def mlp_loss_grad(w, x, labels, with_grad=True):
    """Learned-stop network in FP64: mean softmax cross-entropy and its gradient (flat 5122)."""
    w = np.ascontiguousarray(w, np.float64)
    x = np.ascontiguousarray(x, np.float32)
    labels = np.ascontiguousarray(labels, np.int32)
    g = np.empty(mlp_nparams(), np.float64) if with_grad else None
    loss = lib().oracle_mlp_loss_grad(_ptr(w), _ptr(x), _ptr(labels), x.shape[0], _ptr(g))
    return (loss, g) if with_grad else loss


def mlp_predict(w, x):
    w = np.ascontiguousarray(w, np.float64)
    x = np.ascontiguousarray(x, np.float32)
    p = np.empty(x.shape[0], np.float64)
    lib().oracle_mlp_predict(_ptr(w), _ptr(x), x.shape[0], _ptr(p))
    return p
