"""GB300-native batched search over a Dynamic Exploration Graph (DEG, arXiv 2307.10479).

The compute path lives in ``libdeg.so`` (hand-written CUDA for sm_103a behind the C ABI declared
in ``include/deg.h``). This package is a thin ctypes binding with the same names: it marshals
torch tensors and numpy arrays into pointers, sizes and the current CUDA stream, and raises on
a non-zero status. Importing the package does not load the library; the first call does, and
raises ``RuntimeError`` if the library has not been built (``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

DEG_OK, DEG_EINVAL, DEG_ENOMEM, DEG_ECUDA, DEG_EIO = 0, -1, -2, -3, -4
DEG_EOVERFLOW, DEG_EHOPLIMIT, DEG_ETIMEOUT, DEG_EGRAPH, DEG_ENOTREADY = -5, -6, -7, -8, -9
DEG_F32, DEG_BF16, DEG_FP8 = 0, 1, 2
PRECISIONS = {"f32": DEG_F32, "bf16": DEG_BF16, "fp8": DEG_FP8}

_lock = threading.Lock()
_lib = None


ENTRY_MODES = {"fixed": 0, "pivot": 1, "learned": 2}


class DegError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[deg status {status}] {msg}")
        self.status = status


class BuildParams(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32), ("k_ext", ctypes.c_int32), ("eps_ext", ctypes.c_float),
                ("k_opt", ctypes.c_int32), ("eps_opt", ctypes.c_float), ("i_opt", ctypes.c_int32),
                ("refine_rounds", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class SearchParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("eps", ctypes.c_float), ("precision", ctypes.c_int32),
                ("rerank", ctypes.c_int32), ("max_hops", ctypes.c_int32), ("visited_cap", ctypes.c_int32),
                ("queue_cap", ctypes.c_int32), ("entry_mode", ctypes.c_int32), ("learned_stop", ctypes.c_int32)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int32), ("kmax", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("rerank", ctypes.c_int32), ("entry_mode", ctypes.c_int32), ("learned_stop", ctypes.c_int32),
                ("idle_timeout_s", ctypes.c_double), ("max_blocks", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libdeg.so (built in-tree). Raises RuntimeError if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libdeg.so is not built ({_build.LIB}); run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        P, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        S = ctypes.c_int
        sig = {
            "deg_build": (S, [P, i64, i32, ctypes.POINTER(BuildParams), P, ctypes.POINTER(P)]),
            "deg_build_device": (S, [P, i64, i32, ctypes.POINTER(BuildParams), i32, P, ctypes.POINTER(P), P]),
            "deg_refine_device": (S, [P, ctypes.POINTER(BuildParams), ctypes.POINTER(i64), P]),
            "deg_insert_device": (S, [P, P, i64, ctypes.POINTER(BuildParams), i32, P]),
            "deg_remove": (S, [P, i32, ctypes.POINTER(i32)]),
            "deg_index_from_arrays": (S, [P, P, i64, i32, i32, ctypes.POINTER(P)]),
            "deg_save": (S, [P, ctypes.c_char_p, i32]),
            "deg_load": (S, [ctypes.c_char_p, P, ctypes.POINTER(P)]),
            "deg_index_info": (S, [P, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "deg_get_adjacency": (S, [P, P]),
            "deg_upload": (S, [P, i32, P]),
            "deg_entry_vertex": (i32, [P]),
            "deg_train_entry": (S, [P, i32, i32, P, P]),
            "deg_get_pivots": (i32, [P, i32, P, i32]),
            "deg_export_codes": (S, [P, i32, P, P]),
            "deg_free": (None, [P]),
            "deg_search": (S, [P, P, i64, i32, f32, P, P, P, P, P]),
            "deg_explore": (S, [P, P, i64, i32, f32, P, P, P, P]),
            "deg_search_ex": (S, [P, ctypes.POINTER(SearchParams), P, P, i32, i64, P, P, P, P, P]),
            "deg_set_kernel_timer": (S, [P, P, P]),
            "deg_search_host": (S, [P, ctypes.POINTER(SearchParams), P, P, i32, i64, P, P, P]),
            "knn_exact": (S, [P, i64, P, i64, i32, i32, P, P, P]),
            "knn_exact_noalloc": (S, [P, i64, P, i64, i32, i32, P, P, P]),
            "deg_nearest_rows": (S, [P, i64, i32, P, i64, i32, P, P, P]),
            "deg_stop_record": (S, [P, ctypes.POINTER(SearchParams), P, i64, i32, P, P, P, P]),
            "deg_mlp_loss_grad": (S, [P, P, P, i64, P, P, P, P]),
            "deg_mlp_scratch_floats": (i64, [i64]),
            "deg_mlp_adam": (S, [P, P, P, P, i32, f32, P]),
            "deg_mlp_predict": (S, [P, P, i64, P, P]),
            "deg_set_stop_model": (S, [P, P, f32, P]),
            "deg_serve_start": (S, [P, ctypes.POINTER(ServeConfig), ctypes.POINTER(P)]),
            "deg_serve_submit": (S, [P, P, i32, i32, f32, ctypes.POINTER(i64)]),
            "deg_serve_poll": (i32, [P, i64, P, P, P]),
            "deg_serve_run_trace": (S, [P, P, P, P, P, P, i64, P, P, P, P, P, ctypes.c_double]),
            "deg_serve_slots": (i32, [P]),
            "deg_serve_stop": (S, [P]),
            "deg_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return _lib


def _check(status: int):
    if status != DEG_OK:
        raise DegError(status, lib().deg_last_error().decode(errors="replace"))


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _require_cuda(t, dtype, name):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return t


class Index:
    """A DEG over float32 vectors: host copy, optional device copy (after ``upload``)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.deg_free(h)
            self._h = None

    # ---- construction ---------------------------------------------------------------------
    @classmethod
    def build(cls, base: np.ndarray, degree: int, k_ext: int, eps_ext: float, k_opt: int, eps_opt: float,
              i_opt: int, refine_rounds: int = 0, seed: int = 0) -> "Index":
        base = np.ascontiguousarray(base, np.float32)
        p = BuildParams(degree, k_ext, eps_ext, k_opt, eps_opt, i_opt, refine_rounds, seed)
        h = ctypes.c_void_p()
        _check(lib().deg_build(base.ctypes.data, base.shape[0], base.shape[1], ctypes.byref(p), None, ctypes.byref(h)))
        return cls(h)

    @classmethod
    def build_device(cls, base: np.ndarray, degree: int, k_ext: int, eps_ext: float, k_opt: int = 0,
                     eps_opt: float = 0.001, i_opt: int = 0, refine_rounds: int = 0, seed: int = 0,
                     batch_div: int = 256, stream=None) -> "Index":
        """ExtendGraph in batches on the current GPU (deg_build_device), with optimizeEdge when i_opt > 0."""
        base = np.ascontiguousarray(base, np.float32)
        p = BuildParams(degree, k_ext, eps_ext, k_opt or degree, eps_opt, i_opt, refine_rounds, seed)
        h = ctypes.c_void_p()
        _check(lib().deg_build_device(base.ctypes.data, base.shape[0], base.shape[1], ctypes.byref(p), batch_div, None,
                                      ctypes.byref(h), _stream_ptr(stream)))
        return cls(h)

    def insert_device(self, vectors: np.ndarray, k_ext: int, eps_ext: float, k_opt: int = 0, eps_opt: float = 0.001,
                      i_opt: int = 0, batch_div: int = 256, stream=None):
        """Insert new vectors as vertices n .. n+m-1 (deg_insert_device); upload again afterwards."""
        vectors = np.ascontiguousarray(vectors, np.float32)
        _, _, degree = self.info()
        p = BuildParams(degree, k_ext, eps_ext, k_opt or degree, eps_opt, i_opt, 0, 0)
        _check(lib().deg_insert_device(self._h, vectors.ctypes.data, vectors.shape[0], ctypes.byref(p), batch_div,
                                       _stream_ptr(stream)))

    def remove(self, v: int) -> int:
        """Remove vertex v (deg_remove); the last vertex takes id v. Returns its old id, or -1 if v was last."""
        moved = ctypes.c_int32(-1)
        _check(lib().deg_remove(self._h, int(v), ctypes.byref(moved)))
        return moved.value

    def refine_device(self, rounds: int, k_opt: int, eps_opt: float, i_opt: int, seed: int = 0, stream=None) -> int:
        """Alg. 5 for `rounds` random vertices on the GPU (deg_refine_device); returns the improved count."""
        _, _, degree = self.info()
        p = BuildParams(degree, degree, 0.2, k_opt, eps_opt, i_opt, rounds, seed)
        improved = ctypes.c_int64()
        _check(lib().deg_refine_device(self._h, ctypes.byref(p), ctypes.byref(improved), _stream_ptr(stream)))
        return improved.value

    @classmethod
    def from_arrays(cls, base: np.ndarray, adj: np.ndarray) -> "Index":
        base = np.ascontiguousarray(base, np.float32)
        adj = np.ascontiguousarray(adj, np.int32)
        h = ctypes.c_void_p()
        _check(lib().deg_index_from_arrays(base.ctypes.data, adj.ctypes.data, base.shape[0], base.shape[1],
                                           adj.shape[1], ctypes.byref(h)))
        return cls(h)

    @classmethod
    def load(cls, path: str, base: np.ndarray | None = None) -> "Index":
        b = None if base is None else np.ascontiguousarray(base, np.float32)
        h = ctypes.c_void_p()
        _check(lib().deg_load(path.encode(), None if b is None else b.ctypes.data, ctypes.byref(h)))
        return cls(h)

    def save(self, path: str, with_vectors: bool = False):
        _check(lib().deg_save(self._h, path.encode(), 1 if with_vectors else 0))

    def info(self):
        n, d, g = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().deg_index_info(self._h, ctypes.byref(n), ctypes.byref(d), ctypes.byref(g)))
        return n.value, d.value, g.value

    def adjacency(self) -> np.ndarray:
        n, _, g = self.info()
        out = np.empty((n, g), np.int32)
        _check(lib().deg_get_adjacency(self._h, out.ctypes.data))
        return out

    # ---- device ---------------------------------------------------------------------------
    def upload(self, precisions=("f32",), stream=None):
        mask = 0
        for p in precisions:
            mask |= 1 << PRECISIONS[p]
        _check(lib().deg_upload(self._h, mask, _stream_ptr(stream)))

    def export_codes(self, precision: str):
        """The device's reduced-precision rows: bf16 -> uint16 [n, dim]; fp8 -> (uint8 [n, dim], scales)."""
        n, dim, _ = self.info()
        if precision == "bf16":
            codes = np.empty((n, dim), np.uint16)
            _check(lib().deg_export_codes(self._h, DEG_BF16, codes.ctypes.data, None))
            return codes
        codes = np.empty((n, dim), np.uint8)
        scales = np.empty(n, np.float32)
        _check(lib().deg_export_codes(self._h, DEG_FP8, codes.ctypes.data, scales.ctypes.data))
        return codes, scales

    def train_entry(self, k: int = 4096, iters: int = 10, stream=None) -> np.ndarray:
        """Learned entry points: k-means on the device, pivots = vertices nearest the centroids
        (deg_train_entry). Returns the cluster sizes."""
        sizes = np.empty(k, np.int64)
        _check(lib().deg_train_entry(self._h, k, iters, sizes.ctypes.data, _stream_ptr(stream)))
        return sizes

    def pivots(self, learned: bool = False) -> np.ndarray:
        """The routing pivots (caller ids): sampled at upload, or learned (train_entry)."""
        n = int(lib().deg_get_pivots(self._h, 1 if learned else 0, None, 0))
        if n < 0:
            raise DegError(DEG_ECUDA, "deg_get_pivots failed")
        out = np.empty(n, np.int32)
        if n:
            lib().deg_get_pivots(self._h, 1 if learned else 0, out.ctypes.data, n)
        return out

    @property
    def entry_vertex(self) -> int:
        return int(lib().deg_entry_vertex(self._h))

    def search(self, queries=None, k: int = 10, eps: float = 0.1, seeds=None, explore: bool = False,
               precision: str = "f32", rerank: int = 0, max_hops: int = 0, visited_cap: int = 0,
               queue_cap: int = 0, entry: str = "fixed", learned_stop: bool = False, with_status: bool = False,
               with_trace: bool = False, out=None, stream=None):
        """Alg. 1 for a batch of queries (CUDA tensors). Returns (ids, dists[, status][, trace])."""
        import torch
        if explore:
            seeds = _require_cuda(seeds, torch.int32, "vertex ids")
            nq = seeds.shape[0]
            dev = seeds.device
        else:
            queries = _require_cuda(queries, torch.float32, "queries")
            seeds = _require_cuda(seeds, torch.int32, "seeds")
            nq = queries.shape[0]
            dev = queries.device
        if out is None:
            ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
            dists = torch.empty((nq, k), dtype=torch.float32, device=dev)
        else:
            ids, dists = out
        status = torch.empty(nq, dtype=torch.int32, device=dev) if with_status else None
        trace = torch.empty((nq, 4), dtype=torch.int32, device=dev) if with_trace else None
        p = SearchParams(k, eps, PRECISIONS[precision], rerank, max_hops, visited_cap, queue_cap,
                         ENTRY_MODES[entry], 1 if learned_stop else 0)
        _check(lib().deg_search_ex(self._h, ctypes.byref(p), None if explore else _dptr(queries), _dptr(seeds),
                                   1 if explore else 0, nq, _dptr(ids), _dptr(dists), _dptr(status), _dptr(trace),
                                   _stream_ptr(stream)))
        res = [ids, dists]
        if with_status:
            res.append(status)
        if with_trace:
            res.append(trace)
        return tuple(res)

    def set_kernel_timer(self, start=None, end=None):
        """Record torch.cuda.Event start/end around the search kernels of later calls (None: stop)."""
        _check(lib().deg_set_kernel_timer(self._h, None if start is None else ctypes.c_void_p(start.cuda_event),
                                          None if end is None else ctypes.c_void_p(end.cuda_event)))

    def search_host(self, queries: np.ndarray | None, k: int, eps: float, explore_ids: np.ndarray | None = None,
                    precision: str = "f32", rerank: int = 0, entry: str = "fixed", learned_stop: bool = False,
                    out=None, stream=None):
        """End-to-end form: host arrays in and out (pinned numpy views recommended)."""
        explore = explore_ids is not None
        nq = explore_ids.shape[0] if explore else queries.shape[0]
        ids, dists = out if out is not None else (np.empty((nq, k), np.int32), np.empty((nq, k), np.float32))
        p = SearchParams(k, eps, PRECISIONS[precision], rerank, 0, 0, 0, ENTRY_MODES[entry],
                         1 if learned_stop else 0)
        qptr = None if explore else ctypes.c_void_p(queries.ctypes.data)
        sptr = ctypes.c_void_p(explore_ids.ctypes.data) if explore else None
        _check(lib().deg_search_host(self._h, ctypes.byref(p), qptr, sptr, 1 if explore else 0, nq,
                                     ctypes.c_void_p(ids.ctypes.data), ctypes.c_void_p(dists.ctypes.data),
                                     _stream_ptr(stream)))
        return ids, dists


    # ---- learned early stop -----------------------------------------------------------------
    def stop_record(self, queries, k: int, eps: float, cap: int = 256, precision: str = "f32", rerank: int = 0,
                    entry: str = "fixed", stream=None):
        """Training traces of the plain search: (features [nq, cap, 12], labels [nq, cap], counts [nq])."""
        import torch
        queries = _require_cuda(queries, torch.float32, "queries")
        nq = queries.shape[0]
        feats = torch.zeros((nq, cap, STOP_FEATURES), dtype=torch.float32, device=queries.device)
        labels = torch.zeros((nq, cap), dtype=torch.int32, device=queries.device)
        counts = torch.zeros(nq, dtype=torch.int32, device=queries.device)
        p = SearchParams(k, eps, PRECISIONS[precision], rerank, 0, 0, 0, ENTRY_MODES[entry], 0)
        _check(lib().deg_stop_record(self._h, ctypes.byref(p), _dptr(queries), nq, cap, _dptr(feats), _dptr(labels),
                                     _dptr(counts), _stream_ptr(stream)))
        return feats, labels, counts

    def set_stop_model(self, weights, threshold: float, stream=None):
        import torch
        weights = _require_cuda(weights, torch.float32, "weights")
        _check(lib().deg_set_stop_model(self._h, _dptr(weights), float(threshold), _stream_ptr(stream)))


class Server:
    """Continuous-batching server: a persistent kernel serving requests posted to a ring."""

    def __init__(self, index: "Index", capacity: int = 65536, kmax: int = 128, precision: str = "f32",
                 rerank: int = 0, entry: str = "fixed", learned_stop: bool = False, idle_timeout_s: float = 30.0,
                 max_blocks: int = 0):
        self.index = index
        self.kmax = kmax
        self.dim = index.info()[1]
        cfg = ServeConfig(capacity, kmax, PRECISIONS[precision], rerank, ENTRY_MODES[entry],
                          1 if learned_stop else 0, float(idle_timeout_s), int(max_blocks))
        self._h = ctypes.c_void_p()
        _check(lib().deg_serve_start(index._h, ctypes.byref(cfg), ctypes.byref(self._h)))

    @property
    def slots(self) -> int:
        return int(lib().deg_serve_slots(self._h))

    def submit(self, vec=None, vertex: int = -1, k: int = 10, eps: float = 0.1) -> int:
        seq = ctypes.c_int64()
        v = None if vec is None else np.ascontiguousarray(vec, np.float32)
        _check(lib().deg_serve_submit(self._h, None if v is None else v.ctypes.data, vertex, k, float(eps),
                                      ctypes.byref(seq)))
        return seq.value

    def poll(self, seq: int, k: int):
        ids = np.empty(k, np.int32)
        d = np.empty(k, np.float32)
        st = ctypes.c_int32()
        got = lib().deg_serve_poll(self._h, seq, ids.ctypes.data, d.ctypes.data, ctypes.byref(st))
        if got < 0:
            _check(got)
        return (ids, d, st.value) if got == 1 else None

    def run_trace(self, vecs, vertices, ks, epss, arrival_s, timeout_s: float = 120.0, device_times: bool = False):
        """Replay an arrival trace; returns (latency_s, ids, dists, status[, device_s])."""
        vecs = np.ascontiguousarray(vecs, np.float32)
        vertices = np.ascontiguousarray(vertices, np.int32)
        ks = np.ascontiguousarray(ks, np.int32)
        epss = np.ascontiguousarray(epss, np.float32)
        arrival_s = np.ascontiguousarray(arrival_s, np.float64)
        n = len(ks)
        lat = np.empty(n, np.float64)
        ids = np.full((n, self.kmax), -1, np.int32)
        d = np.full((n, self.kmax), np.inf, np.float32)
        st = np.empty(n, np.int32)
        dev = np.zeros(n, np.float64) if device_times else None
        _check(lib().deg_serve_run_trace(self._h, vecs.ctypes.data, vertices.ctypes.data, ks.ctypes.data,
                                         epss.ctypes.data, arrival_s.ctypes.data, n, lat.ctypes.data, ids.ctypes.data,
                                         d.ctypes.data, st.ctypes.data, None if dev is None else dev.ctypes.data,
                                         float(timeout_s)))
        return (lat, ids, d, st, dev) if device_times else (lat, ids, d, st)

    def stop(self):
        h, self._h = self._h, None
        if h:
            _check(lib().deg_serve_stop(h))


STOP_FEATURES, STOP_PARAMS = 12, 5122


def mlp_loss_grad(w, x, labels, stream=None):
    """Mean loss and gradient of the stop network on the device (the library's kernels)."""
    import torch
    w = _require_cuda(w, torch.float32, "weights")
    x = _require_cuda(x, torch.float32, "features")
    labels = _require_cuda(labels, torch.int32, "labels")
    count = x.shape[0]
    grad = torch.empty(STOP_PARAMS, dtype=torch.float32, device=w.device)
    loss = torch.empty(1, dtype=torch.float32, device=w.device)
    scratch = torch.empty(int(lib().deg_mlp_scratch_floats(count)), dtype=torch.float32, device=w.device)
    _check(lib().deg_mlp_loss_grad(_dptr(w), _dptr(x), _dptr(labels), count, _dptr(grad), _dptr(loss), _dptr(scratch),
                                   _stream_ptr(stream)))
    return loss, grad


def mlp_adam(w, m, v, grad, step: int, lr: float, stream=None):
    _check(lib().deg_mlp_adam(_dptr(w), _dptr(m), _dptr(v), _dptr(grad), step, float(lr), _stream_ptr(stream)))


def mlp_predict(w, x, stream=None):
    import torch
    p = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check(lib().deg_mlp_predict(_dptr(w), _dptr(x), x.shape[0], _dptr(p), _stream_ptr(stream)))
    return p


def mlp_init(seed: int = 0):
    """He-uniform initial weights (host numpy, float32), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((12, 64), (64, 64), (64, 2)):
        lim = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, (fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def train_stop_model(feats, labels, epochs: int = 4, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
                     pos_weight_balance: bool = False, log=None):
    """Train the stop network with the library's kernels: minibatch Adam on (features, labels)
    CUDA tensors. Returns the float32 weights (CUDA tensor) and the per-epoch mean loss."""
    import torch
    w = torch.from_numpy(mlp_init(seed)).cuda()
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    n = feats.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    step, hist = 0, []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        tot = 0.0
        for b0 in range(0, n, batch):
            sel = perm[b0:b0 + batch]
            x = feats[sel].contiguous()
            y = labels[sel].contiguous()
            loss, grad = mlp_loss_grad(w, x, y)
            step += 1
            mlp_adam(w, m, v, grad, step, lr)
            tot += float(loss.item()) * len(sel)
        hist.append(tot / n)
        if log:
            log(f"stop model epoch {ep}: loss {hist[-1]:.4f}")
    return w, hist


def nearest_rows(rows, queries, cap: int = 256, stream=None):
    """Nearest of up to 4096 CUDA float32 rows for each CUDA float32 query (the pivot routing's
    search): (index, float32 distance), exact, ties to the lower index."""
    import torch
    rows = _require_cuda(rows, torch.float32, "rows")
    queries = _require_cuda(queries, torch.float32, "queries")
    nq = queries.shape[0]
    ids = torch.empty(nq, dtype=torch.int32, device=queries.device)
    dists = torch.empty(nq, dtype=torch.float32, device=queries.device)
    _check(lib().deg_nearest_rows(_dptr(rows), rows.shape[0], rows.shape[1], _dptr(queries), nq, cap, _dptr(ids),
                                  _dptr(dists), _stream_ptr(stream)))
    return ids, dists


def knn_exact(base, queries, k: int, stream=None):
    """Eq. 1 on the device: exact k-NN of CUDA float32 queries among CUDA float32 base rows."""
    import torch
    base = _require_cuda(base, torch.float32, "base")
    queries = _require_cuda(queries, torch.float32, "queries")
    nq = queries.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device=queries.device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
    _check(lib().knn_exact(_dptr(base), base.shape[0], _dptr(queries), nq, base.shape[1], k, _dptr(ids),
                           _dptr(dists), _stream_ptr(stream)))
    return ids, dists
