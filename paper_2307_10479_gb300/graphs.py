"""Graph files for the named workloads: load ``data/<workload>.deg``, or build the graph and save it
there. The library's device builder (``deg_build_device``: batched Alg. 3 with optimizeEdge) takes
about a minute for 10^6 vertices on a GB300; the host builder (``deg_build``, the sequential
algorithm, one core) takes 40 minutes for the 1M x 128 workload and hours for the others. A file
stores the adjacency only plus a checksum of the vectors it was built on, and loading fails if the
regenerated vectors differ."""
from __future__ import annotations

import os
import sys
import time

from . import Index, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DATA = os.path.join(ROOT, "data")


def graph_path(w: synth.Workload, builder: str = "host") -> str:
    return os.path.join(DATA, f"{w.name}.deg" if builder == "host" else f"{w.name}.{builder}.deg")


def build(w: synth.Workload, base, builder: str = "host") -> Index:
    """Build the workload's graph with its Table 2 parameters: builder "host" (sequential) or
    "device" (batched, on the current GPU)."""
    t0 = time.time()
    if builder == "device":
        idx = Index.build_device(base, w.degree, w.k_ext, w.eps_ext, k_opt=w.k_opt, eps_opt=w.eps_opt, i_opt=w.i_opt,
                                 batch_div=64)
    else:
        idx = Index.build(base, w.degree, w.k_ext, w.eps_ext, w.k_opt, w.eps_opt, w.i_opt)
    print(f"[graphs] built {w.name} ({w.n} x {w.dim}, d={w.degree}) with the {builder} builder in "
          f"{time.time() - t0:.0f} s", file=sys.stderr)
    return idx


def load_or_build(w: synth.Workload, base, allow_build: bool = True, builder: str = "host") -> Index:
    """The host-built graph file if present; else (allow_build) build it with `builder` and save it
    (a device-built graph is saved under its own name)."""
    for b in ("host", "device") if builder == "device" else ("host",):
        path = graph_path(w, b)
        if os.path.exists(path):
            return Index.load(path, base)
    if not allow_build:
        raise FileNotFoundError(f"graph file {graph_path(w)} is missing")
    idx = build(w, base, builder)
    os.makedirs(DATA, exist_ok=True)
    idx.save(graph_path(w, builder), with_vectors=False)
    return idx
