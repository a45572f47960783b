"""Graph files for the named workloads: load ``data/<workload>.deg`` or build it with the library's
own builder (``deg_build``, host C++) and save it there. A 10^6-vertex build takes hours on one
core, so a built file is reused; it stores the adjacency only plus a checksum of the vectors it
was built on, and loading fails if the regenerated vectors differ."""
from __future__ import annotations

import os
import sys
import time

from . import Index, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DATA = os.path.join(ROOT, "data")


def graph_path(w: synth.Workload) -> str:
    return os.path.join(DATA, f"{w.name}.deg")


def load_or_build(w: synth.Workload, base, allow_build: bool = True) -> Index:
    path = graph_path(w)
    if os.path.exists(path):
        return Index.load(path, base)
    if not allow_build:
        raise FileNotFoundError(f"graph file {path} is missing")
    print(f"[graphs] building {w.name} ({w.n} x {w.dim}, d={w.degree}); this can take long", file=sys.stderr)
    t0 = time.time()
    idx = Index.build(base, w.degree, w.k_ext, w.eps_ext, w.k_opt, w.eps_opt, w.i_opt)
    os.makedirs(DATA, exist_ok=True)
    idx.save(path, with_vectors=False)
    print(f"[graphs] built {w.name} in {time.time() - t0:.0f} s", file=sys.stderr)
    return idx
