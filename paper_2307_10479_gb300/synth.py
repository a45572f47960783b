"""Seeded synthetic workloads shaped like the paper's datasets.

The paper evaluates on SIFT1M, GloVe, Audio and Enron (Sec. 6.1, Table 1). Those files are
not available here, so every input is generated from a fixed seed with the shape and value
distribution of the workload it stands in for:

* ``uniform``          -- iid U[0,1) float32 rows (the small 10k x 32 parity workload).
* ``mixture_u8``       -- SIFT1M-like: Gaussian mixture around integer centres in 0..255,
                          rounded half-to-even and clipped, stored as float32 integers.
* ``mixture``          -- high-dimensional Gaussian mixture (1M x 960 precision workload).
* ``vmf_mixture``      -- GloVe-like unit vectors: a von Mises-Fisher mixture sampled with
                          Wood's (1994) rejection algorithm.

This module holds random inputs only -- none of the search method's arithmetic -- so both the
CUDA path and the CPU oracle can consume it.
"""
from __future__ import annotations

import dataclasses
import numpy as np

_CHUNK = 1 << 14   # rows drawn per generator call; whole chunks are drawn so a smaller n is a prefix


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def uniform(n: int, dim: int, seed: int) -> np.ndarray:
    """iid U[0,1) float32 matrix [n, dim]."""
    rng = np.random.default_rng(int(seed))
    return rng.random((n, dim), dtype=np.float32)


def mixture_u8_centres(n_centres: int, dim: int, seed: int) -> np.ndarray:
    rng = _rng(seed, 0xC0)
    return rng.integers(0, 256, size=(n_centres, dim)).astype(np.float64)


def mixture_u8(n: int, centres: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Rows = centre + N(0, sigma^2) per dim, rounded half-to-even, clipped to [0,255], float32."""
    rng = _rng(seed, 0x51)
    out = np.empty((n, centres.shape[1]), dtype=np.float32)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        a = rng.integers(0, centres.shape[0], size=_CHUNK)
        x = centres[a] + rng.normal(0.0, sigma, size=(_CHUNK, centres.shape[1]))
        out[lo:hi] = np.clip(np.rint(x[:hi - lo]), 0.0, 255.0)
    return out


def mixture_centres(n_centres: int, dim: int, seed: int) -> np.ndarray:
    rng = _rng(seed, 0xC1)
    return rng.standard_normal((n_centres, dim))


def mixture(n: int, centres: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Rows = centre + N(0, sigma^2) per dim, float32."""
    rng = _rng(seed, 0x52)
    out = np.empty((n, centres.shape[1]), dtype=np.float32)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        a = rng.integers(0, centres.shape[0], size=_CHUNK)
        x = centres[a] + rng.normal(0.0, sigma, size=(_CHUNK, centres.shape[1]))
        out[lo:hi] = x[:hi - lo]
    return out


def vmf_directions(n_dirs: int, dim: int, seed: int) -> np.ndarray:
    rng = _rng(seed, 0xC2)
    g = rng.standard_normal((n_dirs, dim))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def _wood_w(rng: np.random.Generator, count: int, dim: int, kappa: float) -> np.ndarray:
    """Wood (1994): sample the cosine w = <x, mu> of a vMF(mu, kappa) draw on S^{dim-1}."""
    m1 = dim - 1.0
    b = (-2.0 * kappa + np.sqrt(4.0 * kappa * kappa + m1 * m1)) / m1
    x0 = (1.0 - b) / (1.0 + b)
    c = kappa * x0 + m1 * np.log(1.0 - x0 * x0)
    w = np.empty(count)
    todo = np.arange(count)
    while todo.size:
        z = rng.beta(m1 / 2.0, m1 / 2.0, size=todo.size)
        cand = (1.0 - (1.0 + b) * z) / (1.0 - (1.0 - b) * z)
        u = rng.random(todo.size)
        ok = kappa * cand + m1 * np.log(1.0 - x0 * cand) - c >= np.log(u)
        w[todo[ok]] = cand[ok]
        todo = todo[~ok]
    return w


def vmf_mixture(n: int, dirs: np.ndarray, kappa: float, seed: int) -> np.ndarray:
    """Unit-norm float32 rows drawn from an equal-weight mixture of vMF(mu_j, kappa)."""
    rng = _rng(seed, 0x53)
    dim = dirs.shape[1]
    out = np.empty((n, dim), dtype=np.float32)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        mu = dirs[rng.integers(0, dirs.shape[0], size=_CHUNK)]
        w = _wood_w(rng, _CHUNK, dim, kappa)
        g = rng.standard_normal((_CHUNK, dim))
        g -= np.sum(g * mu, axis=1, keepdims=True) * mu
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        x = w[:, None] * mu + np.sqrt(np.maximum(0.0, 1.0 - w * w))[:, None] * g
        out[lo:hi] = (x / np.linalg.norm(x, axis=1, keepdims=True))[:hi - lo]
    return out


def distinct_ids(n: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct vertex ids drawn uniformly from [0, n), int32."""
    rng = _rng(seed, 0x1D)
    return rng.choice(n, size=count, replace=False).astype(np.int32)


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds, float64) of a Poisson process with the given rate."""
    rng = _rng(seed, 0xA7)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named workload: how to make its base and query sets, and its graph/search settings."""
    name: str
    n: int
    dim: int
    nq: int
    degree: int
    k: int
    kind: str                   # uniform | mixture_u8 | mixture | vmf
    n_centres: int = 0
    spread: float = 0.0         # sigma for mixtures, kappa for vMF
    # build parameters (Table 2 row the workload follows)
    k_ext: int = 0
    eps_ext: float = 0.2
    k_opt: int = 0
    eps_opt: float = 0.001
    i_opt: int = 5

    def base(self) -> np.ndarray:
        return _make(self, self.n, seed=0)

    def queries(self, nq: int | None = None) -> np.ndarray:
        return _make(self, self.nq if nq is None else nq, seed=1)

    def explore_ids(self, count: int | None = None) -> np.ndarray:
        return distinct_ids(self.n, self.nq if count is None else count, seed=2)

    def training_queries(self, count: int) -> np.ndarray:
        return _make(self, count, seed=3)


def _make(w: Workload, count: int, seed: int) -> np.ndarray:
    if w.kind == "uniform":
        return uniform(count, w.dim, seed)
    if w.kind == "mixture_u8":
        return mixture_u8(count, mixture_u8_centres(w.n_centres, w.dim, 7), w.spread, seed)
    if w.kind == "mixture":
        return mixture(count, mixture_centres(w.n_centres, w.dim, 7), w.spread, seed)
    if w.kind == "vmf":
        return vmf_mixture(count, vmf_directions(w.n_centres, w.dim, 7), w.spread, seed)
    raise ValueError(w.kind)


# The workloads: sizes, distributions and Table 2 build parameters.
WORKLOADS = {
    # 10k x 32 uniform, d=8 (no Table 2 row: k_ext = 2d, as the SIFT/Enron rows use 2d)
    "uniform-10k-d32": Workload("uniform-10k-d32", 10_000, 32, 1_000, 8, 10, "uniform",
                                k_ext=16, eps_ext=0.2, k_opt=8, eps_opt=0.001, i_opt=5),
    # SIFT1M-shaped: 1M x 128 integer mixture, Table 2 SIFT1M row
    "sift-1m-d128": Workload("sift-1m-d128", 1_000_000, 128, 10_000, 30, 10, "mixture_u8",
                             n_centres=1000, spread=20.0,
                             k_ext=60, eps_ext=0.2, k_opt=30, eps_opt=0.001, i_opt=5),
    # 1M x 960 Gaussian mixture, Table 2 Enron row (the paper's high-dimensional set)
    "mix-1m-d960": Workload("mix-1m-d960", 1_000_000, 960, 1_000, 30, 10, "mixture",
                            n_centres=500, spread=0.3,
                            k_ext=60, eps_ext=0.3, k_opt=30, eps_opt=0.001, i_opt=5),
    # GloVe-shaped: 1.2M x 100 unit vectors, Table 2 GloVe row
    "glove-1.2m-d100": Workload("glove-1.2m-d100", 1_200_000, 100, 10_000, 30, 10, "vmf",
                                n_centres=2000, spread=50.0,
                                k_ext=30, eps_ext=0.2, k_opt=30, eps_opt=0.001, i_opt=5),
}


def scaled(w: Workload, n: int, nq: int) -> Workload:
    """Same distribution and parameters at a different size (tests, bounded CPU samples)."""
    return dataclasses.replace(w, name=f"{w.name}@{n}", n=n, nq=nq)
