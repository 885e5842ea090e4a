"""Seeded synthetic inputs for the R-tree range-select and join workloads.

This module only draws numbers.  It holds none of the index's arithmetic (no
predicate, no packing, no traversal), so both the CUDA path and the CPU oracle
can consume what it produces without sharing any of the method's code.

Every generator uses only ``Generator.random()`` (uniform doubles from PCG64)
and derives other distributions from it (Box-Muller for the Gaussian clusters,
inverse CDF for log-uniform sizes), so the same seed gives the same bytes on
any NumPy version that keeps PCG64's uniform stream.

Rectangles are ``float32[n, 4]`` rows ``[xmin, ymin, xmax, ymax]``.  Corners
are drawn in float64 and the upper corner is rounded from ``lo + side``, so
``xmax >= xmin`` always holds after rounding (rounding is monotone).

The paper evaluates on synthetic uniform data only (Section 5: an index of
10M uniform 2-D points, 32-bit keys, fanout 64, selectivity 0.1%).  The
workloads below keep that shape and add the clustered and heavy-tailed mixes
used for the GPU measurements; points are the side-0 special case.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "rng_for",
    "uniform_rects",
    "clustered_rects",
    "mixed_rects",
    "selectivity_queries",
    "uneven_queries",
    "uniform_queries",
    "Workload",
    "workload",
    "WORKLOADS",
]


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _u(rng: np.random.Generator, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    return lo + (hi - lo) * rng.random(n)


def _log_u(rng: np.random.Generator, n: int, lo: float, hi: float) -> np.ndarray:
    return np.exp(_u(rng, n, math.log(lo), math.log(hi)))


def _gauss(rng: np.random.Generator, n: int) -> np.ndarray:
    # Box-Muller from two uniform streams; 1 - U avoids log(0).
    u1 = 1.0 - rng.random(n)
    u2 = rng.random(n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _pack(x0: np.ndarray, y0: np.ndarray, w: np.ndarray, h: np.ndarray) -> np.ndarray:
    out = np.empty((x0.shape[0], 4), dtype=np.float32)
    out[:, 0] = x0.astype(np.float32)
    out[:, 1] = y0.astype(np.float32)
    out[:, 2] = (x0 + w).astype(np.float32)
    out[:, 3] = (y0 + h).astype(np.float32)
    return out


def _sides(rng, n, side_lo, side_hi, log_sides):
    if log_sides:
        return _log_u(rng, n, side_lo, side_hi), _log_u(rng, n, side_lo, side_hi)
    return _u(rng, n, side_lo, side_hi), _u(rng, n, side_lo, side_hi)


def uniform_rects(n: int, rng: np.random.Generator, side_lo: float = 0.0,
                  side_hi: float = 1e-3, log_sides: bool = False) -> np.ndarray:
    """Lower-left corner uniform in [0,1]^2, sides uniform (or log-uniform)."""
    x0 = _u(rng, n)
    y0 = _u(rng, n)
    w, h = _sides(rng, n, side_lo, side_hi, log_sides)
    return _pack(x0, y0, w, h)


def clustered_rects(n: int, rng: np.random.Generator, n_clusters: int = 64,
                    sigma: float = 0.02, side_lo: float = 1e-5, side_hi: float = 1e-3,
                    log_sides: bool = True) -> np.ndarray:
    """Lower-left corner from a mixture of isotropic Gaussians.

    Centres are uniform in [0,1]^2, each draw picks a centre uniformly, adds
    ``sigma * N(0,1)`` per axis and is clipped to the unit square.
    """
    cx = _u(rng, n_clusters)
    cy = _u(rng, n_clusters)
    pick = np.minimum((rng.random(n) * n_clusters).astype(np.int64), n_clusters - 1)
    x0 = np.clip(cx[pick] + sigma * _gauss(rng, n), 0.0, 1.0)
    y0 = np.clip(cy[pick] + sigma * _gauss(rng, n), 0.0, 1.0)
    w, h = _sides(rng, n, side_lo, side_hi, log_sides)
    return _pack(x0, y0, w, h)


def mixed_rects(n: int, rng: np.random.Generator, frac_clustered: float = 0.8,
                side_lo: float = 1e-5, side_hi: float = 1e-3, log_sides: bool = True,
                n_clusters: int = 64, sigma: float = 0.02) -> np.ndarray:
    """A clustered part and a uniform part, interleaved in a seeded order."""
    nc = int(round(n * frac_clustered))
    a = clustered_rects(nc, rng, n_clusters, sigma, side_lo, side_hi, log_sides)
    b = uniform_rects(n - nc, rng, side_lo, side_hi, log_sides)
    out = np.concatenate([a, b], axis=0)
    perm = np.argsort(rng.random(n), kind="stable")
    return np.ascontiguousarray(out[perm])


def uniform_queries(q: int, rng: np.random.Generator, side_lo: float = 0.0,
                    side_hi: float = 0.01) -> np.ndarray:
    return uniform_rects(q, rng, side_lo, side_hi, log_sides=False)


def selectivity_queries(q: int, rng: np.random.Generator, sel_lo: float, sel_hi: float,
                        mean_data_side: float) -> np.ndarray:
    """Square queries whose expected selectivity is log-uniform in [sel_lo, sel_hi].

    At unit density a square of side ``s`` meets a data rectangle of mean side
    ``w`` with probability about ``(s + w)^2``, so the side is
    ``max(0, sqrt(sel) - w)``.  The lower-left corner is uniform in
    ``[0, 1 - s]`` so the query stays inside the unit square.
    """
    sel = _log_u(rng, q, sel_lo, sel_hi)
    s = np.maximum(0.0, np.sqrt(sel) - mean_data_side)
    x0 = _u(rng, q) * (1.0 - s)
    y0 = _u(rng, q) * (1.0 - s)
    return _pack(x0, y0, s, s)


def uneven_queries(q: int, rng: np.random.Generator, heavy_frac: float = 0.01,
                   light=(0.0, 1e-3), heavy=(0.05, 0.2)) -> np.ndarray:
    """Heavy-tailed mix: most queries small, a seeded ``heavy_frac`` large."""
    is_heavy = rng.random(q) < heavy_frac
    lo = np.where(is_heavy, heavy[0], light[0])
    hi = np.where(is_heavy, heavy[1], light[1])
    w = lo + (hi - lo) * rng.random(q)
    h = lo + (hi - lo) * rng.random(q)
    x0 = _u(rng, q) * (1.0 - w)
    y0 = _u(rng, q) * (1.0 - h)
    return _pack(x0, y0, w, h)


def _log_uniform_mean(lo: float, hi: float) -> float:
    return (hi - lo) / math.log(hi / lo)


@dataclass
class Workload:
    """One named workload: data rectangles plus queries or a join partner."""
    name: str
    fanout: int
    rects: np.ndarray
    ids: np.ndarray
    queries: np.ndarray | None = None
    rects_s: np.ndarray | None = None
    ids_s: np.ndarray | None = None
    meta: dict = field(default_factory=dict)


def _ids(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.int32)


# name -> (description, default sizes); sizes can be scaled down for tests.
WORKLOADS = {
    "plain": "100k uniform rects (sides U[0,1e-3]), fanout 16; 1k uniform queries (sides U[0,0.01])",
    "scaled": "10M rects (80% 64-cluster Gaussian, 20% uniform; sides log-U[1e-5,1e-3]); "
              "1M square queries, selectivity log-U[1e-6,1e-3]",
    "join": "R 2M uniform, S 2M clustered, sides U[0,5e-4], fanout 32",
    "uneven": "10M-rect clustered index; 100k queries, 99% sides U[0,1e-3], 1% sides U[0.05,0.2]",
    "serve": "50M rects 50/50 uniform/clustered; Poisson stream of single queries "
             "(selectivity log-U[1e-7,1e-3]) and probe joins of 1k-10k uniform rects",
}


def workload(name: str, seed: int | None = None, n: int | None = None,
             q: int | None = None, fanout: int | None = None) -> Workload:
    """Build a named workload; ``n``/``q`` override the full sizes."""
    if name == "plain":
        seed = 0 if seed is None else seed
        rng = rng_for(seed)
        n = 100_000 if n is None else n
        q = 1_000 if q is None else q
        r = uniform_rects(n, rng, 0.0, 1e-3)
        qs = uniform_queries(q, rng, 0.0, 0.01)
        return Workload(name, fanout or 16, r, _ids(n), qs, meta={"seed": seed})
    if name == "scaled":
        seed = 1 if seed is None else seed
        rng = rng_for(seed)
        n = 10_000_000 if n is None else n
        q = 1_000_000 if q is None else q
        r = mixed_rects(n, rng, 0.8, 1e-5, 1e-3, True)
        mean_side = _log_uniform_mean(1e-5, 1e-3)
        qs = selectivity_queries(q, rng, 1e-6, 1e-3, mean_side)
        return Workload(name, fanout or 16, r, _ids(n), qs, meta={"seed": seed})
    if name == "join":
        seed = 2 if seed is None else seed
        rng = rng_for(seed)
        n = 2_000_000 if n is None else n
        r = uniform_rects(n, rng, 0.0, 5e-4)
        s = clustered_rects(n, rng, 64, 0.02, 0.0, 5e-4, log_sides=False)
        # R is uniform; S is "clustered as in the scaled config": 80/20 mix.
        nu = n - int(round(0.8 * n))
        if nu:
            s[-nu:] = uniform_rects(nu, rng, 0.0, 5e-4)
            s = np.ascontiguousarray(s[np.argsort(rng.random(n), kind="stable")])
        return Workload(name, fanout or 32, r, _ids(n), None, s, _ids(n), meta={"seed": seed})
    if name == "uneven":
        seed = 3 if seed is None else seed
        rng = rng_for(seed)
        n = 10_000_000 if n is None else n
        q = 100_000 if q is None else q
        r = mixed_rects(n, rng, 0.8, 1e-5, 1e-3, True)
        qs = uneven_queries(q, rng, 0.01)
        return Workload(name, fanout or 16, r, _ids(n), qs, meta={"seed": seed})
    if name == "serve":
        seed = 4 if seed is None else seed
        rng = rng_for(seed)
        n = 50_000_000 if n is None else n
        q = 10_000 if q is None else q
        r = mixed_rects(n, rng, 0.5, 1e-5, 1e-3, True)
        mean_side = _log_uniform_mean(1e-5, 1e-3)
        qs = selectivity_queries(q, rng, 1e-7, 1e-3, mean_side)
        return Workload(name, fanout or 16, r, _ids(n), qs, meta={"seed": seed})
    raise KeyError(f"unknown workload {name!r}; known: {sorted(WORKLOADS)}")
