"""Seeded synthetic inputs shaped like the workloads of the IMQ fast-matvec method.

This module holds input generation only: point sets, data values, right-hand
sides and the recipes of the named workloads.  It contains none of the
method's arithmetic (no kernel evaluation, no expansions, no tree), so both
the CUDA path and the FP64 CPU oracle may consume its arrays.

Everything is FP64 numpy on the host and deterministic in its seed.  Each
generator draws from its own `numpy.random.Generator` keyed by
``[seed, stream]`` so that adding a new draw never perturbs another.

Recipes (the paper's only experiment is Section 3, Table 1: Halton points in
[0,1]^2, shape t=1, truncation M=10, a random vector in [-1,1]):

* ``plain_2k``      N=2,000 i.i.d. uniform in [0,1]^2, c=0.1, f=Franke, p=10, leaf=32.
* ``uniform_100k``  N=100,000 uniform, c=2 x (exact mean nearest-neighbour spacing),
                    f=sin(6x)cos(4y)+0.1 N(0,1), p=12, leaf=64.
* ``clustered_1m``  N=1,000,000: 8 isotropic Gaussians (centres uniform in
                    [0.1,0.9]^2, sigma 0.03, 87,500 points each, each coordinate
                    clamped to [0,1]) plus 300,000 uniform; c=0.01, leaf=64.
* ``batched_256``   256 problems, N_i = round(exp(U(ln 1e3, ln 5e4))), c_i ~ U[0.01,0.2],
                    4 right-hand sides each (Franke plus three trig sums).
* ``grad_200k``     200,000 training + 20,000 validation points uniform, c=0.05,
                    f = exp(-10((x-0.5)^2+(y-0.5)^2)).
* ``table1_halton`` Halton points (bases 2 and 3, index from 1), c=1, p=10.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


# --------------------------------------------------------------------------
# point sets
# --------------------------------------------------------------------------

def uniform_points(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """n points i.i.d. uniform in [0,1]^2, shape (n, 2), FP64, row-major."""
    return _rng(seed, stream).random((int(n), 2))


def clustered_points(n_cluster_each: int = 87_500, n_clusters: int = 8,
                     n_uniform: int = 300_000, sigma: float = 0.03,
                     seed: int = 3, stream: int = 0) -> np.ndarray:
    """Gaussian-mixture points clamped to [0,1]^2 followed by uniform points.

    Cluster centres are uniform in [0.1,0.9]^2.  Each cluster contributes
    ``n_cluster_each`` isotropic normal samples with standard deviation
    ``sigma`` whose coordinates are clamped ("clipped") to [0,1].
    """
    g = _rng(seed, stream)
    centres = 0.1 + 0.8 * g.random((n_clusters, 2))
    blocks = []
    for k in range(n_clusters):
        pts = centres[k] + sigma * g.standard_normal((n_cluster_each, 2))
        blocks.append(np.clip(pts, 0.0, 1.0))
    blocks.append(g.random((n_uniform, 2)))
    return np.ascontiguousarray(np.concatenate(blocks, axis=0))


def _radical_inverse(i: np.ndarray, base: int) -> np.ndarray:
    i = i.astype(np.int64).copy()
    out = np.zeros(i.shape, dtype=np.float64)
    f = 1.0 / base
    while np.any(i > 0):
        out += f * (i % base)
        i //= base
        f /= base
    return out


def halton_points(n: int, start: int = 1) -> np.ndarray:
    """First n Halton points in bases (2, 3), indices start..start+n-1 (no scrambling)."""
    idx = np.arange(start, start + int(n), dtype=np.int64)
    return np.stack([_radical_inverse(idx, 2), _radical_inverse(idx, 3)], axis=1)


# --------------------------------------------------------------------------
# data values / vectors
# --------------------------------------------------------------------------

def franke(points: np.ndarray) -> np.ndarray:
    """Franke's bivariate test function (Franke 1982), evaluated at points (n,2)."""
    x, y = points[:, 0], points[:, 1]
    t1 = 0.75 * np.exp(-((9 * x - 2) ** 2 + (9 * y - 2) ** 2) / 4.0)
    t2 = 0.75 * np.exp(-((9 * x + 1) ** 2) / 49.0 - (9 * y + 1) / 10.0)
    t3 = 0.5 * np.exp(-((9 * x - 7) ** 2 + (9 * y - 3) ** 2) / 4.0)
    t4 = -0.2 * np.exp(-(9 * x - 4) ** 2 - (9 * y - 7) ** 2)
    return t1 + t2 + t3 + t4


def sincos_noisy(points: np.ndarray, seed: int, stream: int = 7) -> np.ndarray:
    """sin(6x) cos(4y) + 0.1 N(0,1) with its own noise stream."""
    noise = _rng(seed, stream).standard_normal(points.shape[0])
    return np.sin(6 * points[:, 0]) * np.cos(4 * points[:, 1]) + 0.1 * noise


def gaussian_bump(points: np.ndarray) -> np.ndarray:
    """exp(-10((x-0.5)^2 + (y-0.5)^2))."""
    return np.exp(-10.0 * ((points[:, 0] - 0.5) ** 2 + (points[:, 1] - 0.5) ** 2))


def trig_sum(points: np.ndarray, seed: int, stream: int) -> np.ndarray:
    """sum_{k=1..4} a_k sin(2 pi (alpha_k x + beta_k y) + phi_k), a~N(0,1),
    alpha, beta integers in [1,4], phi ~ U[0, 2 pi)."""
    g = _rng(seed, stream)
    a = g.standard_normal(4)
    al = g.integers(1, 5, size=4)
    be = g.integers(1, 5, size=4)
    ph = g.random(4) * 2 * math.pi
    x, y = points[:, 0], points[:, 1]
    out = np.zeros(points.shape[0])
    for k in range(4):
        out += a[k] * np.sin(2 * math.pi * (al[k] * x + be[k] * y) + ph[k])
    return out


def random_vector(n: int, seed: int, stream: int = 11, nrhs: int = 1) -> np.ndarray:
    """Entries uniform in [-1,1]; shape (n,) or (nrhs, n)."""
    g = _rng(seed, stream)
    if nrhs == 1:
        return g.uniform(-1.0, 1.0, size=int(n))
    return g.uniform(-1.0, 1.0, size=(int(nrhs), int(n)))


def mean_nn_spacing(points: np.ndarray) -> float:
    """Exact mean over points of the Euclidean distance to the nearest other point."""
    from scipy.spatial import cKDTree
    d, _ = cKDTree(points).query(points, k=2)
    return float(np.mean(d[:, 1]))


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    points: np.ndarray
    c: float
    p: int
    leaf: int
    f: np.ndarray | None = None          # interpolation data (CG right-hand side)
    v: np.ndarray | None = None          # matvec vector, entries in [-1,1]
    domain: tuple = (0.0, 0.0, 1.0)      # (x0, y0, side) of the square D
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.points.shape[0])


def plain_2k(seed: int = 1) -> Workload:
    pts = uniform_points(2000, seed)
    return Workload("plain_2k", pts, 0.1, 10, 32, f=franke(pts), v=random_vector(2000, seed))


def uniform_100k(seed: int = 2, n: int = 100_000) -> Workload:
    pts = uniform_points(n, seed)
    c = 2.0 * mean_nn_spacing(pts)
    return Workload("uniform_100k", pts, c, 12, 64, f=sincos_noisy(pts, seed),
                    v=random_vector(n, seed))


def clustered_1m(seed: int = 3, p: int = 12, scale: float = 1.0) -> Workload:
    """N=1M clustered workload; ``scale`` shrinks every count (for quick tests)."""
    each = int(round(87_500 * scale))
    uni = int(round(300_000 * scale))
    pts = clustered_points(each, 8, uni, 0.03, seed)
    n = pts.shape[0]
    return Workload("clustered_1m" if scale == 1.0 else f"clustered_{n}", pts, 0.01, p, 64,
                    f=franke(pts), v=random_vector(n, seed))


def batched_256(seed: int = 4, n_problems: int = 256, n_lo: float = 1e3, n_hi: float = 5e4):
    """List of (points, c, rhs[4][n]) for the batched workload."""
    g = _rng(seed, 0)
    ns = np.rint(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), size=n_problems))).astype(np.int64)
    cs = g.uniform(0.01, 0.2, size=n_problems)
    probs = []
    for b in range(n_problems):
        pts = uniform_points(int(ns[b]), seed, stream=1000 + b)
        rhs = np.stack([franke(pts)] + [trig_sum(pts, seed, 5000 + 4 * b + k) for k in range(3)])
        probs.append((pts, float(cs[b]), rhs))
    return probs


def grad_200k(seed: int = 5, n_train: int = 200_000, n_val: int = 20_000):
    tr = uniform_points(n_train, seed, stream=0)
    va = uniform_points(n_val, seed, stream=1)
    return dict(train=tr, val=va, c=0.05, f=gaussian_bump(tr), y_val=gaussian_bump(va))


def table1_halton(n: int = 20_000, seed: int = 6) -> Workload:
    pts = halton_points(n)
    return Workload(f"table1_halton_{n}", pts, 1.0, 10, 64, f=franke(pts), v=random_vector(n, seed))
