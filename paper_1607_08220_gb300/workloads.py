"""Seeded synthetic workloads shaped like PANDA's datasets (arXiv 1607.08220, Sec. IV-B, Table I).

The paper's datasets (Gadget cosmology, VPIC plasma, Daya Bay features) are not
available; these generators stand in for them with the shapes of Table I
(3-D particle clouds; 10-D feature vectors).  The module holds no part of the
method's arithmetic: it only draws numbers (numpy PCG64, float32 at the end).

Workloads
---------
``uniform_small``      n=100,000 points U[0,1)^3 (seed 0), 10,000 queries (seed 1), k=5, B=32.
``cosmology_self``     n=2^24 points: 80% in 2,000 Gaussian halos (centres U[0,1)^3,
                       sigma log-uniform [0.002, 0.02], membership weights with a
                       power-law density of slope -1.9 on [1, 1e4]), rejection-
                       resampled into [0,1)^3, 20% uniform background, shuffled.
                       Queries are the points themselves, k=10, B=32.
``batched_sets``       512 sets, sizes log-uniform in [1e3, 2e6] (seed 2), each a scaled
                       cosmology mixture; per set 10% queries and k in {4, 8, 16, 32}.
``plasma_serving``     n=1e8 slab in [0,330]^2 x [0,132], density ~ sech^2((z-66)/4) plus a
                       10% uniform floor; a Poisson request stream (2,000 req/s, seed 3)
                       with log-uniform batch sizes in [1, 1e6] and k in {1, 8, 32}; a
                       second 20M-point tree (seed 4) admitted at t=0.5 s.
``features_10d``       n=2^23 points in 10-D, N(0, diag(0.8^i)^2) with 5% outliers U[-6,6]^10;
                       2^20 held-out queries (seed 1) in 64 log-uniform requests, k=16.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "uniform_small", "cosmology_points", "cosmology_self", "batched_sets",
    "plasma_points", "plasma_requests", "features_10d", "lattice_points", "Workload",
]


@dataclass
class Workload:
    name: str
    points: np.ndarray
    queries: np.ndarray
    k: int
    bucket: int
    meta: dict = field(default_factory=dict)


def uniform_small(n: int = 100_000, m: int = 10_000) -> Workload:
    pts = np.random.default_rng(0).random((n, 3), dtype=np.float32)
    q = np.random.default_rng(1).random((m, 3), dtype=np.float32)
    return Workload("uniform_small", pts, q, 5, 32, dict(n=n, m=m, d=3))


def _powerlaw(rng, size, slope=-1.9, lo=1.0, hi=1e4):
    # inverse CDF of p(w) ~ w^slope on [lo, hi]
    a = slope + 1.0
    u = rng.random(size)
    return (lo ** a + u * (hi ** a - lo ** a)) ** (1.0 / a)


def cosmology_points(n: int, seed: int = 0, halos: int = 2000) -> np.ndarray:
    """Clustered 3-D cloud: 80% Gaussian halos, 20% uniform background, in [0,1)^3."""
    rng = np.random.default_rng(seed)
    centres = rng.random((halos, 3))
    sigma = np.exp(rng.uniform(math.log(0.002), math.log(0.02), halos))
    w = _powerlaw(rng, halos)
    n_halo = int(round(0.8 * n))
    counts = rng.multinomial(n_halo, w / w.sum())
    owner = np.repeat(np.arange(halos), counts)
    pts = centres[owner] + sigma[owner, None] * rng.standard_normal((n_halo, 3))
    bad = np.flatnonzero(((pts < 0.0) | (pts >= 1.0)).any(axis=1))
    while bad.size:          # rejection-resample into the box (no wrap)
        o = owner[bad]
        pts[bad] = centres[o] + sigma[o, None] * rng.standard_normal((bad.size, 3))
        sub = ((pts[bad] < 0.0) | (pts[bad] >= 1.0)).any(axis=1)
        bad = bad[sub]
    bg = rng.random((n - n_halo, 3))
    allp = np.concatenate([pts, bg]).astype(np.float32)
    # float32 rounding can land a value on 1.0; keep the half-open box
    np.minimum(allp, np.float32(np.nextafter(np.float32(1.0), np.float32(0.0))), out=allp)
    return allp[rng.permutation(n)]


def cosmology_self(n: int = 1 << 24, k: int = 10, bucket: int = 32) -> Workload:
    pts = cosmology_points(n, seed=0)
    return Workload("cosmology_self", pts, pts, k, bucket, dict(n=n, m=n, d=3, self_query=True))


def batched_sets(nsets: int = 512, seed: int = 2, lo: float = 1e3, hi: float = 2e6,
                 scale: float = 1.0):
    """List of (points, queries, k) for the batched form; ``scale`` shrinks sizes for tests."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), nsets))).astype(np.int64)
    sizes = np.maximum(1, (sizes * scale).astype(np.int64))
    ks = rng.choice(np.array([4, 8, 16, 32]), nsets)
    seeds = rng.integers(0, 2**31 - 1, size=(nsets, 2))
    sets = []
    n1 = 1 << 24
    for i in range(nsets):
        size = int(sizes[i])
        halos = max(1, int(round(2000 * size / n1)))
        pts = cosmology_points(size, seed=int(seeds[i, 0]), halos=halos)
        mq = max(1, int(0.1 * size))
        q = cosmology_points(mq, seed=int(seeds[i, 1]), halos=halos)
        sets.append((pts, q, int(ks[i])))
    return sets


def plasma_points(n: int, seed: int) -> np.ndarray:
    """Slab [0,330]x[0,330]x[0,132], density ~ sech^2((z-66)/4) + 10% uniform floor."""
    rng = np.random.default_rng(seed)
    n_bg = int(round(0.1 * n))
    n_sl = n - n_bg
    xy = rng.uniform(0.0, 330.0, (n_sl, 2))
    z = np.empty(n_sl)
    todo = np.arange(n_sl)
    while todo.size:
        u = rng.random(todo.size)
        zz = 66.0 + 4.0 * np.arctanh(2.0 * u - 1.0)
        ok = (zz >= 0.0) & (zz <= 132.0)
        z[todo[ok]] = zz[ok]
        todo = todo[~ok]
    bg = rng.uniform(0.0, 1.0, (n_bg, 3)) * np.array([330.0, 330.0, 132.0])
    pts = np.concatenate([np.column_stack([xy, z]), bg]).astype(np.float32)
    return pts[rng.permutation(n)]


def plasma_requests(duration_s: float = 1.0, rate: float = 2000.0, seed: int = 3,
                    max_m: int = 1_000_000, t_second_tree: float = 0.5):
    """Poisson request stream: list of dicts(t, m, k, tree, seed)."""
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        m = int(math.floor(math.exp(rng.uniform(0.0, math.log(max_m + 1)))))
        m = max(1, min(max_m, m))
        k = int(rng.choice([1, 8, 32]))
        tree = 0 if t < t_second_tree else int(rng.integers(0, 2))
        reqs.append(dict(t=t, m=m, k=k, tree=tree, seed=int(rng.integers(0, 2**31 - 1))))
    return reqs


def features_10d(n: int = 1 << 23, m: int = 1 << 20, nreq: int = 64, k: int = 16) -> Workload:
    def draw(count, seed):
        rng = np.random.default_rng(seed)
        std = 0.8 ** np.arange(10)
        x = rng.standard_normal((count, 10)) * std
        out = rng.random(count) < 0.05
        x[out] = rng.uniform(-6.0, 6.0, (int(out.sum()), 10))
        return x.astype(np.float32)

    pts = draw(n, 0)
    q = draw(m, 1)
    rng = np.random.default_rng(5)
    raw = np.exp(rng.uniform(0.0, math.log(m), nreq))
    sizes = np.maximum(1, np.floor(raw / raw.sum() * m)).astype(np.int64)
    sizes[-1] += m - sizes.sum()
    return Workload("features_10d", pts, q, k, 32, dict(n=n, m=m, d=10, request_sizes=sizes))


def lattice_points(n: int, d: int, seed: int, side: int = 16, scale_log2: int = 4) -> np.ndarray:
    """Integer lattice coordinates scaled by 2^-scale_log2: every FP32 op on them is exact."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, side, (n, d)).astype(np.float32) * np.float32(2.0 ** -scale_log2))
