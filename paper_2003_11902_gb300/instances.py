"""Seeded synthetic inputs for the MMAS hot path.

This module only draws random inputs. It holds none of the method's arithmetic:
distances, heuristic weights, candidate lists, node selection and the pheromone
rules are computed by the CUDA library and, independently, by the CPU oracle.
Both sides receive the same arrays from here.

The paper evaluates on TSPLIB instances of 198 to 18,512 cities (Sec. 5 and
Sec. 5.7). Those files are not shipped; the generators below stand in for them
with instances of the same sizes and shapes:

* ``uniform``   -- integer coordinates uniform in [0, side)^2 (default side 10,000).
* ``clustered`` -- Gaussian clusters (default 40 centres, sigma 300) in [0, 100,000)^2,
  clipped and rounded, the shape of the clustered TSPLIB instances (e.g. fl3795).
* ``grid``      -- an a x b lattice with a fixed spacing (closed-form optimum).
* ``convex``    -- points in strictly convex position (optimal tour = hull order).

Duplicate points are redrawn, so every distance between distinct cities is
positive, as the problem statement in Sec. 2.1 requires.
All generators use numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform", "clustered", "grid", "convex", "log_uniform_sizes",
    "random_permutation", "random_pheromone",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _fill_distinct(n: int, draw) -> np.ndarray:
    """Call ``draw(k)`` (returning k x 2 int64 points) until n distinct points exist.

    The first occurrence of each point is kept, in draw order.
    """
    pts = np.empty((0, 2), dtype=np.int64)
    while pts.shape[0] < n:
        extra = draw(max(16, 2 * (n - pts.shape[0])))
        allp = np.concatenate([pts, extra], axis=0)
        _, first = np.unique(allp, axis=0, return_index=True)
        keep = np.sort(first)
        pts = allp[keep]
    return np.ascontiguousarray(pts[:n].astype(np.int32))


def uniform(n: int, seed: int, side: int = 10000) -> np.ndarray:
    """n distinct integer points uniform in [0, side)^2, shape (n, 2), int32."""
    if n < 1:
        return np.empty((0, 2), dtype=np.int32)
    rng = _rng(seed)
    return _fill_distinct(n, lambda k: rng.integers(0, side, size=(k, 2), dtype=np.int64))


def clustered(n: int, seed: int, centres: int = 40, sigma: float = 300.0,
              side: int = 100000) -> np.ndarray:
    """n distinct points around ``centres`` Gaussian centres, clipped to [0, side)^2."""
    rng = _rng(seed)
    c = rng.uniform(0.0, float(side), size=(centres, 2))

    def draw(k):
        idx = rng.integers(0, centres, size=k)
        p = c[idx] + rng.normal(0.0, sigma, size=(k, 2))
        p = np.clip(np.rint(p), 0, side - 1)
        return p.astype(np.int64)

    return _fill_distinct(n, draw)


def grid(a: int, b: int, spacing: int = 100, origin: int = 0) -> np.ndarray:
    """An a x b lattice (a columns, b rows) with the given spacing, row-major."""
    xs, ys = np.meshgrid(np.arange(a), np.arange(b))
    pts = np.stack([xs.ravel(), ys.ravel()], axis=1) * spacing + origin
    return np.ascontiguousarray(pts.astype(np.int32))


def convex(n: int, seed: int, radius: int = 5000) -> np.ndarray:
    """n integer points in strictly convex position, returned in a shuffled order.

    Points are drawn on a circle at random angles and rounded; a draw is kept
    only if the rounded points, taken in angle order, turn strictly left at every
    vertex. The returned order is shuffled so the hull order is not the index order.
    """
    rng = _rng(seed)
    for _ in range(10000):
        ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, size=n))
        p = np.rint(np.stack([np.cos(ang), np.sin(ang)], axis=1) * radius).astype(np.int64)
        p += radius + 10
        a = p
        b = np.roll(p, -1, axis=0)
        c = np.roll(p, -2, axis=0)
        cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - b[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - b[:, 0])
        if np.all(cross > 0) and len(np.unique(p, axis=0)) == n:
            perm = rng.permutation(n)
            return np.ascontiguousarray(p[perm].astype(np.int32))
    raise RuntimeError("could not draw a convex configuration")


def log_uniform_sizes(count: int, seed: int, lo: int = 100, hi: int = 2000) -> np.ndarray:
    """``count`` instance sizes round(exp(U[ln lo, ln hi])), int32."""
    rng = _rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int32)


def random_permutation(n: int, seed: int) -> np.ndarray:
    """A uniformly random permutation of 0..n-1, int32."""
    return _rng(seed).permutation(n).astype(np.int32)


def random_pheromone(n: int, seed: int, lo: float, hi: float) -> np.ndarray:
    """A symmetric float32 n x n field with entries uniform in [lo, hi] and a zero diagonal."""
    rng = _rng(seed)
    u = rng.uniform(lo, hi, size=(n, n)).astype(np.float32)
    t = np.triu(u, 1)
    t = t + t.T
    np.fill_diagonal(t, 0.0)
    return np.ascontiguousarray(t.astype(np.float32))


# Parameter vector of the learned edge prior (layout in include/mmas.h):
# (name, rows, cols) for W0 [64][8], b0, W1..W3 [64][128] with biases, Wq [64][64], a, c.
PRIOR_LAYOUT = [("W0", 64, 8), ("b0", 64, 1), ("W1", 64, 128), ("b1", 64, 1), ("W2", 64, 128),
                ("b2", 64, 1), ("W3", 64, 128), ("b3", 64, 1), ("Wq", 64, 64), ("a", 1, 1),
                ("c", 1, 1)]


def prior_params(seed: int) -> np.ndarray:
    """Seeded initial parameters of the learned prior, float32: weight matrices
    N(0, 1/cols), the layer weights halved (the residual stack stays stable),
    zero biases, a = -1, c = 0."""
    rng = _rng(seed)
    parts = []
    for name, rows, cols in PRIOR_LAYOUT:
        if name.startswith("W"):
            std = (1.0 / cols) ** 0.5 * (0.5 if name in ("W1", "W2", "W3") else 1.0)
            parts.append(rng.standard_normal(rows * cols) * std)
        elif name == "a":
            parts.append(np.array([-1.0]))
        else:
            parts.append(np.zeros(rows * cols))
    return np.concatenate(parts).astype(np.float32)
