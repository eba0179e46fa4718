"""Multi-jagged multisection of coordinates (oracle; test infrastructure only).

Sec. 4 of the paper: MJ recursively multisections a point set along the
coordinate dimensions in round-robin order, cut planes in different sections
are independent of each other, and the goal is balanced part weights.  The
paper uses MJ's default settings and gives no split rule; the exact rule taken
here (a bisection per level, so K = 2^m with m = d - 1 dimensions uses every
dimension once, as in the K = 4 example of Sec. 4):

* a section owns parts [lo, lo + k) and splits into k_L = ceil(k/2) parts on
  the left and k_R = floor(k/2) on the right, along dimension level mod D;
* its points are ordered by (coordinate, vertex id), coordinates compared as
  IEEE values (-0 == +0; NaN is rejected);
* the left side is the prefix of length p* = argmin_p |k cumW(p) - k_L W|
  over p = 0..n_s (W the section weight, cumW(p) the weight of the first p
  points), ties going to the smaller p;
* recursion stops at k = 1, which assigns part lo.

Vertex weights are positive integers (unit by default), so cumW is strictly
increasing and every comparison is exact integer arithmetic.

Pins (tests/test_oracle_mj.py): brute force against an independent per-level
implementation, exact part sizes for unit weights, each dimension used once
for K = 2^m, invariance under vertex relabelling of distinct coordinates.
"""

from __future__ import annotations

import numpy as np


def coord_sort_key(c: np.ndarray) -> np.ndarray:
    """Coordinates with -0 folded onto +0 (IEEE comparison semantics)."""
    c = np.asarray(c)
    if np.isnan(c).any():
        raise ValueError("NaN coordinate")
    return c + c.dtype.type(0.0)


def _split_point(w_sorted: np.ndarray, k: int, k_left: int) -> int:
    cum = np.concatenate([[0], np.cumsum(w_sorted, dtype=object)])
    total = cum[-1]
    obj = [abs(k * c - k_left * total) for c in cum]
    return int(min(range(len(obj)), key=lambda p: (obj[p], p)))


def multijagged(coords: np.ndarray, vwts, num_parts: int) -> np.ndarray:
    """Part id (int32) of every point; coords is n x D (D >= 1 unless K == 1)."""
    coords = np.asarray(coords)
    n = coords.shape[0]
    parts = np.zeros(n, dtype=np.int32)
    if num_parts <= 1 or n == 0:
        return parts
    if coords.ndim != 2 or coords.shape[1] < 1:
        raise ValueError("need at least one coordinate dimension")
    dims = coords.shape[1]
    w = np.ones(n, dtype=np.int64) if vwts is None else np.asarray(vwts, dtype=np.int64)
    if np.any(w < 1):
        raise ValueError("vertex weights must be positive integers")
    stack = [(np.arange(n, dtype=np.int64), 0, int(num_parts), 0)]
    while stack:
        verts, lo, k, level = stack.pop()
        if k == 1:
            parts[verts] = lo
            continue
        dim = level % dims
        k_left = (k + 1) // 2
        key = coord_sort_key(coords[verts, dim])
        order = np.lexsort((verts, key))
        vs = verts[order]
        p = _split_point(w[vs], k, k_left)
        stack.append((vs[:p], lo, k_left, level + 1))
        stack.append((vs[p:], lo + k_left, k - k_left, level + 1))
    return parts
