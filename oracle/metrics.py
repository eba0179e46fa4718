"""Partition quality, exact (oracle; test infrastructure only).

Eq. 1: cutsize = sum of the costs of the cut edges, an edge e_ij being cut
when v_i and v_j lie in different parts.  The paper's tables count every cut
edge twice (once from each endpoint, Sec. 6), so both figures are returned.
Sec. 3.1: W_k is the sum of the vertex weights in part k and the imbalance is
reported as max_k W_k / W_avg with W_avg = sum_k W_k / K (Sec. 6.4, Table 7).

FP32 edge weights are summed exactly: every weight is an integer multiple of
2^-s for a common s, the sum is taken over Python integers and divided once,
so the result is the correctly rounded double of the exact cut.

Pins (tests/test_oracle_metrics.py): brute-force edge enumeration and the
identity cut = x^T L_C x / 4 for x in {-1, +1}^n (Sec. 3.2).
"""

from __future__ import annotations

import numpy as np


def _exact_scale(w32: np.ndarray) -> int:
    w = w32.astype(np.float64)
    nz = w[w != 0]
    if nz.size == 0:
        return 0
    _, e = np.frexp(nz)
    return int(24 - e.min())


def cutsize(g, parts: np.ndarray):
    """(cut, cut counted twice) for Eq. 1; both are exact."""
    parts = np.asarray(parts)
    rows = g.rows()
    diff = parts[rows] != parts[g.col.astype(np.int64)]
    if g.w is None:
        twice = int(np.count_nonzero(diff))
        return twice / 2, twice
    s = _exact_scale(g.w)
    ints = (g.w[diff].astype(np.float64) * 2.0 ** s).astype(np.int64)
    if ints.size == 0:
        total = 0
    elif int(ints.max()) * ints.size < 2 ** 62:
        total = int(np.sum(ints, dtype=np.int64))      # exact: no partial sum can overflow
    else:
        total = int(np.sum(ints.astype(object)))
    return total / 2 ** (s + 1), total / 2 ** s


def part_weights(parts: np.ndarray, vwts, num_parts: int) -> np.ndarray:
    """W_k for k = 0..K-1 (int64, exact)."""
    parts = np.asarray(parts, dtype=np.int64)
    w = np.ones(len(parts), dtype=np.int64) if vwts is None else np.asarray(vwts, dtype=np.int64)
    out = np.zeros(num_parts, dtype=np.int64)
    np.add.at(out, parts, w)
    return out


def imbalance(parts: np.ndarray, vwts, num_parts: int) -> float:
    """max_k W_k / W_avg computed as (max W_k * K) / W_total in doubles."""
    pw = part_weights(parts, vwts, num_parts)
    total = int(pw.sum())
    return (float(int(pw.max())) * float(num_parts)) / float(total)
