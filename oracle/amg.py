"""Algebraic multigrid preconditioner (oracle; test infrastructure only).

Sec. 5.3 preconditions LOBPCG with MueLu's aggregation multigrid and Sec. 6.2.2
fixes its parameters: a degree-3 Chebyshev smoother whose largest eigenvalue
comes from 10 steps of power iteration, with eigenvalue ratio 7; plain
(unsmoothed) aggregation; at most 5 levels; and the same Chebyshev settings as
the coarse solver, with 100 power-iteration steps.  MueLu's own aggregation
and Chebyshev code is not in the paper, so this module takes the following
readings (the GPU library implements the same ones independently):

* Operator.  A = L_C, the combinatorial Laplacian (the operator of the
  combinatorial and generalized problems).  With plain aggregation and P the
  0/1 aggregate indicator, P^T L_C P is exactly the combinatorial Laplacian of
  the aggregate graph whose edge weights are the summed fine weights between
  two aggregates, so every level is again a graph.
* Aggregation (distance-2 maximal independent set, then two attachment
  phases).  Vertex v has the key ((h(v) >> 33) + 1) * 2^32 + v, where h(v)
  is SplitMix64 output number v + 1 from state mix(seed + 7 gamma + level).
  Luby rounds: with k(u) the key of an undecided vertex, 0 for a vertex
  ruled out and 2^64 - 1 for a root, m1(v) is the largest k over v and its
  neighbours, and m2(v) the largest m1 over v and its neighbours.  An
  undecided v with m2(v) = 2^64 - 1 is ruled out; one with m2(v) = k(v)
  becomes a root.  Rounds repeat until no vertex is undecided.  Roots, in
  vertex order, number the aggregates.  Phase 1: a vertex adjacent to a root
  joins it (no vertex has two root neighbours).  Phase 2: every other vertex
  joins the phase-1 aggregate of its neighbour with the largest edge weight,
  the smallest neighbour id on ties.
* Hierarchy.  Levels are added while the level has more than 2000 vertices,
  there are fewer than 5 levels, and aggregation shrinks the graph at least
  to 90 % of its size.
* Chebyshev (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
  Algorithm 12.1, applied to D^{-1} A x = D^{-1} b).  lambda_max is 1.1 times
  the last Rayleigh quotient v^T A v of the power iteration (v D-normalised,
  v <- D^{-1} A v), capped at 2, the Gershgorin bound of D^{-1} L_C; the
  start vector is SplitMix64 from state mix(seed + 9 gamma + level), counter
  i + 1.  The interval is [lambda_max / 7, lambda_max].
* Cycle.  Symmetric V-cycle: pre-smooth from zero, restrict the residual
  with P^T, recurse, prolong with P, post-smooth with the same polynomial;
  the coarsest level applies its Chebyshev polynomial once from zero.  A
  level without edges (one aggregate holding a whole graph) has
  lambda_max = 0, and its smoother leaves x unchanged.

Pins (tests/test_oracle_amg.py): the distance-2 independence and maximality of
the roots by breadth-first search; every vertex in one connected aggregate;
the coarse Laplacian against the dense product P^T L P; the Chebyshev error
polynomial against T_3((theta - lambda) / delta) / T_3(theta / delta) on the
eigenvectors of D^{-1} L; the power-iteration estimate against the dense
eigenvalues; the V-cycle's symmetry and positivity on the complement of the
null vector; LOBPCG with it against dense eigenvalues.
"""

from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from .laplacian import laplacian_combinatorial, weighted_degree
from .rng import GAMMA, MASK, _mix64_np, mix64

ROOT_KEY = np.uint64((1 << 64) - 1)
COARSE_MAX = 2000
MAX_LEVELS = 5
CHEB_DEGREE = 3
CHEB_RATIO = 7.0
POWER_ITERS = 10
POWER_ITERS_COARSE = 100
BOOST = 1.1


def vertex_keys(n: int, seed: int, level: int) -> np.ndarray:
    """Luby priority keys of the aggregation (unique, in [2^32, 2^63 + 2^32))."""
    state = mix64((seed + 7 * GAMMA + level) & MASK)
    ctr = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = _mix64_np(np.uint64(state) + ctr * np.uint64(GAMMA))
    return (((h >> np.uint64(33)) + np.uint64(1)) << np.uint64(32)) | np.arange(n, dtype=np.uint64)


def _row_max(g, vals: np.ndarray) -> np.ndarray:
    """max over v and its neighbours of vals (uint64)."""
    out = vals.copy()
    deg = g.degrees()
    nz = deg > 0
    if g.nnz:
        nb = np.maximum.reduceat(vals[g.col], g.row_ptr[:-1][nz])
        out[nz] = np.maximum(out[nz], nb)
    return out


def mis2_roots(g, seed: int, level: int = 0):
    """Distance-2 maximal independent set by Luby rounds; returns (is_root, rounds)."""
    key = vertex_keys(g.n, seed, level)
    undecided, root = np.ones(g.n, dtype=bool), np.zeros(g.n, dtype=bool)
    rounds = 0
    while undecided.any():
        k = np.where(root, ROOT_KEY, np.where(undecided, key, np.uint64(0)))
        m2 = _row_max(g, _row_max(g, k))
        out = undecided & (m2 == ROOT_KEY)
        new = undecided & ~out & (m2 == key)
        undecided &= ~(out | new)
        root |= new
        rounds += 1
    return root, rounds


def aggregate(g, seed: int, level: int = 0):
    """Aggregate id of every vertex (int64) and the number of aggregates."""
    root, _ = mis2_roots(g, seed, level)
    n = g.n
    agg = np.full(n, -1, dtype=np.int64)
    agg[root] = np.arange(int(root.sum()))
    rows = g.rows()
    w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    # phase 1: neighbours of a root
    a1 = agg.copy()
    hit = root[g.col] & ~root[rows]
    a1[rows[hit]] = agg[g.col[hit]]
    # phase 2: the rest join the phase-1 aggregate of the heaviest neighbour (smallest id on ties)
    agg2 = a1.copy()
    cand = (a1[rows] < 0) & (a1[g.col] >= 0)
    cv, cu, cw = rows[cand], g.col[cand].astype(np.int64), w[cand]
    order = np.lexsort((cu, -cw, cv))              # by v, then heaviest, then smallest u
    cv, cu = cv[order], cu[order]
    first = np.ones(cv.size, dtype=bool)
    first[1:] = cv[1:] != cv[:-1]
    agg2[cv[first]] = a1[cu[first]]
    assert (agg2 >= 0).all(), "a vertex was left without an aggregate"
    return agg2, int(root.sum())


def coarse_graph(g, agg: np.ndarray, nc: int):
    """The aggregate graph: edge weight w_IJ = sum of w_ij over fine edges between I != J (FP64)."""
    from workloads.graphs import CSRGraph
    rows = g.rows()
    w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    ai, aj = agg[rows], agg[g.col]
    keep = ai != aj
    m = sp.coo_matrix((w[keep], (ai[keep], aj[keep])), shape=(nc, nc)).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return CSRGraph(n=nc, row_ptr=m.indptr.astype(np.int64), col=m.indices.astype(np.int32),
                    w=m.data.astype(np.float64), name="aggregate graph")


def power_lambda_max(g, iters: int, seed: int, level: int) -> float:
    """1.1 x the Rayleigh quotient of `iters` power steps on D^{-1} L_C, capped at 2."""
    lmat = laplacian_combinatorial(g)
    deg = weighted_degree(g)
    dinv = np.where(deg > 0, 1.0 / np.where(deg > 0, deg, 1.0), 0.0)
    state = mix64((seed + 9 * GAMMA + level) & MASK)
    ctr = np.arange(1, g.n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        v = (_mix64_np(np.uint64(state) + ctr * np.uint64(GAMMA)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    v = 2.0 * v - 1.0
    nrm = np.sqrt(np.sum(deg * v * v))
    if nrm == 0:
        return 0.0                              # a level without edges
    v /= nrm
    lam = 0.0
    for _ in range(iters):
        y = lmat @ v
        lam = float(v @ y)
        wv = dinv * y
        s = np.sqrt(np.sum(deg * wv * wv))
        if s == 0:
            break
        v = wv / s
    return min(BOOST * lam, 2.0)


def chebyshev(lmat, dinv: np.ndarray, lam_max: float, b: np.ndarray, x=None, degree: int = CHEB_DEGREE):
    """Chebyshev acceleration of D^{-1} A x = D^{-1} b on [lam_max/ratio, lam_max] (Saad, Alg. 12.1).
    A level without edges (lam_max = 0) leaves x as it is (zero from a zero start)."""
    if not lam_max > 0:
        return np.zeros_like(b) if x is None else x.copy()
    lam_min = lam_max / CHEB_RATIO
    theta, delta = 0.5 * (lam_max + lam_min), 0.5 * (lam_max - lam_min)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x is None:
        x = np.zeros_like(b)
        r = dinv[:, None] * b
    else:
        x = x.copy()
        r = dinv[:, None] * (b - lmat @ x)
    d = r / theta
    for k in range(1, degree + 1):
        x = x + d
        if k < degree:
            r = r - dinv[:, None] * (lmat @ d)
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * r
            rho = rho_new
    return x


@dataclasses.dataclass
class Level:
    g: object
    lmat: object
    dinv: np.ndarray
    lam_max: float
    agg: np.ndarray = None       # aggregate of each vertex (to the next level)
    nc: int = 0


def build_hierarchy(g, seed: int = 1):
    """Levels 0..L-1 of the plain-aggregation hierarchy with their Chebyshev bounds."""
    levels = []
    cur = g
    while True:
        ell = len(levels)
        deg = weighted_degree(cur)
        dinv = np.where(deg > 0, 1.0 / np.where(deg > 0, deg, 1.0), 0.0)
        lv = Level(cur, laplacian_combinatorial(cur), dinv, 0.0)
        levels.append(lv)
        coarsest = cur.n <= COARSE_MAX or ell + 1 >= MAX_LEVELS
        if not coarsest:
            agg, nc = aggregate(cur, seed, ell)
            if nc > 0.9 * cur.n:
                coarsest = True
            else:
                lv.agg, lv.nc = agg, nc
                cur = coarse_graph(cur, agg, nc)
        lv.lam_max = power_lambda_max(lv.g, POWER_ITERS_COARSE if coarsest else POWER_ITERS, seed, ell)
        if coarsest:
            break
    return levels


def vcycle(levels, b: np.ndarray, ell: int = 0) -> np.ndarray:
    """One symmetric V-cycle x = M b (b: n x k block)."""
    lv = levels[ell]
    if ell == len(levels) - 1:
        return chebyshev(lv.lmat, lv.dinv, lv.lam_max, b)
    x = chebyshev(lv.lmat, lv.dinv, lv.lam_max, b)
    r = b - lv.lmat @ x
    bc = np.zeros((lv.nc, b.shape[1]))
    np.add.at(bc, lv.agg, r)
    ec = vcycle(levels, bc, ell + 1)
    x = x + ec[lv.agg]
    return chebyshev(lv.lmat, lv.dinv, lv.lam_max, b, x)
