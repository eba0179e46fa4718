"""Greedy cut refinement after multi-jagged (oracle; test infrastructure only).

Sec. 7 names a greedy improvement step as a way to lower the cut after the
spectral partition, and says that KL/FM-style refinement is hard to run in
parallel.  The paper gives no algorithm; this is the reading the library
builds (a parallel, deterministic, balance-constrained greedy step), written
here as plain loops.

Weights: edge weights are the exact integers w * 2^s of the cut's fixed point
(s = 0 for unit weights), vertex weights are integers (1 when absent), so
every gain and every part weight is an exact integer.

A round, on parts p with part weights W and capacity
cap = floor((1 + eps) * W_total / K) (evaluated in double):

1. gains: for every vertex v of degree at most max_degree, with a = p[v],
   conn(v, q) = sum of the weights of v's edges into part q;  the target
   b = argmax over q != a with conn(v, q) > 0 of conn(v, q) (smallest q on
   ties) and gain(v) = conn(v, b) - conn(v, a).  v is a candidate when
   gain(v) > 0.
2. selection: a candidate v is selected when every candidate neighbour u has
   a lower priority, the priority being (gain, -id) compared
   lexicographically.  Selected vertices are pairwise non-adjacent, so each
   one's gain is exactly the cut it removes when they all move at once.
3. capacity: for every target part b, if W_b plus the weight of all selected
   vertices aimed at b stays within cap, all of them move; otherwise only
   the one of highest priority moves, if its own weight fits.
4. the accepted vertices move; the cut falls by the sum of their gains.

Rounds repeat until none moves or max_rounds is reached.  Part weights that
exceed cap never grow, and the cut never rises.

Pins (tests/test_oracle_refine.py): gains against a dense connectivity
matrix A P (P the part indicator matrix); the cut after each round equals
the cut before minus the round's gains (recomputed by metrics.cutsize);
moved vertices of a round are pairwise non-adjacent; part weights stay
within max(cap, their weight before); a hand-worked path example.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from .metrics import _exact_scale, cutsize, part_weights


@dataclasses.dataclass
class RefineResult:
    parts: np.ndarray
    cut: float
    cut_twice: float
    moves: int
    rounds: int
    round_moves: list          # per round: the vertices that moved
    round_gains: list          # per round: the summed integer gain
    scale: int                 # s of the integer edge weights w * 2^s


def integer_weights(g) -> tuple:
    """(omega, s): edge weights as the exact integers w * 2^s."""
    if g.w is None:
        return np.ones(g.nnz, dtype=np.int64), 0
    s = _exact_scale(g.w)
    return (g.w.astype(np.float64) * 2.0 ** s).astype(np.int64), s


def capacity(total_weight: int, num_parts: int, eps: float) -> int:
    """floor((1 + eps) * W_total / K), evaluated in double."""
    return int(math.floor((1.0 + eps) * float(total_weight) / float(num_parts)))


def vertex_gains(g, parts, omega, max_degree: int):
    """(gain, target) per vertex; gain 0 and target -1 when v is no candidate."""
    n = g.n
    gain = np.zeros(n, dtype=np.int64)
    target = np.full(n, -1, dtype=np.int64)
    for v in range(n):
        b0, b1 = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
        if b1 - b0 > max_degree:
            continue
        a = int(parts[v])
        conn = {}
        for e in range(b0, b1):
            q = int(parts[int(g.col[e])])
            conn[q] = conn.get(q, 0) + int(omega[e])
        internal = conn.get(a, 0)
        best_q, best_c = -1, 0
        for q in sorted(conn):
            if q != a and conn[q] > best_c:
                best_q, best_c = q, conn[q]
        if best_q >= 0 and best_c - internal > 0:
            gain[v] = best_c - internal
            target[v] = best_q
    return gain, target


def refine(g, parts, num_parts: int, vwts=None, eps: float = 0.01, max_rounds: int = 20,
           max_degree: int = 256) -> RefineResult:
    """Rounds of the greedy step above, from the partition `parts`."""
    p = np.asarray(parts, dtype=np.int64).copy()
    vw = np.ones(g.n, dtype=np.int64) if vwts is None else np.asarray(vwts, dtype=np.int64)
    omega, s = integer_weights(g)
    W = part_weights(p, vw, num_parts)
    cap = capacity(int(W.sum()), num_parts, eps)
    moves, rounds = 0, 0
    round_moves, round_gains = [], []
    for _ in range(max_rounds):
        gain, target = vertex_gains(g, p, omega, max_degree)
        selected = []
        for v in range(g.n):
            if gain[v] <= 0:
                continue
            ok = True
            for e in range(int(g.row_ptr[v]), int(g.row_ptr[v + 1])):
                u = int(g.col[e])
                if gain[u] > 0 and (gain[u] > gain[v] or (gain[u] == gain[v] and u < v)):
                    ok = False
                    break
            if ok:
                selected.append(v)
        incoming = {}
        best = {}
        for v in selected:
            b = int(target[v])
            incoming[b] = incoming.get(b, 0) + int(vw[v])
            if b not in best or (gain[v], -v) > (gain[best[b]], -best[b]):
                best[b] = v
        accepted = []
        for v in selected:
            b = int(target[v])
            if int(W[b]) + incoming[b] <= cap or (best[b] == v and int(W[b]) + int(vw[v]) <= cap):
                accepted.append(v)
        rounds += 1
        if not accepted:
            round_moves.append([])
            round_gains.append(0)
            break
        for v in accepted:
            W[p[v]] -= vw[v]
            W[target[v]] += vw[v]
            p[v] = target[v]
        moves += len(accepted)
        round_moves.append(accepted)
        round_gains.append(int(sum(int(gain[v]) for v in accepted)))
    cut, cut2 = cutsize(g, p.astype(np.int32))
    return RefineResult(p.astype(np.int32), cut, cut2, moves, rounds, round_moves, round_gains, s)
