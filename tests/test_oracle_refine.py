"""Pins for the greedy cut refinement (oracle.refine, the library's reading of
the greedy improvement step Sec. 7 proposes)."""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads as W
from oracle.refine import capacity, integer_weights, refine, vertex_gains


def test_hand_worked_path():
    # path 0-1-2-3-4-5 with parts [0,0,1,0,1,1]: vertices 2 and 3 both gain 2
    # (two cut edges become internal); 2 has the lower id, so it alone moves;
    # the cut falls from 3 to 1 and the parts weigh 4 and 2
    g = W.path_graph(6)
    parts = np.array([0, 0, 1, 0, 1, 1], dtype=np.int32)
    assert O.cutsize(g, parts)[0] == 3
    r = refine(g, parts, 2, eps=0.34)
    assert list(r.parts) == [0, 0, 0, 0, 1, 1]
    assert r.cut == 1 and r.moves == 1 and r.round_moves[0] == [2] and r.round_gains[0] == 2
    # cap = floor(1.01 * 3) = 3: neither part may grow, nothing moves
    r2 = refine(g, parts, 2, eps=0.01)
    assert r2.moves == 0 and list(r2.parts) == list(parts) and r2.cut == 3


@pytest.mark.parametrize("weighted", [False, True])
def test_gains_equal_the_dense_connectivity_matrix(weighted):
    """conn = A P (P the n x K part indicators), from a dense product rather
    than the per-vertex loops; the best target and the gain follow from it."""
    g = W.largest_component(W.rmat(9, seed=4))
    if weighted:
        g = W.random_edge_weights(g, 0.5, 1.5, 2)
    K = 5
    parts = np.random.default_rng(1).integers(0, K, g.n).astype(np.int32)
    omega, _ = integer_weights(g)
    A = sp.csr_matrix((omega.astype(np.float64), g.col, g.row_ptr), shape=(g.n, g.n)).toarray()
    P = np.zeros((g.n, K))
    P[np.arange(g.n), parts] = 1.0
    conn = A @ P                                   # exact: integers below 2^53
    gain, target = vertex_gains(g, parts, omega, max_degree=10 ** 9)
    for v in range(g.n):
        a = parts[v]
        ext = conn[v].copy()
        ext[a] = -1.0
        b = int(np.argmax(ext))                    # first maximum: smallest part on ties
        gv = ext[b] - conn[v, a]
        if ext[b] > 0 and gv > 0:
            assert target[v] == b and gain[v] == gv, v
        else:
            assert gain[v] == 0 and target[v] == -1, v


@pytest.mark.parametrize("make", [lambda: W.grid2d(40, 31), lambda: W.largest_component(W.rmat(10, seed=5)),
                                  lambda: W.random_edge_weights(W.grid3d(9, 8, 7, 27), 0.5, 1.5, 3)])
def test_rounds_lower_the_cut_by_their_gains_and_keep_balance(make):
    g = make()
    K = 6
    rng = np.random.default_rng(7)
    # a rough partition: blocks of consecutive ids with 5 % of the vertices relabelled
    parts = (np.arange(g.n) * K // g.n).astype(np.int32)
    flip = rng.random(g.n) < 0.05
    parts[flip] = rng.integers(0, K, int(flip.sum()))
    vw = W.random_vertex_weights(g.n, 1, 4, 9)
    eps = 0.05
    W0 = O.part_weights(parts, vw, K)
    cap = capacity(int(W0.sum()), K, eps)
    cut0 = O.cutsize(g, parts)[0]
    r = refine(g, parts, K, vwts=vw, eps=eps, max_rounds=30)
    assert r.moves > 0
    # replay the rounds: each one removes exactly its gains from the cut (in
    # units of the integer weights) and moves pairwise non-adjacent vertices
    cur = parts.astype(np.int64).copy()
    cut = cut0
    adj = sp.csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    for moved, gsum in zip(r.round_moves, r.round_gains):
        if not moved:
            continue
        omega, s = integer_weights(g)
        _, target = vertex_gains(g, cur, omega, 256)
        m = np.zeros(g.n)
        m[moved] = 1.0
        assert float(m @ (adj @ m)) == 0.0                      # independent set
        cur[moved] = target[moved]
        new_cut = O.cutsize(g, cur.astype(np.int32))[0]
        assert new_cut == cut - gsum / 2 ** s                  # exact: dyadic values below 2^53
        cut = new_cut
    assert np.array_equal(cur.astype(np.int32), r.parts)
    assert r.cut == cut < cut0
    W1 = O.part_weights(r.parts, vw, K)
    assert np.all(W1 <= np.maximum(W0, cap))


def test_the_fixed_point_has_no_fitting_selected_move():
    """With unit vertex weights, when a round moves nothing every selected
    vertex (a local maximum of the priority with positive gain) aims at a
    part that is already full."""
    g = W.grid2d(30, 30)
    K = 4
    parts = (np.arange(g.n) * K // g.n).astype(np.int32)
    rng = np.random.default_rng(3)
    flip = rng.random(g.n) < 0.2
    parts[flip] = rng.integers(0, K, int(flip.sum()))
    r = refine(g, parts, K, eps=0.02, max_rounds=1000)
    assert r.round_moves[-1] == []
    omega, _ = integer_weights(g)
    gain, target = vertex_gains(g, r.parts, omega, 256)
    Wf = O.part_weights(r.parts, None, K)
    cap = capacity(g.n, K, 0.02)
    for v in np.nonzero(gain > 0)[0]:
        nb = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        beaten = any(gain[u] > 0 and (gain[u] > gain[v] or (gain[u] == gain[v] and u < v)) for u in nb)
        if not beaten:
            assert Wf[target[v]] + 1 > cap
