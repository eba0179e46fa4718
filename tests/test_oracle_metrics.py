"""Pins for oracle.metrics: Eq. 1 cutsize and the imbalance of Sec. 3.1."""

from fractions import Fraction

import numpy as np

import oracle as O
import workloads as W


def test_cut_brute_force_and_quadratic_form():
    g = W.largest_component(W.rmat(9, seed=8))
    parts = (np.arange(g.n) * 7919 % 5).astype(np.int32)
    cut, twice = O.cutsize(g, parts)
    edges = set()
    rows = g.rows()
    for i, j in zip(rows, g.col):
        if i < j:
            edges.add((int(i), int(j)))
    brute = sum(1 for i, j in edges if parts[i] != parts[j])
    assert cut == brute and twice == 2 * brute
    # Sec. 3.2: for x in {-1, +1}^n, cut = x^T L_C x / 4
    x = np.where(parts % 2 == 0, 1.0, -1.0)
    cut2, _ = O.cutsize(g, (parts % 2).astype(np.int32))
    lc = O.laplacian_combinatorial(g)
    assert abs(x @ (lc @ x) / 4 - cut2) < 1e-9


def test_weighted_cut_is_exact():
    g = W.random_edge_weights(W.grid2d(30, 20), 0.5, 1.5, seed=3)
    parts = (np.arange(g.n) % 3).astype(np.int32)
    cut, twice = O.cutsize(g, parts)
    rows = g.rows()
    exact = Fraction(0)
    for i, j, w in zip(rows, g.col, g.w):
        if i < j and parts[i] != parts[j]:
            exact += Fraction(float(w))
    assert cut == float(exact)
    assert twice == float(2 * exact)


def test_imbalance_definition():
    parts = np.array([0, 0, 0, 1, 2, 2], dtype=np.int32)
    assert O.imbalance(parts, None, 3) == 3 * 3 / 6
    w = np.array([1, 2, 3, 4, 5, 6])
    assert list(O.part_weights(parts, w, 3)) == [6, 4, 11]
    assert O.imbalance(parts, w, 3) == 11 * 3 / 21
