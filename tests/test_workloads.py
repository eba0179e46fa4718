"""The native generator helpers (workloads/_gen.c) build the same graphs as
the numpy reference code, bit for bit, and the generators' structural
promises hold (symmetric, sorted, no duplicates, no self-loops)."""

import numpy as np
import pytest

import workloads as W
from workloads import _native


def _same(g, h):
    assert g.n == h.n
    assert np.array_equal(g.row_ptr, h.row_ptr)
    assert np.array_equal(g.col, h.col)
    if g.w is None:
        assert h.w is None
    else:
        assert np.array_equal(g.w, h.w)


def _simple_undirected(g):
    r = g.rows()
    c = g.col.astype(np.int64)
    assert np.all(r != c)
    # sorted and distinct within each row
    same_row = r[1:] == r[:-1]
    assert np.all(c[1:][same_row] > c[:-1][same_row])
    # symmetric
    fwd = np.sort(r * g.n + c)
    bwd = np.sort(c * g.n + r)
    assert np.array_equal(fwd, bwd)


@pytest.fixture(scope="module")
def native():
    L = _native.lib()
    if L is None:
        pytest.skip("no C compiler for the native generator helpers")
    return L


@pytest.mark.parametrize("scale,seed,lcc", [(10, 7, False), (12, 3, True), (13, 11, True)])
def test_native_rmat_matches_numpy(native, scale, seed, lcc):
    g = W.rmat(scale, seed=seed, lcc=lcc, native=False)
    h = W.rmat(scale, seed=seed, lcc=lcc, native=True)
    _same(g, h)
    _simple_undirected(h)


def test_native_largest_component_matches_numpy(native):
    # several components of equal size: the one with the smallest vertex wins
    parts = [W.grid2d(5, 4), W.grid2d(4, 5), W.path_graph(3)]
    n = sum(p.n for p in parts)
    src, dst, off = [], [], 0
    for p in parts:
        r = p.rows() + off
        src.append(r)
        dst.append(p.col.astype(np.int64) + off)
        off += p.n
    g = W.symmetrize_edges(n, np.concatenate(src), np.concatenate(dst))
    _same(W.largest_component(g, native=False), W.largest_component(g, native=True))
    gw = W.random_edge_weights(W.rmat(11, seed=5, lcc=False, native=False), native=False)
    _same(W.largest_component(gw, native=False), W.largest_component(gw, native=True))


def test_native_edge_weights_match_numpy(native):
    g = W.rmat(12, seed=9, native=False)
    _same(W.random_edge_weights(g, 0.5, 1.5, 5, native=False), W.random_edge_weights(g, 0.5, 1.5, 5, native=True))


@pytest.mark.parametrize("n,seed", [(500, 4), (3000, 17), (20000, 5)])
def test_native_rgg_matches_numpy(native, n, seed):
    g = W.rgg(n, seed=seed, native=False)
    h = W.rgg(n, seed=seed, native=True)
    _same(g, h)
    _simple_undirected(h)
