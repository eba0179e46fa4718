"""Pins for oracle.laplacian and for the mesh generator's structure.

Everything here is fixed by the paper (Table 1 counts, Eqs. 2-3) or by
mathematics (closed-form spectra of paths, cycles and grids; null vectors).
"""

import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brick27_offdiag(m: int) -> int:
    """Off-diagonal entries of the m^3 27-point mesh: ordered pairs along
    1, 2 and 3 axes (6, 12 and 8 neighbour directions)."""
    return 6 * (m - 1) * m * m + 12 * (m - 1) ** 2 * m + 8 * (m - 1) ** 3


def test_brick3d_formula_matches_generator_small():
    for m in (2, 3, 4, 7):
        g = W.grid3d(m, m, m, 27)
        assert g.nnz == brick27_offdiag(m)


def test_brick3d_table1_counts():
    rows = [list(map(int, line.split())) for line in open(os.path.join(GOLDEN, "brick3d_table1.txt"))
            if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for m, nv, nedges, maxdeg, avgdeg in rows:
        assert m ** 3 == nv
        assert brick27_offdiag(m) + nv == nedges
        assert maxdeg == 27  # 26 neighbours + the diagonal of A + A^T + I
        assert abs((brick27_offdiag(m) + nv) / nv - avgdeg) < 0.6
    g = W.grid3d(100, 100, 100, 27)
    assert g.nnz + g.n == rows[0][2]
    assert g.degrees().max() + 1 == rows[0][3]


def test_generator_structure_is_simple_and_symmetric():
    for g in (W.grid2d(7, 5), W.grid3d(4, 5, 3, 27), W.grid3d(3, 4, 5, 7, periodic=True),
              W.rmat(9, seed=7), W.erdos_renyi(60, 0.1, 3), W.star_graph(20)):
        a = O.adjacency(g).toarray()
        assert np.allclose(a, a.T)
        assert np.all(np.diag(a) == 0)
        rows = g.rows()
        same = rows[1:] == rows[:-1]
        assert np.all(np.diff(g.col.astype(np.int64))[same] > 0)


def test_combinatorial_rows_sum_to_zero_and_diag_is_degree():
    g = W.random_edge_weights(W.rmat(10, seed=2))
    lc = O.laplacian_combinatorial(g).toarray()
    assert np.allclose(lc.sum(axis=1), 0.0, atol=1e-12)
    a = O.adjacency(g).toarray()
    assert np.allclose(np.diag(lc), a.sum(axis=1))
    off = lc - np.diag(np.diag(lc))
    assert np.allclose(off, -a)
    assert np.allclose(lc, lc.T)


def test_normalized_unit_diagonal_and_null_vector():
    g = W.rmat(10, seed=4)
    ln = O.laplacian_normalized(g).toarray()
    assert np.allclose(np.diag(ln), 1.0)
    z = O.null_vector(g, O.NORMALIZED)
    assert np.allclose(ln @ z, 0.0, atol=1e-12)
    deg = O.weighted_degree(g)
    rows, cols = np.nonzero(O.adjacency(g).toarray())
    assert np.allclose(ln[rows, cols], -1.0 / np.sqrt(deg[rows] * deg[cols]))
    lc = O.laplacian_combinatorial(g)
    assert np.allclose(lc @ O.null_vector(g, O.COMBINATORIAL), 0.0)


def test_path_and_cycle_spectra():
    n = 37
    ev = np.linalg.eigvalsh(O.laplacian_combinatorial(W.path_graph(n)).toarray())
    k = np.arange(n)
    assert np.allclose(ev, np.sort(2 - 2 * np.cos(np.pi * k / n)), atol=1e-12)
    ev = np.linalg.eigvalsh(O.laplacian_combinatorial(W.cycle_graph(n)).toarray())
    assert np.allclose(ev, np.sort(2 - 2 * np.cos(2 * np.pi * k / n)), atol=1e-12)


def test_grid_spectra_are_kronecker_sums():
    nx, ny = 9, 6
    ev = np.linalg.eigvalsh(O.laplacian_combinatorial(W.grid2d(nx, ny)).toarray())
    px = 2 - 2 * np.cos(np.pi * np.arange(nx) / nx)
    py = 2 - 2 * np.cos(np.pi * np.arange(ny) / ny)
    assert np.allclose(ev, np.sort((px[:, None] + py[None, :]).ravel()), atol=1e-12)
    g = W.grid3d(4, 3, 5, 7)
    ev = np.linalg.eigvalsh(O.laplacian_combinatorial(g).toarray())
    p = [2 - 2 * np.cos(np.pi * np.arange(m) / m) for m in (4, 3, 5)]
    ks = (p[0][:, None, None] + p[1][None, :, None] + p[2][None, None, :]).ravel()
    assert np.allclose(ev, np.sort(ks), atol=1e-12)


def test_periodic_27_point_torus_spectrum():
    m = 5
    g = W.grid3d(m, m, m, 27, periodic=True)
    ev = np.linalg.eigvalsh(O.laplacian_combinatorial(g).toarray())
    c = 1 + 2 * np.cos(2 * np.pi * np.arange(m) / m)
    prod = (c[:, None, None] * c[None, :, None] * c[None, None, :]).ravel()
    assert np.allclose(ev, np.sort(26 - (prod - 1)), atol=1e-10)


def test_normalized_spectrum_bounds_and_bipartite_top():
    ev_even = np.linalg.eigvalsh(O.laplacian_normalized(W.cycle_graph(12)).toarray())
    ev_odd = np.linalg.eigvalsh(O.laplacian_normalized(W.cycle_graph(13)).toarray())
    assert ev_even.min() > -1e-12 and ev_even.max() < 2 + 1e-12
    assert abs(ev_even.max() - 2.0) < 1e-12          # bipartite
    assert ev_odd.max() < 2.0 - 1e-3                 # not bipartite


def test_generalized_equals_normalized_spectrum():
    import scipy.linalg as sla
    g = W.erdos_renyi(80, 0.08, 5)
    g = W.largest_component(g)
    lc = O.laplacian_combinatorial(g).toarray()
    d = O.b_diag_for(g, O.GENERALIZED)
    ev_gen = sla.eigh(lc, np.diag(d), eigvals_only=True)
    ev_norm = np.linalg.eigvalsh(O.laplacian_normalized(g).toarray())
    assert np.allclose(ev_gen, ev_norm, atol=1e-10)


def test_generalized_requires_positive_degrees():
    g = W.symmetrize_edges(4, np.array([0]), np.array([1]))
    with pytest.raises(ValueError):
        O.b_diag_for(g, O.GENERALIZED)
