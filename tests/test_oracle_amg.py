"""Pins of the oracle's aggregation multigrid preconditioner (Sec. 5.3, with the
parameters of Sec. 6.2.2) against breadth-first search, dense linear algebra
and the closed form of the Chebyshev polynomial."""

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.csgraph as csg

import oracle as O
import oracle.amg as A
import workloads as W


def small_graphs():
    return {
        "path": W.path_graph(37),
        "grid": W.grid2d(23, 17),
        "grid27": W.grid3d(9, 8, 7, 27),
        "star": W.star_graph(40),
        "rmat": W.rmat(9, seed=5),
        "weighted": W.random_edge_weights(W.grid2d(15, 14), 0.5, 1.5, 3),
    }


GRAPHS = small_graphs()


def hop_distances(g):
    return csg.shortest_path(O.adjacency(g), unweighted=True, directed=False)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_roots_are_a_maximal_distance_two_independent_set(name):
    g = GRAPHS[name]
    root, rounds = A.mis2_roots(g, seed=3)
    dist = hop_distances(g)
    r = np.flatnonzero(root)
    assert r.size > 0 and rounds >= 1
    sub = dist[np.ix_(r, r)]
    np.fill_diagonal(sub, np.inf)
    assert sub.min() >= 3                               # no two roots within distance 2
    assert dist[:, r].min(axis=1).max() <= 2            # every vertex within distance 2 of a root


@pytest.mark.parametrize("name", list(GRAPHS))
def test_aggregates_partition_the_vertices_into_connected_sets(name):
    g = GRAPHS[name]
    agg, nc = A.aggregate(g, seed=3)
    root, _ = A.mis2_roots(g, seed=3)
    assert nc == root.sum() and agg.min() == 0 and agg.max() == nc - 1
    # aggregate ids follow the roots in vertex order, each root in its own aggregate
    assert np.array_equal(agg[root], np.arange(nc))
    adj = O.adjacency(g)
    for a in range(nc):
        mem = np.flatnonzero(agg == a)
        ncomp, _ = csg.connected_components(adj[mem][:, mem], directed=False)
        assert ncomp == 1
    # phase 1: every neighbour of a root is in the root's aggregate
    dist = hop_distances(g)
    for rr in np.flatnonzero(root):
        assert np.all(agg[dist[rr] == 1] == agg[rr])


def test_phase_two_joins_the_heaviest_neighbour():
    g = GRAPHS["weighted"]
    agg, _ = A.aggregate(g, seed=3)
    root, _ = A.mis2_roots(g, seed=3)
    dist = hop_distances(g)
    near = (dist[:, np.flatnonzero(root)] <= 1).any(axis=1)
    for v in np.flatnonzero(~near):
        lo, hi = g.row_ptr[v], g.row_ptr[v + 1]
        nb, wv = g.col[lo:hi], g.w[lo:hi]
        ok = near[nb]
        best = max(zip(wv[ok], -nb[ok]))                 # heaviest, then smallest id
        assert agg[v] == agg[-best[1]]


@pytest.mark.parametrize("name", list(GRAPHS))
def test_coarse_graph_laplacian_is_the_galerkin_product(name):
    g = GRAPHS[name]
    agg, nc = A.aggregate(g, seed=3)
    gc = A.coarse_graph(g, agg, nc)
    p = np.zeros((g.n, nc))
    p[np.arange(g.n), agg] = 1.0
    l = O.laplacian_combinatorial(g).toarray()
    lc = O.laplacian_combinatorial(gc).toarray()
    assert np.allclose(lc, p.T @ l @ p, rtol=0, atol=1e-12)
    assert np.all(np.diff(gc.row_ptr) >= 0) and np.all(gc.col >= 0)


def test_chebyshev_error_is_the_scaled_chebyshev_polynomial():
    """From x0 = 0 on L x = b with b = L u and L u = mu D u, the Chebyshev
    iterate is (1 - T_3((theta - mu)/delta) / T_3(theta/delta)) u."""
    g = GRAPHS["grid"]
    l = O.laplacian_combinatorial(g)
    deg = O.weighted_degree(g)
    mu, u = sla.eigh(l.toarray(), np.diag(deg))
    lam_max = 1.7
    lam_min = lam_max / 7.0
    theta, delta = 0.5 * (lam_max + lam_min), 0.5 * (lam_max - lam_min)

    def t3(t):
        return 4.0 * t ** 3 - 3.0 * t                   # T_3 in closed form

    x = A.chebyshev(l, 1.0 / deg, lam_max, l @ u)
    factor = 1.0 - t3((theta - mu) / delta) / t3(theta / delta)
    assert np.allclose(x, u * factor[None, :], rtol=0, atol=1e-10)


def test_power_iteration_bounds_the_top_of_the_spectrum():
    for name in ("grid27", "rmat", "weighted", "star"):
        g = GRAPHS[name]
        deg = O.weighted_degree(g)
        mu = sla.eigh(O.laplacian_combinatorial(g).toarray(), np.diag(deg), eigvals_only=True)
        est = A.power_lambda_max(g, 100, seed=1, level=0)
        assert est <= min(A.BOOST * mu[-1], 2.0) + 1e-12
        assert est >= min(0.95 * A.BOOST * mu[-1], 2.0)
        assert A.power_lambda_max(g, 10, seed=1, level=0) <= 2.0


def test_hierarchy_stops_at_the_size_and_level_limits():
    g = W.grid3d(30, 30, 30, 27)
    lv = A.build_hierarchy(g, seed=1)
    assert 2 <= len(lv) <= A.MAX_LEVELS
    assert lv[-1].g.n <= A.COARSE_MAX and all(x.g.n > A.COARSE_MAX for x in lv[:-1])
    for a, b in zip(lv[:-1], lv[1:]):
        assert a.nc == b.g.n and a.agg.size == a.g.n
    assert lv[-1].agg is None


@pytest.mark.parametrize("name", ["grid", "grid27", "rmat", "weighted"])
def test_vcycle_is_symmetric_and_positive_off_the_null_vector(name):
    g = GRAPHS[name]
    levels = A.build_hierarchy(g, seed=2)
    # force at least two levels on these small graphs
    if len(levels) == 1:
        agg, nc = A.aggregate(g, 2, 0)
        levels[0].agg, levels[0].nc = agg, nc
        gc = A.coarse_graph(g, agg, nc)
        deg = O.weighted_degree(gc)
        levels.append(A.Level(gc, O.laplacian_combinatorial(gc), 1.0 / deg, A.power_lambda_max(gc, 100, 2, 1)))
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal((g.n, 3)), rng.standard_normal((g.n, 3))
    mx, my = A.vcycle(levels, x), A.vcycle(levels, y)
    assert np.allclose(x.T @ my, mx.T @ y, rtol=1e-10, atol=1e-12)
    x -= x.mean(axis=0)                                 # off the null vector of L_C
    assert np.all(np.einsum("ij,ij->j", x, A.vcycle(levels, x)) > 0)


def test_lobpcg_with_multigrid_matches_dense_eigenvalues():
    for g, K in ((W.grid2d(30, 20), 8), (W.grid3d(10, 9, 8, 27), 4)):
        r = O.partition(g, K, problem="combinatorial", precond="amg", tol=1e-6, seed=4)
        ref = sla.eigh(O.laplacian_combinatorial(g).toarray(), eigvals_only=True)[:r.eigenvalues.size]
        assert r.status == "ok"
        assert np.allclose(r.eigenvalues[1:], ref[1:], rtol=1e-6)
        rg = O.partition(g, K, problem="generalized", precond="amg", tol=1e-6, seed=4)
        refg = sla.eigh(O.laplacian_combinatorial(g).toarray(), np.diag(O.weighted_degree(g)),
                        eigvals_only=True)[:rg.eigenvalues.size]
        assert np.allclose(rg.eigenvalues[1:], refg[1:], rtol=1e-6)
    with pytest.raises(ValueError):
        O.partition(W.grid2d(8, 8), 4, problem="normalized", precond="amg")
