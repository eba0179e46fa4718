"""Pins for oracle.rng and oracle.sphynx (Algorithm 2 and Eq. 4)."""

import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.rng import mix64, GAMMA

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_outputs():
    ref = [int(line, 16) for line in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
           if line.strip() and not line.startswith("#")]
    assert [mix64(GAMMA * (i + 1)) for i in range(3)] == ref


def test_random_block_layout_and_range():
    x = O.splitmix64_block(5, 3, 42)
    state = mix64(42 + GAMMA)
    z = mix64(state + 4 * GAMMA)          # counter i*b + j + 1 for (1, 0)
    assert x[1, 0] == 2.0 * ((z >> 11) * 2.0 ** -53) - 1.0
    assert np.all(x >= -1.0) and np.all(x < 1.0)


def test_eq4_number_of_eigenvectors():
    assert O.num_eigenvectors(4) == 3       # worked example of Sec. 4
    assert O.num_eigenvectors(24) == 5      # Sec. 6.4: 4 coordinate vectors for K = 24
    assert O.num_eigenvectors(1) == 1
    assert [O.num_eigenvectors(k) for k in (64, 256, 8, 1024)] == [7, 9, 4, 11]


def test_piecewise_initial_block():
    g = W.grid2d(5, 4)
    x = O.initial_block(g, O.COMBINATORIAL, 3, "piecewise", 0)
    assert np.all(x[:, 0] == 1.0)
    assert list(x[:, 1]) == [1.0] * 6 + [0.0] * 14
    assert list(x[:, 2]) == [0.0] * 6 + [1.0] * 7 + [0.0] * 7
    xn = O.initial_block(g, O.NORMALIZED, 3, "piecewise", 0)
    assert np.allclose(xn[:, 0], np.sqrt(O.weighted_degree(g)))


def test_two_cliques_bisect_on_the_bridge():
    a, b = np.triu_indices(8, 1)
    src = np.concatenate([a, a + 8, [7]])
    dst = np.concatenate([b, b + 8, [8]])
    g = W.symmetrize_edges(16, src, dst)
    for prob in (O.COMBINATORIAL, O.GENERALIZED, O.NORMALIZED):
        r = O.partition(g, 2, problem=prob, tol=1e-6, seed=3)
        assert r.cut == 1 and r.imbalance == 1.0
        assert len(set(r.parts[:8])) == 1 and len(set(r.parts[8:])) == 1


def test_rectangular_grid_fiedler_bisection():
    g = W.grid2d(64, 48)
    r = O.partition(g, 2, tol=1e-6, seed=1)
    assert r.status == "ok"
    assert r.cut == 48 and r.imbalance == 1.0


def test_c1_small_grid_partition_quality():
    g = W.grid2d(64, 64)
    r = O.partition(g, 4, problem=O.COMBINATORIAL, precond="jacobi", tol=1e-2, seed=1)
    exact = 2 - 2 * np.cos(np.pi / 64)
    assert r.status == "ok"
    assert np.allclose(r.eigenvalues[1:], exact, rtol=1e-3)
    assert r.imbalance == 1.0
    # lambda_2 = lambda_3: any rotation of the pair is a valid embedding, so
    # only a loose bound holds (two straight cuts give 128)
    assert 128 <= r.cut <= 4 * 64


@pytest.mark.parametrize("prob,pc", [(O.GENERALIZED, "poly"), (O.NORMALIZED, "poly"),
                                     (O.GENERALIZED, "jacobi"), (O.NORMALIZED, "none")])
def test_problem_and_preconditioner_variants_agree_on_spectrum(prob, pc):
    g = W.grid2d(30, 22)
    r = O.partition(g, 8, problem=prob, precond=pc, tol=1e-6, seed=2, poly_degree=8)
    assert r.status == "ok"
    ref = np.linalg.eigvalsh(O.laplacian_normalized(g).toarray())[:4]
    assert np.allclose(r.eigenvalues, ref, rtol=1e-5, atol=1e-12)
    assert r.imbalance == 83 * 8 / 660      # 660 unit vertices into 8 parts: best is 83


def test_reference_block_layout():
    z = O.reference_block(4, 5, 9)
    state = mix64(9 + 5 * GAMMA)
    v = mix64(state + (2 * 5 + 3 + 1) * GAMMA)   # entry (2, 3): counter i*d + j + 1
    assert z[2, 3] == 2.0 * ((v >> 11) * 2.0 ** -53) - 1.0


def test_eigen_clusters():
    th = np.array([0.0, 1.0, 1.0 + 1e-9, 1.0 + 2e-9, 2.0, 3.0, 3.0 * (1 + 5e-4)])
    assert O.eigen_clusters(th, 1e-3) == [(1, 3), (5, 6)]
    assert O.eigen_clusters(th, 1e-4) == [(1, 3)]
    # the eigenvalue-zero column never joins a cluster, even with a zero neighbour
    assert O.eigen_clusters(np.array([0.0, 0.0, 1.0]), 1e-3) == []


def _orthonormal(n, d, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, d)))
    return q


def test_canonical_rotation_depends_on_the_span_only():
    n, d = 300, 7
    e = _orthonormal(n, d, 1)
    th = np.array([0.0, 0.5, 0.5, 0.5, 0.9, 1.3, 1.3])
    rng = np.random.default_rng(2)
    ref = O.canonical_rotation(e, th, 1e-6, seed=4)
    for _ in range(3):
        r = e.copy()
        for a, b in ((1, 3), (5, 6)):
            q, _ = np.linalg.qr(rng.standard_normal((b - a + 1, b - a + 1)))
            r[:, a:b + 1] = r[:, a:b + 1] @ q
        got = O.canonical_rotation(r, th, 1e-6, seed=4)
        assert np.allclose(got, ref, atol=1e-12)
    # columns outside clusters are untouched; the result stays orthonormal and
    # spans the same subspaces
    assert np.array_equal(ref[:, [0, 4]], e[:, [0, 4]])
    assert np.allclose(ref.T @ ref, np.eye(d), atol=1e-12)
    for a, b in ((1, 3), (5, 6)):
        p = e[:, a:b + 1] @ e[:, a:b + 1].T
        assert np.allclose(p @ ref[:, a:b + 1], ref[:, a:b + 1], atol=1e-12)


def test_canonical_rotation_is_the_procrustes_optimum():
    n, d = 200, 4
    e = _orthonormal(n, d, 3)
    th = np.array([0.0, 2.0, 2.0, 2.0])
    got = O.canonical_rotation(e, th, 1e-6, seed=7)
    z = O.reference_block(n, d, 7)[:, 1:4]
    best = np.trace(got[:, 1:4].T @ z)
    rng = np.random.default_rng(5)
    for _ in range(200):
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        assert np.trace((e[:, 1:4] @ q).T @ z) <= best + 1e-12


def test_degenerate_mesh_partition_independent_of_eigenvector_rotation():
    """On a 27-point mesh the eigenvalues come in triples; once the clusters
    are canonically rotated, the multi-jagged parts no longer depend on the
    basis LOBPCG happened to return inside each triple."""
    g = W.grid3d(16, 16, 16, 27)
    res = O.partition(g, 64, problem="generalized", precond="poly", poly_degree=10, tol=1e-3, seed=2)
    clusters = O.eigen_clusters(res.eigenvalues, 1e-3)
    assert clusters == [(1, 3), (4, 6)]
    rng = np.random.default_rng(0)
    for _ in range(2):
        e = res.eigvecs.copy()
        for a, b in clusters:
            q, _ = np.linalg.qr(rng.standard_normal((b - a + 1, b - a + 1)))
            e[:, a:b + 1] = e[:, a:b + 1] @ q
        coords = O.sign_normalise(O.canonical_rotation(e, res.eigenvalues, 1e-3, 2))[:, 1:]
        assert np.array_equal(O.multijagged(np.ascontiguousarray(coords), None, 64), res.parts)


def test_graph_type_and_defaults_follow_the_decision_flow():
    # meshes: max/avg degree near 1 (Sec. 6.1 quotes 1.00 to 4.36 for its regular graphs)
    mesh = W.grid3d(6, 5, 4, 27)
    assert O.is_regular(mesh)
    assert O.default_options(mesh, "jacobi") == dict(problem="combinatorial", tol=1e-3, init="random",
                                                     precond="jacobi")
    assert O.default_options(mesh, "poly")["problem"] == "combinatorial"
    # a star: one vertex adjacent to all others, ratio about n / 2
    star = W.star_graph(100)
    assert not O.is_regular(star)
    assert O.default_options(star, "jacobi") == dict(problem="generalized", tol=1e-2, init="piecewise",
                                                     precond="jacobi")
    assert O.default_options(star, "poly")["problem"] == "normalized"
    # multigrid (MueLu): tol 1e-2 on regular graphs too, the generalized problem on irregular ones
    assert O.default_options(mesh, "amg") == dict(problem="combinatorial", tol=1e-2, init="random", precond="amg")
    assert O.default_options(star, "amg") == dict(problem="generalized", tol=1e-2, init="piecewise",
                                                  precond="amg")
    # the boundary: max degree exactly 10 x average is still regular
    # (star of 11 vertices: max 10, average 20 / 11; ratio 5.5 -> regular)
    assert O.is_regular(W.star_graph(11))
    # 20 vertices: max 19, average 38 / 20, ratio exactly 10 -> regular
    assert O.is_regular(W.star_graph(20))
    # 21 vertices: max 20, average 40 / 21, ratio 10.5 -> irregular
    assert not O.is_regular(W.star_graph(21))
