"""Pins for oracle.lobpcg (Algorithm 1) and its Rayleigh-Ritz step."""

import numpy as np
import scipy.linalg as sla

import oracle as O
import workloads as W
from oracle.lobpcg import lobpcg, rayleigh_ritz, residual_norms


def _run(g, problem, nev, tol=1e-8, precond="jacobi", maxit=3000, seed=3):
    lmat = O.operator_for(g, problem)
    bd = O.b_diag_for(g, problem)
    jd = O.jacobi_diag(g, problem)
    m = (lambda r: jd[:, None] * r) if precond == "jacobi" else None
    x0 = O.splitmix64_block(g.n, nev, seed)
    rho = 2.0 * O.weighted_degree(g).max() if problem == O.COMBINATORIAL else 2.0
    return lobpcg(lambda v: lmat @ v, bd, m, x0, tol, maxit, rho), lmat, bd


def test_rayleigh_ritz_matches_generalized_eigh():
    rng = np.random.default_rng(0)
    n, m = 200, 9
    a = rng.standard_normal((n, n))
    a = a @ a.T
    bd = rng.uniform(1, 3, n)
    s = rng.standard_normal((n, m))
    ga, gb = s.T @ a @ s, s.T @ (bd[:, None] * s)
    th, y, svqb = rayleigh_ritz(ga, gb, 4)
    ref = sla.eigh(ga, gb, eigvals_only=True)[:4]
    assert not svqb
    assert np.allclose(th, ref, rtol=1e-10)
    assert np.allclose(y.T @ gb @ y, np.eye(4), atol=1e-10)
    assert np.allclose(y.T @ ga @ y, np.diag(th), atol=1e-8)


def test_rayleigh_ritz_rank_deficient_basis_takes_svqb():
    rng = np.random.default_rng(1)
    n = 100
    a = np.diag(np.arange(1.0, n + 1))
    s = rng.standard_normal((n, 5))
    s = np.concatenate([s, s[:, :2] * 3.0], axis=1)  # two dependent columns
    th, y, svqb = rayleigh_ritz(s.T @ a @ s, s.T @ s, 3)
    assert svqb
    q, _ = np.linalg.qr(s[:, :5])
    ref = np.linalg.eigvalsh(q.T @ a @ q)[:3]
    assert np.allclose(th, ref, rtol=1e-10)


def test_path_spectrum_closed_form():
    n, nev = 120, 4
    res, lmat, _ = _run(W.path_graph(n), O.COMBINATORIAL, nev, tol=1e-9)
    exact = 2 - 2 * np.cos(np.pi * np.arange(nev) / n)
    assert res.status == "ok"
    # Bauer-Fike for a symmetric matrix and unit x: |theta - lambda| <= ||r||
    assert np.all(np.abs(res.theta - exact) <= res.resnorm + 1e-14)
    assert np.allclose(res.theta, exact, rtol=1e-8, atol=1e-14)


def test_grid_nondegenerate_matches_dense_eigh_and_subspace():
    g = W.grid2d(17, 11)
    nev = 5
    res, lmat, _ = _run(g, O.COMBINATORIAL, nev, tol=1e-10)
    ev, vec = np.linalg.eigh(lmat.toarray())
    assert np.allclose(res.theta, ev[:nev], rtol=1e-9, atol=1e-13)
    # principal angles between span(X) and the exact eigenvectors
    q, _ = np.linalg.qr(res.x)
    cosines = np.linalg.svd(vec[:, :nev].T @ q, compute_uv=False)
    assert np.all(cosines > 1 - 1e-8)


def test_generalized_problem_matches_dense_and_is_b_orthonormal():
    g = W.largest_component(W.rmat(8, seed=11))
    nev = 4
    res, lmat, bd = _run(g, O.GENERALIZED, nev, tol=1e-9)
    ref = sla.eigh(lmat.toarray(), np.diag(bd), eigvals_only=True)[:nev]
    assert res.status == "ok"
    assert np.allclose(res.theta, ref, rtol=1e-7, atol=1e-12)
    assert np.allclose(res.x.T @ (bd[:, None] * res.x), np.eye(nev), atol=1e-10)
    r = lmat @ res.x - bd[:, None] * res.x * res.theta[None, :]
    assert np.allclose(residual_norms(r, bd), res.resnorm, rtol=1e-6, atol=1e-14)


def test_normalized_problem_star_graph():
    g = W.star_graph(40)
    res, lmat, _ = _run(g, O.NORMALIZED, 3, tol=1e-9, precond=None)
    # star: normalized spectrum is {0, 1 (multiplicity n-2), 2}
    assert np.allclose(res.theta, [0.0, 1.0, 1.0], atol=1e-9)


def test_convergence_test_uses_relative_theta_and_floor():
    g = W.grid2d(12, 9)
    res, lmat, _ = _run(g, O.COMBINATORIAL, 3, tol=1e-2)
    floor = 10 * 2.0 ** -53 * 2 * 4
    ok = (res.resnorm <= 1e-2 * np.abs(res.theta)) | ((np.abs(res.theta) <= floor) & (res.resnorm <= floor))
    assert ok.all()
    assert res.resnorm[0] <= floor and abs(res.theta[0]) <= floor  # the null vector converges on the floor
    # every other column meets the relative test itself
    assert np.all(res.resnorm[1:] <= 1e-2 * np.abs(res.theta[1:]))


def test_null_vector_rounding_grows_with_row_terms():
    """The exact eigenvalue-zero vector of L_N, multiplied out in FP64, leaves a
    residual that grows with the entries of the longest row (the hub of a
    star): above 10 u rho already at 999 leaves, and inside the residual floor
    10 u rho (d_max + 1) at every size."""
    u = 2.0 ** -53
    for nv in (1000, 20000):
        g = W.star_graph(nv)                 # a hub joined to nv - 1 leaves
        lmat = O.operator_for(g, O.NORMALIZED)
        x = np.sqrt(O.weighted_degree(g))
        x /= np.linalg.norm(x)
        r = np.linalg.norm(lmat @ x)
        assert O.max_row_terms(g) == nv
        assert r > 10 * u * 2.0
        assert r <= 10 * u * 2.0 * O.max_row_terms(g)


def test_hub_graph_converges_and_floor_admits_only_theta_zero():
    """On an R-MAT graph with hub rows the FP64 solve converges: the null vector
    on the residual floor, every other column on its relative test."""
    g = W.largest_component(W.rmat(12, seed=7))
    assert O.max_row_terms(g) > 200
    res = O.partition(g, 8, problem=O.NORMALIZED, precond="jacobi", tol=1e-3, seed=1)
    assert res.status == "ok"
    floor_th = 10 * 2.0 ** -53 * 2.0
    assert abs(res.eigenvalues[0]) <= floor_th
    assert np.all(res.resnorm[1:] <= 1e-3 * np.abs(res.eigenvalues[1:]))


def test_absolute_convergence_test_meets_its_bound_and_orders_the_iteration_counts():
    """conv="abs" stops at ||r_i||_{B^-1} <= tol.  On a grid whose wanted
    eigenvalues are all below 1, that bound is looser than tol |theta_i|, so
    the absolute test stops no later than the relative one; every returned
    residual meets its own test, and Bauer-Fike still bounds each eigenvalue's
    error by its residual (dense eigh as the reference)."""
    g = W.grid2d(23, 19)
    lmat = O.operator_for(g, O.COMBINATORIAL)
    exact = np.linalg.eigvalsh(lmat.toarray())[:4]
    x0 = O.splitmix64_block(g.n, 4, 3)
    rho = 2.0 * O.weighted_degree(g).max()
    jd = O.jacobi_diag(g, O.COMBINATORIAL)
    m = lambda r: jd[:, None] * r  # noqa: E731
    tol = 1e-4
    rel = lobpcg(lambda v: lmat @ v, None, m, x0, tol, 3000, rho, conv="rel_theta")
    ab = lobpcg(lambda v: lmat @ v, None, m, x0, tol, 3000, rho, conv="abs")
    assert rel.status == "ok" and ab.status == "ok"
    assert np.all(exact < 1.0)
    assert ab.iterations <= rel.iterations
    assert np.all(ab.resnorm <= tol)
    ok_rel = (rel.resnorm[1:] <= tol * np.abs(rel.theta[1:]))
    assert np.all(ok_rel)
    assert np.all(np.abs(ab.theta - exact) <= ab.resnorm + 1e-14)
    # the absolute test with tol below every |theta| * tol_rel stops later
    tight = lobpcg(lambda v: lmat @ v, None, m, x0, tol * 1e-3, 3000, rho, conv="abs")
    assert tight.iterations >= ab.iterations and np.all(tight.resnorm <= tol * 1e-3)
