"""Pins for oracle.precond: Jacobi (Sec. 5.1) and the GMRES polynomial (Sec. 5.2)."""

import numpy as np

import oracle as O
import workloads as W
from oracle.precond import lanczos, harmonic_ritz, leja_order, poly_apply


def _poly_scalar(roots, lam):
    """p(lambda) from the product-form recurrence applied to a 1 x 1 'matrix'."""
    return poly_apply(lambda t: lam * t, roots, np.array([[1.0]]))[0, 0]


def test_jacobi_is_inverse_operator_diagonal():
    g = W.random_edge_weights(W.rmat(9, seed=3))
    for prob in (O.COMBINATORIAL, O.GENERALIZED, O.NORMALIZED):
        lmat = O.operator_for(g, prob).toarray()
        assert np.allclose(O.jacobi_diag(g, prob), 1.0 / np.diag(lmat))


def test_harmonic_ritz_against_nonsymmetric_form():
    g = W.largest_component(W.rmat(8, seed=5))
    lmat = O.laplacian_combinatorial(g)
    v = O.poly_start_vector(g.n, 2)
    v -= v.mean()
    alpha, beta = lanczos(lambda x: lmat @ x, v, 8)
    k = alpha.size
    t = np.diag(alpha) + np.diag(beta[:k - 1], 1) + np.diag(beta[:k - 1], -1)
    ek = np.zeros(k)
    ek[-1] = 1.0
    ns = t + beta[k - 1] ** 2 * np.linalg.solve(t, np.outer(ek, ek))
    ref = np.sort(np.linalg.eigvals(ns).real)
    assert np.allclose(harmonic_ritz(alpha, beta), ref, rtol=1e-9)


def test_poly_roots_zero_residual_polynomial_and_in_spectrum():
    g = W.grid2d(10, 7)
    lmat = O.laplacian_combinatorial(g)
    roots = O.gmres_poly_roots(g, O.COMBINATORIAL, lambda x: lmat @ x, 6, 1)
    ev = np.linalg.eigvalsh(lmat.toarray())
    assert np.all(roots > ev[1] * (1 - 1e-9)) and np.all(roots < ev[-1] * (1 + 1e-9))
    for th in roots:
        assert abs(1.0 - th * _poly_scalar(roots, th)) < 1e-9


def test_poly_apply_matches_spectral_definition():
    g = W.largest_component(W.erdos_renyi(60, 0.1, 9))
    lmat = O.laplacian_normalized(g)
    roots = O.gmres_poly_roots(g, O.NORMALIZED, lambda x: lmat @ x, 5, 4)
    lam, vec = np.linalg.eigh(lmat.toarray())
    pl = np.array([_poly_scalar(roots, x) for x in lam])
    # independent evaluation: 1 - lambda p(lambda) = prod (1 - lambda / theta_i)
    nz = np.abs(lam) > 1e-10
    ref = np.where(nz, (1 - np.prod(1 - lam[:, None] / roots[None, :], axis=1)) / np.where(nz, lam, 1),
                   np.sum(1 / roots))
    assert np.allclose(pl, ref, rtol=1e-9)
    v = np.random.default_rng(0).standard_normal((g.n, 3))
    y = poly_apply(lambda t: lmat @ t, roots, v)
    assert np.allclose(y, vec @ (pl[:, None] * (vec.T @ v)), rtol=1e-9, atol=1e-10)


def test_gmres_polynomial_minimises_krylov_residual():
    """The GMRES residual polynomial pi(A) v, pi(0) = 1, deg <= k, has the
    smallest norm over the Krylov space (Loe-Morgan's definition); compare
    with a least-squares solve on an explicit Krylov basis."""
    g = W.largest_component(W.erdos_renyi(50, 0.12, 2))
    lmat = O.laplacian_combinatorial(g)
    a = lmat.toarray()
    k = 5
    v = O.poly_start_vector(g.n, 7)
    v -= v.mean()
    roots = O.gmres_poly_roots(g, O.COMBINATORIAL, lambda x: lmat @ x, k, 7)
    y = poly_apply(lambda t: a @ t, roots, v[:, None])[:, 0]
    res_poly = np.linalg.norm(v - a @ y)
    kb = np.zeros((g.n, k))
    w = v.copy()
    for j in range(k):
        kb[:, j] = w
        w = a @ w
    q, _ = np.linalg.qr(kb)
    c, *_ = np.linalg.lstsq(a @ q, v, rcond=None)
    res_ls = np.linalg.norm(v - a @ q @ c)
    assert abs(res_poly - res_ls) <= 1e-8 * np.linalg.norm(v)


def test_leja_order():
    th = np.array([0.5, 3.0, 1.0, 2.0, 0.1])
    out = leja_order(th)
    assert out[0] == 3.0
    assert out[1] == 0.1                      # farthest from 3
    assert sorted(out) == sorted(th)


def _harmonic(g, seed, k=25):
    lmat = O.laplacian_combinatorial(g)
    v = O.poly_start_vector(g.n, seed)
    v -= v.mean()
    alpha, beta = lanczos(lambda x: lmat @ x, v, k)
    return harmonic_ritz(alpha, beta)


def _p_applied(roots, lam):
    """p(lambda_j) for every point of lam as LOBPCG applies it: the product-form
    recurrence on the diagonal operator diag(lam)."""
    return poly_apply(lambda t: lam[:, None] * t, roots, np.ones((lam.size, 1)))[:, 0]


def test_definite_roots_leaves_a_positive_polynomial_of_odd_degree_alone():
    th = _harmonic(W.grid2d(16, 16), 1, 13)
    fine = np.linspace(0.0, 1.5 * th.max(), 40001)[1:]
    assert _p_applied(th, fine).min() > 0.0
    assert np.array_equal(O.definite_roots(th), th)


def test_definite_roots_makes_an_even_count_odd():
    """Above the largest root every factor is negative: with an even number of
    roots the product grows past 1 and p < 0 there (a degree-12 polynomial on
    a 16 x 16 grid graph, at 1.5 theta_max); the parity copy of theta_max
    makes p positive above theta_max and keeps it positive below."""
    th = _harmonic(W.grid2d(16, 16), 1, 12)
    fine = np.linspace(0.0, 1.5 * th.max(), 40001)[1:]
    assert _p_applied(th, fine).min() < 0.0
    th2 = O.definite_roots(th)
    assert th2.size == 13 and np.array_equal(th2[:12], th) and th2[12] == th.max()
    assert _p_applied(th2, fine).min() > 0.0


def test_definite_roots_makes_an_indefinite_polynomial_positive():
    """A 1000-vertex geometric graph whose degree-25 GMRES polynomial dips far
    below zero between its largest roots (step 2b of oracle.precond): each
    added root repeats an existing one, the count ends odd, p as applied is
    positive on a grid five times finer than the one the rule scans and
    reaching 1.5 theta_max, and the residual polynomial still vanishes at
    every root."""
    th = _harmonic(W.rgg(1000, seed=11), 27)
    fine = np.linspace(0.0, 1.5 * th.max(), 5 * O.precond.DEFINITE_GRID + 1)[1:]
    assert _p_applied(th, fine).min() < -1.0
    th2 = O.definite_roots(th)
    added = th2[th.size:]
    assert np.array_equal(th2[:th.size], th) and 1 <= added.size <= O.precond.MAX_ADDED_ROOTS
    assert th2.size % 2 == 1
    assert all(np.any(th == r) for r in added)
    assert _p_applied(th2, fine).min() > 0.0
    ordered = leja_order(th2)
    assert np.array_equal(np.sort(ordered), np.sort(th2))
    for r in th2:
        assert abs(1.0 - r * _poly_scalar(ordered, r)) < 1e-8


def test_definite_roots_adds_the_root_nearest_the_minimum():
    """Hand-made roots.  With 0.5, 0.8 and 1, 1 - lambda p lies below 1 on all
    of (0, 1] and the count is odd, so nothing is added.  With 0.05, 0.6 and 1
    the product (1 - 20 lambda)(1 - lambda / 0.6)(1 - lambda) is about
    (-15.5)(-0.375)(0.175) = 1.017 at lambda = 0.825, so p < 0 there; the root
    nearest that point is 1, whose second factor (0.175) brings the product
    under 1; the count is then 4, and the parity copy of 1 makes it 5."""
    assert np.array_equal(O.definite_roots(np.array([0.5, 0.8, 1.0])), [0.5, 0.8, 1.0])
    th = np.array([0.05, 0.6, 1.0])
    lam = np.linspace(0.0, 1.5, 60001)[1:]
    assert _p_applied(th, lam).min() < 0.0
    th2 = O.definite_roots(th)
    assert np.array_equal(th2, [0.05, 0.6, 1.0, 1.0, 1.0])
    assert _p_applied(th2, lam).min() > 0.0
