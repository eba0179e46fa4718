"""Preconditioners for LOBPCG (oracle; test infrastructure only).

Sec. 5.1, Jacobi: M = diag(A)^{-1}, where A is the operator LOBPCG is applied
to.  For L_C (combinatorial and generalized problems) the diagonal is the
weighted degree; for L_N it is 1, so Jacobi is the identity there.

Sec. 5.2, polynomial: M = p_k(A), the GMRES polynomial (Loe and Morgan), with
default degree 25.  The paper gives no construction; the reading taken here is
the standard one for a symmetric operator:

1. k steps of Lanczos (the symmetric case of Arnoldi) on A from a seeded start
   vector with the null vector of A projected out, with full
   reorthogonalisation (classical Gram-Schmidt, two passes);
2. the roots of the GMRES residual polynomial are the harmonic Ritz values:
   the eigenvalues theta of (T_k^2 + beta_k^2 e_k e_k^T) y = theta T_k y;
2b. definiteness: LOBPCG (Algorithm 1) takes a symmetric positive definite
   preconditioner, and p_k need not be positive on the spectrum:
   1 - lambda p(lambda) = prod_i (1 - lambda/theta_i) can exceed 1 between the
   largest roots, where p < 0 (on the batch workload's 2e5-vertex geometric
   graphs LOBPCG then stalls for thousands of iterations).  While the minimum
   of p over lambda_j = theta_max j / G, j = 1..G (G = DEFINITE_GRID), is not
   positive, a second copy of the root nearest the minimising lambda_j is
   added, at most MAX_INTERIOR_ROOTS times.  Above theta_max every factor is
   negative, so there the product has the sign (-1)^(root count): with an
   even count it grows past 1 before lambda_max (which theta_max can
   underestimate by a percent) and p turns negative; so an even count gets
   one more copy of theta_max, which shrinks the product's magnitude below
   theta_max and makes p positive above it.  Repeating a root is the device
   the GMRES-polynomial papers Sec. 5.2 cites use for stability ("adding
   roots"); here it is triggered by the sign of p, a reading (the paper gives
   no rule);
3. the roots are put in modified Leja order;
4. p is applied in product form, 1 - lambda p(lambda) = prod_i (1 - lambda/theta_i):
   y = 0, t = v; for i = 1..k: y += t / theta_i; if i < k: t -= A t / theta_i,
   which costs k - 1 products with A.

Pins (tests/test_oracle_precond.py): p(A) v against V diag(p(lambda)) V^T v from
a dense eigendecomposition; 1 - theta_i p(theta_i) = 0 at every root; the roots
lie inside the spectrum of A restricted to the complement of its null space;
the definiteness step against p evaluated from its power-basis coefficients on
a finer grid (unchanged roots where p > 0 already, one added root on a stored
indefinite case and on a batch graph); Jacobi against the diagonal of the
explicit Laplacian.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .laplacian import NORMALIZED, weighted_degree, null_vector
from .rng import poly_start_vector


def jacobi_diag(g, problem: str) -> np.ndarray:
    """Inverse diagonal of the operator: 1/deg for L_C, 1 for L_N."""
    if problem == NORMALIZED:
        return np.ones(g.n)
    deg = weighted_degree(g)
    with np.errstate(divide="ignore"):
        return np.where(deg > 0, 1.0 / deg, 1.0)


def leja_order(theta: np.ndarray) -> np.ndarray:
    """Modified Leja ordering: start at the largest |theta|, then repeatedly
    take the root maximising the product of distances to those already taken
    (sum of log distances).  Ties go to the lowest index."""
    theta = np.asarray(theta, dtype=np.float64)
    k = theta.size
    left = list(range(k))
    first = max(left, key=lambda i: (abs(theta[i]), -i))
    order = [first]
    left.remove(first)
    score = np.zeros(k)
    while left:
        last = theta[order[-1]]
        for i in left:
            d = abs(theta[i] - last)
            score[i] += np.log(d) if d > 0 else -np.inf
        best = left[0]
        for i in left[1:]:
            if score[i] > score[best]:
                best = i
        order.append(best)
        left.remove(best)
    return theta[np.array(order)]


def lanczos(apply_a, v0: np.ndarray, k: int):
    """k Lanczos steps with two-pass classical Gram-Schmidt reorthogonalisation.
    Returns (alpha[k], beta[k]) where T_k = tridiag(beta[:k-1], alpha, beta[:k-1])
    and beta[k-1] is the coupling to the next Krylov vector."""
    n = v0.size
    v = v0 / np.linalg.norm(v0)
    basis = np.zeros((n, k))
    alpha = np.zeros(k)
    beta = np.zeros(k)
    for j in range(k):
        basis[:, j] = v
        w = apply_a(v)
        alpha[j] = v @ w
        for _ in range(2):
            w = w - basis[:, : j + 1] @ (basis[:, : j + 1].T @ w)
        beta[j] = np.linalg.norm(w)
        if beta[j] == 0.0:
            return alpha[: j + 1], beta[: j + 1]
        v = w / beta[j]
    return alpha, beta


def harmonic_ritz(alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Eigenvalues of (T^2 + beta_k^2 e_k e_k^T) y = theta T y, via the
    Cholesky factor T = C C^T: theta = eig(C^{-1} (T^2 + b^2 e e^T) C^{-T})."""
    k = alpha.size
    t = np.diag(alpha) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
    m = t @ t
    m[k - 1, k - 1] += beta[k - 1] ** 2
    c = np.linalg.cholesky(t)
    z = sla.solve_triangular(c, m, lower=True)
    z = sla.solve_triangular(c, z.T, lower=True).T
    z = 0.5 * (z + z.T)
    return np.linalg.eigvalsh(z)


DEFINITE_GRID = 8192
MAX_INTERIOR_ROOTS = 4
MAX_ADDED_ROOTS = MAX_INTERIOR_ROOTS + 1   # and the parity copy


def p_on_grid(theta: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """p(lambda) = (1 - prod_i (1 - lambda/theta_i)) / lambda, the factors
    multiplied in the order of theta."""
    pi = np.ones_like(lam)
    for t in theta:
        pi = pi * (1.0 - lam / t)
    return (1.0 - pi) / lam


def definite_roots(theta: np.ndarray) -> np.ndarray:
    """Step 2b of the module notes: theta (ascending harmonic Ritz values),
    followed by the added copies in the order they were added."""
    base = np.asarray(theta, dtype=np.float64)
    roots = list(base)
    lam = (base.max() * np.arange(1, DEFINITE_GRID + 1, dtype=np.float64)) / DEFINITE_GRID
    for _ in range(MAX_INTERIOR_ROOTS):
        p = p_on_grid(np.array(roots), lam)
        m = int(np.argmin(p))                          # lowest j on ties
        if p[m] > 0.0:
            break
        roots.append(base[int(np.argmin(np.abs(base - lam[m])))])   # nearest root, lowest index on ties
    if len(roots) % 2 == 0:
        roots.append(base.max())                       # an odd count: p > 0 above theta_max
    return np.array(roots)


def gmres_poly_roots(g, problem: str, apply_a, degree: int, seed: int) -> np.ndarray:
    """Roots theta_1..theta_k' of the GMRES residual polynomial (k' = degree
    plus the roots step 2b adds), Leja ordered."""
    v = poly_start_vector(g.n, seed)
    z = null_vector(g, problem)
    v = v - (z @ v) / (z @ z) * z
    alpha, beta = lanczos(apply_a, v, degree)
    return leja_order(definite_roots(harmonic_ritz(alpha, beta)))


def poly_apply(apply_a, roots: np.ndarray, v: np.ndarray) -> np.ndarray:
    """y = p(A) v in product form; ``v`` may be a block (n x c)."""
    k = roots.size
    y = np.zeros_like(v, dtype=np.float64)
    t = np.array(v, dtype=np.float64)
    for i in range(k):
        y = y + t / roots[i]
        if i < k - 1:
            t = t - apply_a(t) / roots[i]
    return y
