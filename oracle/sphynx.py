"""Algorithm 2 (Sphynx), end to end in FP64 (oracle; test infrastructure only).

1. L <- createLaplacian(G) for the chosen problem (Sec. 3.2, Sec. 4);
2. d <- floor(log2 K) + 1 (Eq. 4);
3. E <- LOBPCG(L, d) (Algorithm 1), with Jacobi or polynomial preconditioning
   (Sec. 5) and a random or piecewise-constant initial block (Sec. 6.2.1);
4. coords[i, j] <- E[i, j + 1], j = 1..d-1: the first (eigenvalue-zero)
   eigenvector is dropped (Sec. 4);
5. parts <- MJ(coords, weights, K) (Sec. 4).

Readings where the paper is silent: within each cluster of Ritz values
closer than tol the eigenvectors are rotated to their orthogonal Procrustes
alignment with a seeded reference block (canonical_rotation), and then every
eigenvector is sign-normalised (entry of largest magnitude positive, first one
on ties), so that the embedding is a function of the eigen-subspaces only; K = 1 returns part 0 for every vertex
without an eigensolve; the piecewise-constant block puts the null vector
(1, or D^{1/2} 1 for L_N) in column 0 and the indicators of index blocks
[floor(j n / d), floor((j + 1) n / d)), j = 0..d-2, in columns 1..d-1.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from .laplacian import (COMBINATORIAL, GENERALIZED, NORMALIZED, operator_for,
                        b_diag_for, null_vector, weighted_degree)
from .lobpcg import lobpcg, U_FP64
from .mj import multijagged
from .metrics import cutsize, imbalance
from .precond import jacobi_diag, gmres_poly_roots, poly_apply
from .amg import build_hierarchy, vcycle
from .rng import reference_block, splitmix64_block


def is_regular(g) -> bool:
    """Sec. 6.1: a graph is regular when its largest degree is at most 10
    times its average degree (degrees count neighbours)."""
    deg = np.diff(g.row_ptr)
    return int(deg.max()) * g.n <= 10 * int(g.row_ptr[-1])


def default_options(g, precond: str) -> dict:
    """Sphynx's defaults (Sec. 6.3.1, Fig. 2; initial vectors Sec. 6.2.1):
    regular graphs use the combinatorial problem with tol 1e-3 (Jacobi and
    polynomial preconditioners; 1e-2 with multigrid) and random initial
    vectors; irregular graphs use the generalized problem (Jacobi, multigrid)
    or the normalized problem (polynomial), tol 1e-2 and piecewise-constant
    initial vectors."""
    if is_regular(g):
        return dict(problem=COMBINATORIAL, tol=1e-2 if precond == "amg" else 1e-3, init="random", precond=precond)
    return dict(problem=NORMALIZED if precond == "poly" else GENERALIZED, tol=1e-2, init="piecewise",
                precond=precond)


def num_eigenvectors(num_parts: int) -> int:
    """Eq. 4: d = floor(log2 K) + 1."""
    if num_parts < 1:
        raise ValueError("K must be >= 1")
    return int(num_parts).bit_length()


def initial_block(g, problem: str, d: int, init: str, seed: int) -> np.ndarray:
    if init == "random":
        return splitmix64_block(g.n, d, seed)
    if init == "piecewise":
        x = np.zeros((g.n, d))
        x[:, 0] = null_vector(g, problem)
        for j in range(d - 1):
            x[(j * g.n) // d:((j + 1) * g.n) // d, j + 1] = 1.0
        return x
    raise ValueError(init)


def eigen_clusters(theta: np.ndarray, tol: float) -> list:
    """Runs (a, b) of consecutive columns a..b (a >= 1: the eigenvalue-zero
    column is never part of one) whose neighbouring Ritz values differ by at
    most tol relative to the larger; runs of one column are not listed."""
    out = []
    j = 1
    while j < len(theta):
        k = j
        while k + 1 < len(theta) and abs(theta[k + 1] - theta[k]) <= tol * max(abs(theta[k]), abs(theta[k + 1])):
            k += 1
        if k > j:
            out.append((j, k))
        j = k + 1
    return out


def canonical_rotation(e: np.ndarray, theta: np.ndarray, tol: float, seed: int) -> np.ndarray:
    """Fix the basis of every cluster of Ritz values closer than tol.

    Eigenvectors of (nearly) equal eigenvalues are determined only up to a
    rotation within their span, and LOBPCG returns whichever rotation its
    rounding led to; the multi-jagged cuts depend on it (a few percent of the
    cut on the 27-point meshes, whose eigenvalues come in triples).  Within each
    cluster the columns E_c are replaced by E_c Q, Q the orthogonal polar factor
    of E_c^T Z_c: the rotation of the span closest to the seeded reference
    block Z (orthogonal Procrustes).  The result depends on the span only."""
    clusters = eigen_clusters(theta, tol)
    if not clusters:
        return e
    e = e.copy()
    z = reference_block(e.shape[0], e.shape[1], seed)
    for a, b in clusters:
        m = e[:, a:b + 1].T @ z[:, a:b + 1]
        u, _, vt = np.linalg.svd(m)
        e[:, a:b + 1] = e[:, a:b + 1] @ (u @ vt)
    return e


def sign_normalise(x: np.ndarray) -> np.ndarray:
    idx = np.argmax(np.abs(x), axis=0)
    s = np.sign(x[idx, np.arange(x.shape[1])])
    s[s == 0] = 1.0
    return x * s


def gershgorin_rho(g, problem: str) -> float:
    if problem == COMBINATORIAL:
        return 2.0 * float(weighted_degree(g).max())
    return 2.0


def max_row_terms(g) -> int:
    """Most terms a row of the Laplacian adds up: max degree + 1."""
    return int(np.diff(g.row_ptr).max()) + 1 if g.n else 1


@dataclasses.dataclass
class PartitionResult:
    parts: np.ndarray
    cut: float
    cut_twice: float
    imbalance: float
    eigenvalues: np.ndarray
    resnorm: np.ndarray
    iterations: int
    status: str
    coords: np.ndarray
    eigvecs: np.ndarray
    roots: np.ndarray


def partition(g, num_parts: int, problem: str = COMBINATORIAL, precond: str = "jacobi",
              tol: float = 1e-3, maxit: int = 1000, init: str = "random", seed: int = 1,
              poly_degree: int = 25, vwts=None, u_work: float = U_FP64, conv: str = "rel_theta",
              on_iteration=None) -> PartitionResult:
    """K-way partition of g by Algorithm 2."""
    if num_parts == 1:
        z = np.zeros(g.n, dtype=np.int32)
        return PartitionResult(z, 0.0, 0.0, 1.0, np.zeros(0), np.zeros(0), 0, "ok",
                               np.zeros((g.n, 0)), np.zeros((g.n, 0)), np.zeros(0))
    lmat = operator_for(g, problem)

    def apply_l(v):
        return lmat @ v

    bdiag = b_diag_for(g, problem)
    d = num_eigenvectors(num_parts)
    roots = np.zeros(0)
    if precond == "jacobi":
        jd = jacobi_diag(g, problem)

        def apply_m(r):
            return jd[:, None] * r
    elif precond == "poly":
        roots = gmres_poly_roots(g, problem, apply_l, poly_degree, seed)

        def apply_m(r):
            return poly_apply(apply_l, roots, r)
    elif precond == "amg":
        if problem == NORMALIZED:
            raise ValueError("the multigrid preconditioner approximates L_C^{-1}: combinatorial or generalized only")
        levels = build_hierarchy(g, seed)

        def apply_m(r):
            return vcycle(levels, r)
    elif precond == "none":
        apply_m = None
    else:
        raise ValueError(precond)
    x0 = initial_block(g, problem, d, init, seed)
    res = lobpcg(apply_l, bdiag, apply_m, x0, tol, maxit, gershgorin_rho(g, problem), u_work, max_row_terms(g),
                 conv, on_iteration)
    e = sign_normalise(canonical_rotation(res.x, res.theta, tol, seed))
    coords = np.ascontiguousarray(e[:, 1:d])
    parts = multijagged(coords, vwts, num_parts)
    cut, cut2 = cutsize(g, parts)
    return PartitionResult(parts, cut, cut2, imbalance(parts, vwts, num_parts), res.theta,
                           res.resnorm, res.iterations, res.status, coords, e, roots)
