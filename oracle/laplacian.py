"""Graph Laplacians, explicit and in FP64 (oracle; test infrastructure only).

Follows Sec. 3.2 of the paper:

* Eq. 2, combinatorial Laplacian L_C = D - A: diagonal deg(v_i), off-diagonal
  -1 on every edge.
* Eq. 3, normalized Laplacian L_N = I - D^{-1/2} A D^{-1/2}.
* Weighted graphs: off-diagonal entries are the negated edge weights and the
  diagonal is the sum of incident edge weights (Sec. 3.2, last paragraph).
* Generalized problem: L_C x = lambda D x, i.e. operator L_C with B = D.

Self-loops are not part of the Laplacian (Eqs. 2-3 define off-diagonal entries
for i != j only); the input CSR carries none.

Pins (tests/test_oracle_laplacian.py): zero row sums of L_C, unit diagonal of
L_N, symmetry, the null vectors 1 and D^{1/2} 1, path / cycle / grid spectra
in closed form, the Brick3D structure counts of Table 1.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

COMBINATORIAL = "combinatorial"
GENERALIZED = "generalized"
NORMALIZED = "normalized"


def adjacency(g) -> sp.csr_matrix:
    """Weighted adjacency A (FP64); unit weights when the graph has none."""
    data = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    return sp.csr_matrix((data, g.col.astype(np.int64), g.row_ptr), shape=(g.n, g.n))


def weighted_degree(g) -> np.ndarray:
    """deg(v_i) = sum of incident edge weights (number of neighbours when unweighted)."""
    return np.asarray(adjacency(g).sum(axis=1)).ravel()


def laplacian_combinatorial(g) -> sp.csr_matrix:
    """Eq. 2 (weighted form): L_C = D - A."""
    a = adjacency(g)
    return (sp.diags(weighted_degree(g)) - a).tocsr()


def laplacian_normalized(g) -> sp.csr_matrix:
    """Eq. 3 (weighted form): L_N = I - D^{-1/2} A D^{-1/2}."""
    deg = weighted_degree(g)
    if np.any(deg <= 0):
        raise ValueError("normalized Laplacian needs every vertex to have an edge")
    s = sp.diags(1.0 / np.sqrt(deg))
    return (sp.identity(g.n) - s @ adjacency(g) @ s).tocsr()


def operator_for(g, problem: str) -> sp.csr_matrix:
    """The matrix LOBPCG is applied to: L_C for the combinatorial and the
    generalized problems, L_N for the normalized one (Sec. 4, the first step of Algorithm 2)."""
    if problem in (COMBINATORIAL, GENERALIZED):
        return laplacian_combinatorial(g)
    if problem == NORMALIZED:
        return laplacian_normalized(g)
    raise ValueError(problem)


def b_diag_for(g, problem: str):
    """Diagonal of B in L x = lambda B x: D for the generalized problem, None (B = I) otherwise."""
    if problem == GENERALIZED:
        deg = weighted_degree(g)
        if np.any(deg <= 0):
            raise ValueError("generalized problem needs every vertex to have an edge")
        return deg
    return None


def null_vector(g, problem: str) -> np.ndarray:
    """Eigenvector of eigenvalue zero: the constant vector for L_C (and the
    generalized problem), D^{1/2} 1 for L_N (Sec. 3.2)."""
    if problem == NORMALIZED:
        return np.sqrt(weighted_degree(g))
    return np.ones(g.n)
