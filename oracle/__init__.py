"""FP64 CPU oracle for the Sphynx hot path (test infrastructure only).

This package is the independent, slow, obviously-correct restatement of what
the GPU path computes.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product library never
calls into it and shares no code, constants or helpers with it.

Modules and the parts of the paper they follow:

* ``laplacian``  Eqs. 2 and 3 (combinatorial and normalized Laplacians), the
  weighted rule of Sec. 3.2 and the generalized problem L_C x = lambda D x.
* ``rng``        the seeded initial block and the polynomial start vector
  (SplitMix64, counter based; the paper leaves the distribution open).
* ``precond``    Jacobi (Sec. 5.1) and the GMRES polynomial preconditioner
  (Sec. 5.2): Lanczos, harmonic Ritz values, Leja order, product form.
* ``amg``        the aggregation multigrid preconditioner of Sec. 5.3 with the
  parameters of Sec. 6.2.2 (Chebyshev smoothing, plain aggregation).
* ``lobpcg``     Algorithm 1 (LOBPCG with Rayleigh-Ritz and soft locking),
  generalized to a diagonal B.
* ``mj``         the multi-jagged multisection of Sec. 4 with an exact,
  integer split rule.
* ``metrics``    cutsize (Eq. 1) and imbalance (Sec. 3.1).
* ``refine``     the greedy cut refinement Sec. 7 proposes as future work, in
  the library's parallel, balance-constrained reading.
* ``sphynx``     Algorithm 2, the whole partitioner.

Pins: every function is checked in ``tests/test_oracle_*.py`` against closed
forms, invariants, dense eigendecompositions and brute force; see the header
of each module for its pins.
"""

from .laplacian import (  # noqa: F401
    COMBINATORIAL, GENERALIZED, NORMALIZED,
    adjacency, weighted_degree, laplacian_combinatorial, laplacian_normalized,
    operator_for, b_diag_for, null_vector,
)
from .rng import splitmix64_block, poly_start_vector, reference_block  # noqa: F401
from .precond import jacobi_diag, gmres_poly_roots, poly_apply, leja_order, definite_roots, p_on_grid  # noqa: F401
from .lobpcg import lobpcg, rayleigh_ritz, LobpcgResult  # noqa: F401
from .amg import (aggregate, mis2_roots, coarse_graph, build_hierarchy, vcycle, chebyshev,  # noqa: F401
                  power_lambda_max, vertex_keys)
from .mj import multijagged, coord_sort_key  # noqa: F401
from .metrics import cutsize, imbalance, part_weights  # noqa: F401
from .refine import refine, vertex_gains, capacity, integer_weights  # noqa: F401
from .sphynx import (partition, num_eigenvectors, initial_block, canonical_rotation, eigen_clusters,  # noqa: F401
                     sign_normalise, is_regular, default_options, gershgorin_rho, max_row_terms)
