"""Seeded synthetic graph workloads.

This package only builds inputs: CSR adjacency structures (and optional edge
weights) for regular meshes and power-law / geometric graphs with the structure
classes the paper evaluates (Sec. 6.1, Table 1).  It holds none of the method's
arithmetic (no Laplacian, no eigensolver, no partitioner) and is the one module
shared by the CPU oracle, the tests and the benchmark.
"""

from .graphs import (  # noqa: F401
    CSRGraph,
    path_graph,
    cycle_graph,
    grid2d,
    grid3d,
    star_graph,
    erdos_renyi,
    rmat,
    rgg,
    largest_component,
    symmetrize_edges,
    random_coords,
    random_vertex_weights,
    random_edge_weights,
    concat_graphs,
    rgg_batch,
)
