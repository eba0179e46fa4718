"""End-to-end GPU partitions (Algorithm 2) against the FP64 oracle."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import torch_mod

pytestmark = pytest.mark.gpu


def _gpu_partition(g, K, **kw):
    import paper_2105_00578_gb300 as spx
    graph = spx.Graph(g, validate=True)
    try:
        return graph.partition(K, **kw)
    finally:
        graph.close()


def test_c1_grid_64x64_fp64_jacobi():
    """2D 5-point 64x64 mesh, combinatorial, Jacobi, K = 4, tol 1e-2, FP64."""
    g = W.grid2d(64, 64)
    ref = O.partition(g, 4, problem="combinatorial", precond="jacobi", tol=1e-2, seed=1)
    parts, cut, imb, st, code = _gpu_partition(g, 4, laplacian="combinatorial", precond="jacobi",
                                               precision="fp64", tol=1e-2, seed=1)
    assert code == 0
    exact = 2 - 2 * np.cos(np.pi / 64)
    assert np.allclose(st["eigenvalues"][1:], ref.eigenvalues[1:], rtol=1e-6)
    assert np.allclose(st["eigenvalues"][1:], exact, rtol=1e-3)
    # the partition's metrics are the oracle's metrics of the same part ids
    c, c2 = O.cutsize(g, parts)
    assert cut == c and imb == O.imbalance(parts, None, 4) == 1.0
    assert all(r <= 1e-2 * t or r < 1e-12 for r, t in zip(st["resnorm"], st["eigenvalues"]))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nondegenerate_grid_cut_within_two_percent(precision):
    g = W.grid2d(64, 48)
    ref = O.partition(g, 4, problem="combinatorial", precond="jacobi", tol=1e-3, seed=1)
    parts, cut, imb, st, code = _gpu_partition(g, 4, laplacian="combinatorial", precond="jacobi",
                                               precision=precision, tol=1e-3, seed=1)
    assert code == 0
    rtol = 1e-6 if precision == "fp64" else 1e-3
    assert np.allclose(st["eigenvalues"][1:], ref.eigenvalues[1:], rtol=rtol)
    assert abs(cut - ref.cut) <= 0.02 * ref.cut
    assert imb == ref.imbalance


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed_bf16"])
def test_small_27_point_generalized_poly(precision):
    """Scaled-down 27-point mesh (box 24 x 20 x 16), generalized problem,
    polynomial preconditioner of degree 25, K = 64, tol 1e-3."""
    g = W.grid3d(24, 20, 16, 27)
    ref = O.partition(g, 64, problem="generalized", precond="poly", poly_degree=25, tol=1e-3, seed=2)
    parts, cut, imb, st, code = _gpu_partition(g, 64, laplacian="generalized", precond="poly", poly_degree=25,
                                               precision=precision, tol=1e-3, seed=2)
    assert code == 0
    rtol = 1e-6 if precision == "fp64" else 1e-3
    assert np.allclose(st["eigenvalues"][1:], ref.eigenvalues[1:], rtol=rtol)
    assert abs(cut - ref.cut) <= 0.02 * ref.cut
    assert imb <= ref.imbalance + 1e-12
    c, _ = O.cutsize(g, parts)
    assert c == cut


def test_rmat_normalized_jacobi_fp32():
    g = W.rmat(12, seed=3)
    ref = O.partition(g, 16, problem="normalized", precond="jacobi", tol=1e-2, seed=3)
    parts, cut, imb, st, code = _gpu_partition(g, 16, laplacian="normalized", precond="jacobi",
                                               precision="fp32", tol=1e-2, seed=3)
    assert code == 0
    assert np.allclose(st["eigenvalues"][1:], ref.eigenvalues[1:], rtol=1e-3)
    assert O.cutsize(g, parts)[0] == cut
    assert imb == O.imbalance(parts, None, 16)


def test_weighted_piecewise_init_and_vertex_weights():
    import paper_2105_00578_gb300 as spx
    g = W.random_edge_weights(W.largest_component(W.rmat(10, seed=8)), 0.5, 1.5, 9)
    vw = W.random_vertex_weights(g.n, 1, 4, 3)
    # eigenvalues agree to 1e-6 only when both solves are converged past that
    # level (|theta - lambda| <= ||r||^2 / gap), hence the tight tolerance
    ref = O.partition(g, 8, problem="normalized", precond="poly", poly_degree=10, tol=1e-6, init="piecewise",
                      seed=5, vwts=vw)
    graph = spx.Graph(g, vtx_w=vw, validate=True)
    parts, cut, imb, st, code = graph.partition(8, laplacian="normalized", precond="poly", poly_degree=10,
                                                precision="fp64", tol=1e-6, init="piecewise", seed=5)
    graph.close()
    assert code == 0
    assert np.allclose(st["eigenvalues"][1:], ref.eigenvalues[1:], rtol=1e-6)
    c, _ = O.cutsize(g, parts)
    assert c == cut and imb == O.imbalance(parts, vw, 8)


def test_k_one_and_more_parts_than_vertices():
    g = W.path_graph(5)
    parts, cut, imb, st, code = _gpu_partition(g, 1)
    assert list(parts) == [0] * 5 and cut == 0 and imb == 1.0
    parts, cut, imb, st, code = _gpu_partition(g, 8, tol=1e-6)
    assert code == 0
    assert sorted(parts) == sorted(O.multijagged(np.zeros((5, 3)) + np.arange(5)[:, None], None, 8))


def _fp64_residuals(g, problem, x, theta):
    """||L x - theta B x||_{B^-1} / ||x||_B per column, recomputed in FP64 with
    the oracle's explicit Laplacian from the returned vectors."""
    lmat = O.operator_for(g, problem)
    bd = O.b_diag_for(g, problem)
    if bd is None:
        bd = np.ones(g.n)
    r = lmat @ x - (bd[:, None] * x) * theta[None, :]
    return np.sqrt(np.sum(r * r / bd[:, None], axis=0)) / np.sqrt(np.sum(bd[:, None] * x * x, axis=0))


def test_c2_full_size_mixed_and_fp64():
    """128^3 27-point mesh, generalized, polynomial degree 25, K = 64, tol 1e-3,
    against the oracle's full run (tests/golden/c2_oracle.json): both
    precisions converge, eigenvalues agree with the oracle within 1e-6 (FP64)
    and 1e-3 (mixed), the cut is within 2 % of the oracle's and is the exact
    cut of the returned parts, and residuals recomputed in FP64 from the
    returned eigenvectors meet the convergence test."""
    import json
    import os
    torch = torch_mod()
    import paper_2105_00578_gb300 as spx
    with open(os.path.join(os.path.dirname(__file__), "golden", "c2_oracle.json")) as f:
        ref = json.load(f)
    g = W.grid3d(128, 128, 128, 27)
    graph = spx.Graph(g)
    kw = dict(laplacian="generalized", precond="poly", poly_degree=25, tol=1e-3, seed=2)
    ev_ref = np.array(ref["eigenvalues"])
    for precision in ("mixed_bf16", "fp64"):
        parts, cut, imb, st, code = graph.partition(64, precision=precision, **kw)
        assert code == 0, precision
        c, _ = O.cutsize(g, parts)
        assert c == cut
        assert imb <= 1.0 + 64 / g.n
        rtol = 1e-6 if precision == "fp64" else 1e-3
        assert np.allclose(st["eigenvalues"][1:], ev_ref[1:], rtol=rtol), precision
        assert abs(cut - ref["cut"]) <= 0.02 * ref["cut"], (precision, cut, ref["cut"])
        # the eigenvectors themselves, through the eigensolver entry point
        dt = torch.float64 if precision == "fp64" else torch.float32
        x = torch.zeros((g.n, 8), dtype=dt, device="cuda")
        code, theta, res, _ = spx.sphynx_eigensolve(graph.h, spx.options(precision=precision, **kw), 7, x, 8)
        assert code == 0
        torch.cuda.synchronize()
        got = _fp64_residuals(g, "generalized", x.double().cpu().numpy()[:, :7], theta)
        # FP32 storage of x alone puts a floor of about 10 u_f32 rho (rho = 2 here)
        # under any recomputed residual; FP64 has to meet the test outright
        floor = 10 * (2.0 ** -24 if precision != "fp64" else 2.0 ** -53) * 2.0
        for j in range(1, 7):
            assert got[j] <= 1e-3 * abs(theta[j]) + floor, (precision, j, got[j], theta[j])
    graph.close()


def test_default_options_follow_the_oracle_decision_flow():
    import paper_2105_00578_gb300 as spx
    names = {spx.COMBINATORIAL: "combinatorial", spx.GENERALIZED: "generalized", spx.NORMALIZED: "normalized"}
    inits = {spx.INIT_RANDOM: "random", spx.INIT_PIECEWISE: "piecewise"}
    for g in (W.grid3d(6, 5, 4, 27), W.star_graph(20), W.star_graph(21), W.rmat(12, seed=3)):
        h = spx.sphynx_create(g.row_ptr, g.col)
        try:
            assert spx.sphynx_get_info(h)["regular"] == int(O.is_regular(g))
            for pc in ("jacobi", "poly", "none", "amg"):
                o = spx.sphynx_default_options_for(h, pc)
                ref = O.default_options(g, pc)
                assert (names[o.laplacian], o.tol, inits[o.init]) == (ref["problem"], ref["tol"], ref["init"])
                assert o.precond == spx.PRECONDS[pc]
        finally:
            spx.sphynx_destroy(h)


def test_stall_window_stops_an_unreachable_fp32_target():
    """tol 1e-6 relative is below what FP32 blocks can resolve on this grid:
    without a stall window the solve runs to max_iter; with one it stops as
    soon as every unconverged column stopped improving, still NOCONV, with a
    valid partition of its best iterate."""
    g = W.grid2d(120, 100)
    kw = dict(laplacian="combinatorial", precond="jacobi", precision="fp32", tol=1e-6, seed=1, max_iter=600)
    _, _, _, st0, code0 = _gpu_partition(g, 4, **kw)
    assert code0 != 0 and st0["iterations"] == 600
    parts, cut, imb, st1, code1 = _gpu_partition(g, 4, stall_window=20, **kw)
    assert code1 != 0 and st1["iterations"] < 600
    assert O.cutsize(g, parts)[0] == cut and imb == O.imbalance(parts, None, 4)
