"""GPU parity of the aggregation multigrid preconditioner (Sec. 5.3, with the
parameters of Sec. 6.2.2) against the oracle: the aggregates and coarse graphs
of every level bit for bit, the Chebyshev bounds, one V-cycle in FP64 and
FP32, and whole partitions preconditioned with it."""

import numpy as np
import pytest

import oracle as O
import oracle.amg as A
import workloads as W
from gpu_helpers import assert_elementwise, dev_block, torch_mod

pytestmark = pytest.mark.gpu


def graphs():
    return {
        "grid2d": W.grid2d(67, 45),                                   # 3015 vertices: two levels
        "grid27": W.grid3d(31, 29, 27, 27),                           # 24,273 vertices: three levels
        "weighted": W.random_edge_weights(W.grid2d(80, 61), 0.5, 1.5, 8),
        "rmat": W.rmat(13, seed=7),                                   # irregular, small hubs
        # a dozen aggregates hold more than 8192 entries (up to 340,000): their
        # coarse rows sort in global scratch, grouped by their own size class
        "rmat16": W.rmat(16, seed=7),
    }


GRAPHS = graphs()


def gpu_levels(spx, h, torch):
    """Every level's aggregates and CSR, read back through the C ABI."""
    info0 = spx.sphynx_amg_level(h, 0)
    out = []
    for ell in range(info0["levels"]):
        info = spx.sphynx_amg_level(h, ell)
        n, nnz = info["n"], info["nnz"]
        rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        cl = torch.zeros(max(nnz, 1), dtype=torch.int32, device="cuda")
        w = torch.zeros(max(nnz, 1), dtype=torch.float32, device="cuda") if ell > 0 else None
        agg = torch.zeros(n, dtype=torch.int32, device="cuda") if info["n_next"] > 0 else None
        spx.sphynx_amg_level(h, ell, agg, rp, cl, w)
        torch.cuda.synchronize()
        out.append(dict(info=info, agg=None if agg is None else agg.cpu().numpy(), row_ptr=rp.cpu().numpy(),
                        col=cl.cpu().numpy()[:nnz], w=None if w is None else w.cpu().numpy()[:nnz]))
    return out


@pytest.mark.parametrize("name", list(GRAPHS))
def test_hierarchy_matches_the_oracle_level_by_level(name):
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    g = GRAPHS[name]
    seed = 11
    h = spx.sphynx_create(g.row_ptr, g.col, g.w, None, g.n, g.nnz, spx.VALIDATE)
    try:
        spx.sphynx_precond_setup(h, spx.options(precond="amg", seed=seed))
        got = gpu_levels(spx, h, torch)
        ref = A.build_hierarchy(g, seed)
        assert len(got) == len(ref)
        for ell, (a, b) in enumerate(zip(got, ref)):
            assert a["info"]["n"] == b.g.n and a["info"]["nnz"] == b.g.nnz
            if ell > 0:
                # the aggregate graph: structure exact; weights are sums of float
                # fine weights, exact in double on both sides, and the C ABI
                # returns them rounded to float once
                assert np.array_equal(a["row_ptr"], b.g.row_ptr) and np.array_equal(a["col"], b.g.col)
                assert np.array_equal(a["w"], b.g.w.astype(np.float32))
            if b.agg is None:
                assert a["agg"] is None and a["info"]["n_next"] == 0
            else:
                assert np.array_equal(a["agg"].astype(np.int64), b.agg), ell   # integer work: bit for bit
                assert a["info"]["n_next"] == b.nc
            assert a["info"]["lambda_max"] == pytest.approx(b.lam_max, rel=1e-9)
    finally:
        spx.sphynx_destroy(h)


@pytest.mark.parametrize("name", ["grid2d", "grid27", "weighted", "rmat", "rmat16", "star"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_one_vcycle_matches_the_oracle(name, precision):
    """"star": one aggregate holds the whole graph (its 18,000 entries take the
    global-memory sort) and the coarse level has no edges.  "rmat16": a dozen
    hub aggregates of up to 340,000 entries sort in global scratch."""
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    g = W.star_graph(9001) if name == "star" else GRAPHS[name]
    seed = 5
    h = spx.sphynx_create(g.row_ptr, g.col, g.w, None)
    try:
        opt = spx.options(precond="amg", seed=seed, precision=precision)
        spx.sphynx_precond_setup(h, opt)
        levels = A.build_hierarchy(g, seed)
        rng = np.random.default_rng(3)
        for ncols in (1, 3, 7):
            ld = (ncols + 3) // 4 * 4
            r = rng.standard_normal((g.n, ncols))
            dt = "f64" if precision == "fp64" else "f32"
            rd = dev_block(r, ld, dt)
            hd = torch.zeros_like(rd)
            spx.sphynx_precond_apply(h, opt, rd, hd, ld, ncols)
            torch.cuda.synchronize()
            rin = rd.double().cpu().numpy()[:, :ncols]
            ref = A.vcycle(levels, rin)
            got = hd.double().cpu().numpy()
            # element by element, against each column's largest entry (a V-cycle
            # mixes every entry with its neighbourhood, so no entry has a scale
            # of its own).  FP64 cycles run the coarse levels on their double
            # weights, as the oracle does
            tol = 1e-8 if precision == "fp64" else 2e-4
            colmax = np.max(np.abs(ref), axis=0, keepdims=True)
            assert_elementwise(got[:, :ncols], ref, tol * colmax, f"{name} {precision} ncols {ncols}")
            assert np.all(got[:, ncols:] == 0)                        # zero padding columns stay zero
    finally:
        spx.sphynx_destroy(h)


@pytest.mark.parametrize("problem", ["combinatorial", "generalized"])
def test_partition_with_multigrid_matches_the_oracle(problem):
    import paper_2105_00578_gb300 as spx
    for g, K in ((W.grid2d(64, 48), 4), (W.grid3d(24, 22, 20, 27), 8)):
        ref = O.partition(g, K, problem=problem, precond="amg", tol=1e-3, seed=2)
        graph = spx.Graph(g)
        try:
            for precision, rtol in (("fp64", 1e-6), ("fp32", 1e-3)):
                parts, cut, imb, st, code = graph.partition(K, laplacian=problem, precond="amg", precision=precision,
                                                            tol=1e-3, seed=2)
                assert code == spx.OK, (precision, code)
                ev = np.array(st["eigenvalues"])
                assert np.allclose(ev[1:], ref.eigenvalues[1:], rtol=rtol), (precision, ev, ref.eigenvalues)
                assert abs(cut - ref.cut) <= 0.02 * ref.cut, (precision, cut, ref.cut)
                c_or, _ = O.cutsize(g, parts)
                assert c_or == cut and imb == O.imbalance(parts, None, K)
                # multigrid converges in far fewer iterations than Jacobi needs
                assert st["iterations"] <= 2 * ref.iterations + 5
        finally:
            graph.close()


def test_multigrid_rejects_what_it_does_not_cover():
    import paper_2105_00578_gb300 as spx
    g = W.grid2d(50, 50)
    h = spx.sphynx_create(g.row_ptr, g.col)
    try:
        parts = np.zeros(g.n, dtype=np.int32)
        with pytest.raises(spx.SphynxError) as e:                     # normalized: M approximates L_C^{-1}
            spx.sphynx_partition(h, 4, spx.options(laplacian="normalized", precond="amg"), parts)
        assert e.value.code == spx.ERR_INVALID_ARG
        with pytest.raises(spx.SphynxError) as e:                     # no hierarchy yet
            spx.sphynx_amg_level(h, 0)
        assert e.value.code == spx.ERR_INVALID_ARG
        spx.sphynx_precond_setup(h, spx.options(precond="amg"))
        with pytest.raises(spx.SphynxError) as e:
            spx.sphynx_amg_level(h, 7)
        assert e.value.code == spx.ERR_INVALID_ARG
    finally:
        spx.sphynx_destroy(h)

