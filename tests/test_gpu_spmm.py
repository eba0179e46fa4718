"""GPU parity of the fused Laplacian SpMM (Y = L X without forming L) against
the oracle's explicit FP64 Laplacians (Eqs. 2-3, weighted rule)."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import abs_operator, assert_elementwise, bf16_round, dev_block, spmm_bound, torch_mod

pytestmark = pytest.mark.gpu


def graphs():
    return {
        "grid2d": W.grid2d(67, 45),                                   # ragged row tail
        "grid27": W.grid3d(19, 13, 11, 27),
        "rmat": W.rmat(12, seed=7),                                   # power law: long rows
        "rmat_w": W.random_edge_weights(W.rmat(11, seed=9), 0.5, 1.5, 5),
        "star": W.star_graph(9001),                                   # one row split in 3 chunks
        # wrap-around edges reach 44,700 rows: the boundary slices keep 32-bit
        # indices, the interior ones 16-bit offsets
        "torus_wide": W.grid2d(300, 150, periodic=True),
        "torus_wide_w": W.random_edge_weights(W.grid2d(300, 150, periodic=True), 0.5, 1.5, 8),
        "rmat16": W.rmat(16, seed=11),                                # mostly 32-bit slices, long rows
    }


GRAPHS = graphs()


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("lap", ["combinatorial", "normalized"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("ncols", [1, 3, 7, 9, 16])
def test_spmm_matches_oracle(gname, lap, dtype, ncols):
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    if ncols == 1 and dtype == "bf16":
        pytest.skip("single-column products are float/double only")
    g = GRAPHS[gname]
    h = spx.sphynx_create(g.row_ptr, g.col, g.w, None, g.n, g.nnz, spx.VALIDATE)
    try:
        rng = np.random.default_rng(ncols)
        x = rng.standard_normal((g.n, ncols))
        ld = 1 if ncols == 1 else (ncols + 3) // 4 * 4
        xd = dev_block(x, ld, dtype)
        ydt = torch.float64 if dtype == "f64" else torch.float32
        y = torch.zeros((g.n, ld), dtype=ydt, device="cuda")
        dt = {"f64": spx.DT_F64, "f32": spx.DT_F32, "bf16": spx.DT_BF16}[dtype]
        xin = x if dtype == "f64" else (x.astype(np.float32).astype(np.float64) if dtype == "f32" else bf16_round(x))
        lmat = O.operator_for(g, lap)
        ref = lmat @ xin
        # element by element: the rounding bound of each row's sum (FP64: both
        # the library's and the oracle's own rounding)
        u = 2.0 ** -53 if dtype == "f64" else 2.0 ** -24
        bound = spmm_bound(lmat, xin, u, c=3.0 if dtype == "f64" else 2.0)
        # every short-row schedule and, on graphs with longer rows, every
        # medium-row ceiling the autotuner chooses from
        ceilings = (32, 128, 4096) if int(g.degrees().max()) > 32 else (4096,)
        for med_max in ceilings:
            spx.sphynx_set_spmm_med_max(h, med_max)
            # CSR staged; SELL-32 under every slice stride (slices a block's
            # warps take apart), which must not change any row's value; and the
            # shared-pattern slices where the graph has them, which sum every
            # row in the explicit slices' order
            schedules = [(0, 1), (1, 1), (1, 2), (1, 4), (1, 8), (1, 16)]
            if spx.sphynx_get_info(h)["sell_pattern_slices"] > 0:
                schedules += [(2, 1), (2, 4), (2, 16)]
            for variant, stride in schedules:
                spx.sphynx_set_spmm_variant(h, variant)
                spx.sphynx_set_spmm_sell_stride(h, stride)
                y.zero_()
                spx.sphynx_laplacian_apply(h, lap, dt, xd, ld, y, ld, ncols)
                torch.cuda.synchronize()
                got = y.cpu().numpy().astype(np.float64)[:, :ncols]
                assert_elementwise(got, ref, bound, f"variant {variant} stride {stride} med_max {med_max}")
                if variant == 1 and stride == 1:
                    first = got
                elif variant >= 1:
                    # the same sums in the same order, whichever block runs them
                    assert np.array_equal(got, first), (variant, stride)
            # padding columns stay zero when the input padding is zero
            if ld > ncols and ncols > 1:
                assert np.all(y.cpu().numpy()[:, ncols:] == 0)
    finally:
        spx.sphynx_destroy(h)


def test_degrees_exact():
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    for g in GRAPHS.values():
        h = spx.sphynx_create(g.row_ptr, g.col, g.w, None)
        d = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        spx.sphynx_degrees(h, d)
        torch.cuda.synchronize()
        ref = O.weighted_degree(g)
        if g.w is None:
            assert np.array_equal(d.cpu().numpy(), ref)
        else:
            assert np.allclose(d.cpu().numpy(), ref, rtol=1e-15)
        info = spx.sphynx_get_info(h)
        assert info["max_degree"] == int(g.degrees().max())
        assert info["long_rows"] == int(np.sum(g.degrees() > 32))
        assert info["spmm_variant"] in (0, 1, 2) and info["tuned_us_csr"] > 0 and info["tuned_us_sell"] > 0
        # the tuner kept the fastest schedule it timed (the shared-pattern one
        # only where the graph has such slices)
        times = [info["tuned_us_csr"], info["tuned_us_sell"]]
        if info["sell_pattern_slices"] > 0:
            assert info["tuned_us_pattern"] > 0
            times.append(info["tuned_us_pattern"])
        else:
            assert info["tuned_us_pattern"] == 0 and info["spmm_variant"] != 2
        assert info["spmm_variant"] == int(np.argmin(times))
        assert info["sell_stride"] in (1, 2, 4, 8, 16)
        if info["spmm_variant"] == 0:
            assert info["sell_stride"] == 1
        spx.sphynx_destroy(h)


def pattern_slices(g) -> np.ndarray:
    """Per 32-row slice: True when the offsets col - row of its short rows (at
    most 32 neighbours) all fit 16 bits and take at most 31 distinct values
    (unweighted graphs only), written from that definition."""
    n_sl = (g.n + 31) // 32
    if g.w is not None:
        return np.zeros(n_sl, dtype=bool)
    deg = g.degrees()
    r = g.rows()
    off = g.col.astype(np.int64) - r
    keep = deg[r] <= 32
    out = np.ones(n_sl, dtype=bool)
    sl = r[keep] >> 5
    o = off[keep]
    bad = (o < -32768) | (o > 32767)
    out[np.unique(sl[bad])] = False
    pairs = np.unique(np.stack([sl, o]), axis=1)
    cnt = np.bincount(pairs[0], minlength=n_sl)
    out[cnt > 31] = False
    return out


def test_sell_slice_formats_follow_the_offset_range():
    """A slice stores 16-bit offsets exactly when every short-row entry of its
    32 rows lies within [-32768, 32767] of its row; the byte count a product
    reads from the layout follows."""
    import paper_2105_00578_gb300 as spx
    for name in ("torus_wide", "rmat16", "grid27", "rmat"):
        g = GRAPHS[name]
        r = g.rows()
        off = g.col.astype(np.int64) - r
        deg = g.degrees()
        short_entry = deg[r] <= 32
        wide = np.zeros((g.n + 31) // 32, dtype=bool)
        np.logical_or.at(wide, r >> 5, short_entry & ((off < -32768) | (off > 32767)))
        h = spx.sphynx_create(g.row_ptr, g.col, g.w, None)
        try:
            info = spx.sphynx_get_info(h)
            assert info["sell_slices"] == wide.size
            assert info["sell_narrow_slices"] == int((~wide).sum()), name
            # medium rows (33 to the tuned ceiling): their entries, 20 bytes a
            # row (id and row pointers), 8 per warp unit; long rows: CSR
            # entries, 32 bytes per 1024-entry item and 24 per row
            mm = info["spmm_med_max"]
            assert mm in (32, 128, 4096)
            med = (deg > 32) & (deg <= mm)
            med_bytes = 4.0 * deg[med].sum() + 20.0 * int(med.sum()) + 8.0 * medium_units(deg[med])
            lng = deg > mm
            long_bytes = 4.0 * deg[lng].sum() + 32 * int(np.sum((deg[lng] + 1023) // 1024)) + 24 * int(lng.sum())
            short_per_slice = np.bincount(r[short_entry] >> 5, minlength=wide.size)
            pat = pattern_slices(g)
            assert info["sell_pattern_slices"] == int(pat.sum()), name
            if info["spmm_variant"] == 1:
                idx = float(np.sum(np.where(wide, 4, 2) * short_per_slice))
                expect = idx + g.n + 8 * wide.size
            elif info["spmm_variant"] == 2:
                rows_in = np.minimum(32, g.n - 32 * np.arange(wide.size))
                idx = np.where(pat, 192.0, np.where(wide, 4, 2) * short_per_slice + rows_in)
                expect = float(idx.sum()) + 8 * wide.size
            else:
                expect = 8 * (g.n + 1) + 4 * deg[deg <= 32].sum()
            expect += med_bytes + long_bytes
            assert info["spmm_graph_bytes"] == pytest.approx(expect, rel=1e-12), name
        finally:
            spx.sphynx_destroy(h)


def medium_units(degs: np.ndarray) -> int:
    """Warp units of the medium-row kernel: rows by degree, descending; a row
    of d entries takes G = 2^lg lanes, the smallest with d <= 16 G (G <= 32),
    and consecutive rows of one G share a unit up to 32 / G rows."""
    lg = np.zeros(len(degs), dtype=np.int64)
    for k in range(5):
        lg += (16 << k) < degs
    units = 0
    for v in np.unique(lg):
        units += -(-int(np.sum(lg == v)) // (32 >> int(v)))
    return units


@pytest.mark.parametrize("lap", ["normalized", "combinatorial"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_null_vector_is_annihilated_to_rounding(lap, dtype):
    """L D^{1/2} 1 = 0 (L_N) and L 1 = 0 (L_C): the products of a row must
    cancel to rounding level even for rows of thousands of entries (LOBPCG
    recognises the eigenvalue-zero column by it).  Bound: about (32 + d / 32)
    roundings of a row's largest term, as the blocked per-lane summation
    gives, times a safety factor of 4."""
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    g = W.random_edge_weights(GRAPHS["rmat16"], 0.5, 1.5, 3) if lap == "combinatorial" else GRAPHS["rmat16"]
    deg = O.weighted_degree(g)
    z = np.sqrt(deg) if lap == "normalized" else np.ones(g.n)
    h = spx.sphynx_create(g.row_ptr, g.col, g.w, None)
    try:
        xd = dev_block(z[:, None], 1, dtype)
        y = torch.zeros((g.n, 1), dtype=torch.float64 if dtype == "f64" else torch.float32, device="cuda")
        for variant, med_max in ((0, 4096), (1, 4096), (1, 128), (1, 32)):
            spx.sphynx_set_spmm_med_max(h, med_max)
            spx.sphynx_set_spmm_variant(h, variant)
            spx.sphynx_laplacian_apply(h, lap, spx.DT_F64 if dtype == "f64" else spx.DT_F32, xd, 1, y, 1, 1)
            torch.cuda.synchronize()
            got = np.abs(y.cpu().numpy().astype(np.float64)[:, 0])
            u = 2.0 ** -24 if dtype == "f32" else 2.0 ** -53
            d = np.diff(g.row_ptr)
            scale = z if lap == "normalized" else deg     # size of a row's largest partial sums
            bound = 4 * u * (32 + d / 32 + 1) * np.maximum(scale, 1.0)
            assert np.all(got <= bound), (variant, float(np.max(got / bound)))
    finally:
        spx.sphynx_destroy(h)


def test_input_rows_wider_than_the_block_are_packed():
    """sphynx_laplacian_apply accepts X rows further apart than the block
    width (the kernels read them exactly bp apart, so the call packs X first):
    same result as the packed layout."""
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    g = GRAPHS["rmat"]
    h = spx.sphynx_create(g.row_ptr, g.col, g.w, None)
    try:
        x = np.random.default_rng(4).standard_normal((g.n, 7))
        packed = dev_block(x, 8, "f32")
        wide = dev_block(x, 12, "f32")
        y1 = torch.zeros((g.n, 8), dtype=torch.float32, device="cuda")
        y2 = torch.zeros((g.n, 8), dtype=torch.float32, device="cuda")
        spx.sphynx_laplacian_apply(h, "normalized", spx.DT_F32, packed, 8, y1, 8, 7)
        spx.sphynx_laplacian_apply(h, "normalized", spx.DT_F32, wide, 12, y2, 8, 7)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
    finally:
        spx.sphynx_destroy(h)


def test_full_size_27_point_mesh_sampled_rows():
    """128^3 27-point mesh (the 2.1M-vertex workload): sampled rows of L_C X
    recomputed by the oracle row by row."""
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    g = W.grid3d(128, 128, 128, 27)
    h = spx.sphynx_create(g.row_ptr, g.col, None, None)
    try:
        rng = np.random.default_rng(5)
        for dtype, ld, variant, stride in (("f32", 8, 0, 1), ("f32", 8, 1, 1), ("f32", 8, 1, 4), ("f64", 8, 1, 4),
                                           ("bf16", 8, 1, 4), ("bf16", 8, 1, 16), ("bf16", 8, 0, 1)):
            spx.sphynx_set_spmm_variant(h, variant)
            spx.sphynx_set_spmm_sell_stride(h, stride)
            x = rng.standard_normal((g.n, 7))
            xd = dev_block(x, ld, dtype)
            y = torch.zeros((g.n, ld), dtype=torch.float64 if dtype == "f64" else torch.float32, device="cuda")
            spx.sphynx_laplacian_apply(h, "combinatorial", {"f64": 0, "f32": 1, "bf16": 2}[dtype], xd, ld, y, ld, 7)
            torch.cuda.synchronize()
            xin = xd.double().cpu().numpy()[:, :7]
            rows = np.concatenate([np.arange(5), rng.integers(0, g.n, 2000), [g.n - 1]])
            got = y.cpu().numpy().astype(np.float64)[rows, :7]
            ref = np.zeros_like(got)
            mag = np.zeros_like(got)
            for k, i in enumerate(rows):
                nb = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
                ref[k] = len(nb) * xin[i] - xin[nb].sum(axis=0)
                mag[k] = len(nb) * np.abs(xin[i]) + np.abs(xin[nb]).sum(axis=0)
            # element by element: c (t + 6) u (|L| |X|) for the row's t terms
            u = 2.0 ** -53 if dtype == "f64" else 2.0 ** -24
            terms = np.diff(g.row_ptr)[rows].astype(np.float64)
            bound = (3.0 if dtype == "f64" else 2.0) * u * (terms + 6.0)[:, None] * mag
            assert_elementwise(got, ref, bound, f"{dtype} variant {variant} stride {stride}")
    finally:
        spx.sphynx_destroy(h)


def test_invalid_inputs_are_rejected():
    import paper_2105_00578_gb300 as spx
    g = W.grid2d(5, 4)
    col = g.col.copy()
    col[3] = g.n + 5                                   # out of range
    with pytest.raises(spx.SphynxError) as e:
        spx.sphynx_create(g.row_ptr, col, None, None)
    assert e.value.code == spx.ERR_INVALID_ARG
    # drop one direction of an edge: not symmetric
    rows = g.rows()
    keep = ~((rows == 0) & (g.col == 1))
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=g.n))])
    with pytest.raises(spx.SphynxError) as e:
        spx.sphynx_create(rp, g.col[keep], None, None, flags=spx.VALIDATE)
    assert e.value.code == spx.ERR_NOT_SYMMETRIC
    # isolated vertex: normalized problem refused
    g2 = W.symmetrize_edges(4, np.array([0, 1]), np.array([1, 2]))
    h = spx.sphynx_create(g2.row_ptr, g2.col, None, None)
    parts = np.zeros(4, dtype=np.int32)
    with pytest.raises(spx.SphynxError) as e:
        spx.sphynx_partition(h, 2, spx.options(laplacian="normalized"), parts)
    assert e.value.code == spx.ERR_ISOLATED
    for stride in (0, 3, 32):                          # slice strides are 1, 2, 4, 8, 16 (or -1: tune)
        with pytest.raises(spx.SphynxError) as e:
            spx.sphynx_set_spmm_sell_stride(h, stride)
        assert e.value.code == spx.ERR_INVALID_ARG
    spx.sphynx_destroy(h)


@pytest.mark.parametrize("dtype_in,dtype_out", [("bf16", "bf16"), ("f32", "bf16"), ("f32", "f32"), ("f64", "f64")])
def test_polynomial_chain_step_full_size_mesh_elementwise(dtype_in, dtype_out):
    """One product-form step of the polynomial preconditioner (Sec. 5.2) on the
    full 128^3 27-point mesh (2,097,152 rows), every row and column checked
    element by element, in the schedule the autotuner picks at create (the
    launch configuration of the benchmark) and in the CSR-staged one.  With
    t the exact input block:
      t_out = t - (L t) / theta_cur: float (or double) rounding of each row's
        sum, c (t_i + 6) u (|t| + |L| |t| / theta_cur), then one rounding to the
        stored type, u_out |ref|;
      y (two terms): y0 + t / theta_cur + t_out / theta_next with the library's
        own stored t_out, three roundings of the magnitudes;
      y (no term): unchanged bit for bit.
    Float steps use the float-rounded reciprocals of the roots, so the oracle
    side uses the same reciprocals."""
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    g = W.grid3d(128, 128, 128, 27)
    lmat = O.operator_for(g, "combinatorial")
    alap = abs_operator(lmat)
    terms = np.diff(lmat.indptr).astype(np.float64)[:, None]
    codes = {"f64": spx.DT_F64, "f32": spx.DT_F32, "bf16": spx.DT_BF16}
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
    u_acc = 2.0 ** -53 if dtype_in == "f64" else 2.0 ** -24
    u_out = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8}[dtype_out]
    theta_cur, theta_next = 3.7, 11.3
    if dtype_in == "f64":
        ic, inx = 1.0 / theta_cur, 1.0 / theta_next
    else:
        ic, inx = float(np.float32(1.0 / theta_cur)), float(np.float32(1.0 / theta_next))
    rng = np.random.default_rng(21)
    ncols, ld = 7, 8
    h = spx.sphynx_create(g.row_ptr, g.col, None, None)
    try:
        td = dev_block(rng.standard_normal((g.n, ncols)), ld, dtype_in)
        tin = td.double().cpu().numpy()[:, :ncols]
        ref_t = tin - (lmat @ tin) * ic
        mag_t = np.abs(tin) + (alap @ np.abs(tin)) * ic
        c = 3.0 if dtype_in == "f64" else 2.0
        bound_t = u_out * np.abs(ref_t) + (1 + u_out) * c * u_acc * (terms + 6.0) * mag_t
        ydt = torch.float64 if dtype_in == "f64" else torch.float32
        y0 = torch.from_numpy(rng.standard_normal((g.n, ld))).to(device="cuda", dtype=ydt)
        for variant in ("tuned", "csr"):
            if variant == "csr":
                spx.sphynx_set_spmm_variant(h, 0)
            for yterms, first in ((2, 0), (2, 1), (1, 0), (0, 0)):
                tout = torch.zeros((g.n, ld), dtype=tdt[dtype_out], device="cuda")
                y = y0.clone()
                spx.sphynx_poly_step(h, "combinatorial", codes[dtype_in], td, codes[dtype_out], tout, y, ld, ncols,
                                     theta_cur, theta_next, yterms, first)
                torch.cuda.synchronize()
                tg = tout.double().cpu().numpy()[:, :ncols]
                what = f"{dtype_in}->{dtype_out} {variant} yterms {yterms} first {first}"
                assert_elementwise(tg, ref_t, bound_t, "t_out " + what)
                yg = y.double().cpu().numpy()[:, :ncols]
                yin = y0.double().cpu().numpy()[:, :ncols]
                if yterms == 0:
                    assert np.array_equal(yg, yin), what
                    continue
                base = np.zeros_like(yin) if first else yin
                ref_y = base + (tin * ic if yterms == 2 else 0.0) + tg * inx
                mag_y = np.abs(base) + (np.abs(tin) * ic if yterms == 2 else 0.0) + np.abs(tg) * inx
                assert_elementwise(yg, ref_y, 4.0 * u_acc * mag_y, "y " + what)
    finally:
        spx.sphynx_destroy(h)
