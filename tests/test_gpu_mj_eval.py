"""GPU multi-jagged and partition metrics: bit-exact against the oracle."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import torch_mod

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 7, 1000, 100003])
@pytest.mark.parametrize("K", [2, 3, 5, 8, 13, 64, 256])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("weighted", [False, True])
def test_mj_bit_exact(n, K, dtype, weighted):
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    dims = max(1, K.bit_length() - 1)
    npd = np.float64 if dtype == "f64" else np.float32
    c = W.random_coords(n, dims, seed=n + K, dtype=npd, ties=(K % 2 == 1))
    vw = W.random_vertex_weights(n, 1, 9, seed=K) if weighted else None
    cd = torch.from_numpy(c).cuda()
    vd = None if vw is None else torch.from_numpy(vw).cuda()
    part = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    spx.sphynx_mj(spx.DT_F64 if dtype == "f64" else spx.DT_F32, cd, dims, dims, n, vd, K, part)
    torch.cuda.synchronize()
    assert np.array_equal(part.cpu().numpy(), O.multijagged(c, vw, K))


def test_mj_strided_coordinates_and_signed_zero():
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    c = np.array([[0.0, 9.0], [-0.0, 9.0], [0.0, 9.0], [-1.0, 9.0], [2.0, 9.0], [-0.0, 9.0]], dtype=np.float32)
    part = torch.zeros(6, dtype=torch.int32, device="cuda")
    spx.sphynx_mj(spx.DT_F32, torch.from_numpy(c).cuda(), 2, 1, 6, None, 2, part)
    torch.cuda.synchronize()
    assert list(part.cpu().numpy()) == list(O.multijagged(c[:, :1], None, 2)) == [0, 0, 1, 0, 1, 1]


def test_mj_rejects_nan():
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    c = torch.tensor([[0.0], [float("nan")]], dtype=torch.float64, device="cuda")
    part = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(spx.SphynxError) as e:
        spx.sphynx_mj(spx.DT_F64, c, 1, 1, 2, None, 2, part)
    assert e.value.code == spx.ERR_INVALID_ARG


def test_mj_full_size_bit_exact():
    """2.1M points in 6 dimensions into 64 parts (the 128^3 mesh's embedding size)."""
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    n, K, dims = 128 ** 3, 64, 6
    c = W.random_coords(n, dims, seed=77, dtype=np.float32)
    part = torch.zeros(n, dtype=torch.int32, device="cuda")
    spx.sphynx_mj(spx.DT_F32, torch.from_numpy(c).cuda(), dims, dims, n, None, K, part)
    torch.cuda.synchronize()
    assert np.array_equal(part.cpu().numpy(), O.multijagged(c, None, K))


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("vweights", [False, True])
def test_eval_bit_exact(weighted, vweights):
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    g = W.largest_component(W.rmat(12, seed=5))
    if weighted:
        g = W.random_edge_weights(g, 0.5, 1.5, 3)
    vw = W.random_vertex_weights(g.n, 1, 5, 2) if vweights else None
    K = 37
    parts = (np.arange(g.n) * 2654435761 % K).astype(np.int32)
    h = spx.sphynx_create(g.row_ptr, g.col, g.w, vw)
    cut, cut2, imb = spx.sphynx_eval(h, torch.from_numpy(parts).cuda(), K)
    spx.sphynx_destroy(h)
    rc, rc2 = O.cutsize(g, parts)
    assert cut == rc and cut2 == rc2
    assert imb == O.imbalance(parts, vw, K)


def test_eval_rejects_out_of_range_parts():
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    g = W.grid2d(6, 5)
    h = spx.sphynx_create(g.row_ptr, g.col, None, None)
    parts = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    parts[3] = 9
    with pytest.raises(spx.SphynxError):
        spx.sphynx_eval(h, parts, 4)
    spx.sphynx_destroy(h)


@pytest.mark.parametrize("make,K,eps", [(lambda: W.grid2d(97, 61), 6, 0.03),
                                        (lambda: W.largest_component(W.rmat(12, seed=5)), 8, 0.05),
                                        (lambda: W.random_edge_weights(W.grid3d(21, 17, 13, 27), 0.5, 1.5, 3), 5,
                                         0.02)])
@pytest.mark.parametrize("vertex_weights", [False, True])
def test_greedy_refinement_is_bit_exact(make, K, eps, vertex_weights):
    """sphynx_refine (the greedy improvement step Sec. 7 proposes) against the
    oracle's restatement: the same parts vertex for vertex (every decision is
    an integer comparison), the same move and round counts, the exact cut."""
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    g = make()
    rng = np.random.default_rng(11)
    parts = (np.arange(g.n) * K // g.n).astype(np.int32)
    flip = rng.random(g.n) < 0.08
    parts[flip] = rng.integers(0, K, int(flip.sum()))
    vw = W.random_vertex_weights(g.n, 1, 5, 2) if vertex_weights else None
    ref = O.refine(g, parts, K, vwts=vw, eps=eps, max_rounds=25)
    h = spx.sphynx_create(g.row_ptr, g.col, g.w, vw)
    try:
        pd = torch.from_numpy(parts).cuda()
        cut, imb, moves, rounds = spx.sphynx_refine(h, pd, K, eps, 25)
        got = pd.cpu().numpy()
        assert np.array_equal(got, ref.parts)
        assert moves == ref.moves and rounds == ref.rounds
        assert cut == ref.cut and imb == O.imbalance(got, vw, K)
        assert ref.moves > 0
    finally:
        spx.sphynx_destroy(h)


def test_partition_with_refinement_lowers_the_cut():
    """refine_rounds > 0 in sphynx_partition: the multi-jagged partition is
    refined in place; its cut is at most the unrefined one, the imbalance
    stays within 1 % (or what multi-jagged left), and the result is what the
    oracle's refinement makes of the unrefined partition."""
    import paper_2105_00578_gb300 as spx
    g = W.largest_component(W.rmat(14, seed=3))
    graph = spx.Graph(g)
    try:
        kw = dict(laplacian="normalized", precond="jacobi", precision="fp64", tol=1e-2, seed=3)
        p0, cut0, imb0, st0, code0 = graph.partition(16, **kw)
        p1, cut1, imb1, st1, code1 = graph.partition(16, refine_rounds=20, **kw)
        assert code0 == code1 == spx.OK
        ref = O.refine(g, p0, 16, eps=0.01, max_rounds=20)
        assert np.array_equal(p1, ref.parts) and cut1 == ref.cut <= cut0
        assert st1["refine_moves"] == ref.moves
        assert imb1 <= max(imb0, 1.01)
    finally:
        graph.close()
