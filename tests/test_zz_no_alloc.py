"""sphynx_mj_noalloc: multi-jagged for callers that cannot let the library
allocate device memory (a framework whose caching allocator has already
reserved the device's memory, an application that allows no allocation after
start-up).

It must give exactly what sphynx_mj gives (part ids are integers, so the
comparison is exact), call after call, although every call reuses the same
fixed scratch array.  This file is collected last so that a run stopping at
the first failure has already run every other test.
"""

import numpy as np
import pytest

import workloads as W
from gpu_helpers import torch_mod

pytestmark = pytest.mark.gpu


def _both(c, vw, K, dtype_code):
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    n, dims = c.shape
    cd = torch.from_numpy(c).cuda()
    vd = None if vw is None else torch.from_numpy(vw).cuda()
    ref = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    got = torch.full((n,), -2, dtype=torch.int32, device="cuda")
    spx.sphynx_mj(dtype_code, cd, dims, dims, n, vd, K, ref)
    spx.sphynx_mj_noalloc(dtype_code, cd, dims, dims, n, vd, K, got)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy()


def test_no_alloc_matches_allocating_entry_point_on_consecutive_calls():
    import paper_2105_00578_gb300 as spx
    # first call: float coordinates, unit weights, K = 64 on 300k points
    c1 = W.random_coords(300_000, 6, seed=11, dtype=np.float32)
    ref, got = _both(c1, None, 64, spx.DT_F32)
    assert np.array_equal(got, ref)
    # second call reuses the scratch left by the first: double coordinates
    # with ties, vertex weights, a different K and size
    c2 = W.random_coords(70_001, 3, seed=12, dtype=np.float64, ties=True)
    vw = W.random_vertex_weights(70_001, 1, 9, seed=13)
    ref, got = _both(c2, vw, 13, spx.DT_F64)
    assert np.array_equal(got, ref)
    # and the first problem again, after the second left its contents behind
    ref, got = _both(c1, None, 64, spx.DT_F32)
    assert np.array_equal(got, ref)


def test_no_alloc_rejects_problems_beyond_its_scratch():
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    n = 3_000_000                                   # 8 n bytes alone exceed 16 MiB
    c = torch.zeros((n, 1), dtype=torch.float32, device="cuda")
    part = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(spx.SphynxError) as e:
        spx.sphynx_mj_noalloc(spx.DT_F32, c, 1, 1, n, None, 2, part)
    assert e.value.code == spx.ERR_UNSUPPORTED
    assert "scratch" in spx.last_error() or "16777216" in str(e.value)


def test_no_alloc_leaves_device_memory_untouched_at_its_documented_bound():
    """n = 2^20 points with K = 1024 parts is the documented bound that fits the
    fixed array; the call must succeed there, agree with sphynx_mj, and leave
    the device's free memory exactly as it found it."""
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    n, K, dims = 1 << 20, 1024, 4
    c = W.random_coords(n, dims, seed=14, dtype=np.float32)
    cd = torch.from_numpy(c).cuda()
    ref = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    got = torch.full((n,), -2, dtype=torch.int32, device="cuda")
    spx.sphynx_mj(spx.DT_F32, cd, dims, dims, n, None, K, ref)
    # the allocating call's pool returns its memory at synchronisation points
    torch.cuda.synchronize()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    spx.sphynx_mj_noalloc(spx.DT_F32, cd, dims, dims, n, None, K, got)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_no_alloc_and_allocating_entry_points_agree_on_error_codes():
    import paper_2105_00578_gb300 as spx
    torch = torch_mod()
    c = torch.zeros((8, 1), dtype=torch.float32, device="cuda")
    part = torch.zeros(8, dtype=torch.int32, device="cuda")
    for fn in (spx.sphynx_mj, spx.sphynx_mj_noalloc):
        with pytest.raises(spx.SphynxError) as e:
            fn(spx.DT_F32, c, 1, 1, 8, None, (1 << 20) + 1, part)
        assert e.value.code == spx.ERR_UNSUPPORTED
        for bad_k, bad_n in ((0, 8), (2, -1)):
            with pytest.raises(spx.SphynxError) as e:
                fn(spx.DT_F32, c, 1, 1, bad_n, None, bad_k, part)
            assert e.value.code == spx.ERR_INVALID_ARG
