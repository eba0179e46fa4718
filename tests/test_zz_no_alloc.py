"""sphynx_mj_noalloc: multi-jagged for callers that cannot let the library
allocate device memory (a framework owning the whole memory pool, a
latency-bound loop that must not synchronise on cudaMalloc).

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
