"""Python binding of libsphynx, the GB300 spectral partitioner (Sphynx hot path).

The library is a C ABI (include/sphynx.h); this module only marshals
arguments through ctypes.  Device buffers are passed as torch CUDA tensors (or
raw integer device pointers); host buffers as numpy arrays.  Every step runs
in the library's CUDA kernels: if the shared library is missing, importing
this package raises, there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsphynx.so")

# status codes
OK, ERR_INVALID_ARG, ERR_NOT_SYMMETRIC, ERR_ISOLATED, ERR_OOM, ERR_CUDA, ERR_NOCONV, ERR_BREAKDOWN, \
    ERR_UNSUPPORTED = range(9)
HOST_PTRS, DEVICE_PTRS, VALIDATE = 0, 1, 2
COMBINATORIAL, GENERALIZED, NORMALIZED = 0, 1, 2
PRECOND_NONE, PRECOND_JACOBI, PRECOND_POLY, PRECOND_AMG = 0, 1, 2, 3
FP64, FP32, MIXED_BF16 = 0, 1, 2
INIT_RANDOM, INIT_PIECEWISE = 0, 1
CONV_REL_THETA, CONV_ABS = 0, 1
DT_F64, DT_F32, DT_BF16 = 0, 1, 2
OUT_DEVICE = 1
MAX_NEV = 16
MAX_POLY_DEGREE = 64

LAPLACIANS = {"combinatorial": COMBINATORIAL, "generalized": GENERALIZED, "normalized": NORMALIZED}
PRECONDS = {"none": PRECOND_NONE, "jacobi": PRECOND_JACOBI, "poly": PRECOND_POLY, "amg": PRECOND_AMG}
PRECISIONS = {"fp64": FP64, "fp32": FP32, "mixed_bf16": MIXED_BF16}
INITS = {"random": INIT_RANDOM, "piecewise": INIT_PIECEWISE}
CONVS = {"rel_theta": CONV_REL_THETA, "abs": CONV_ABS}


class Options(C.Structure):
    _fields_ = [("laplacian", C.c_int32), ("precond", C.c_int32), ("poly_degree", C.c_int32),
                ("precision", C.c_int32), ("init", C.c_int32), ("max_iter", C.c_int32),
                ("tol", C.c_double), ("seed", C.c_uint64), ("flags", C.c_uint32),
                ("sync_every", C.c_int32), ("stall_window", C.c_int32), ("conv", C.c_int32),
                ("refine_rounds", C.c_int32), ("reserved", C.c_int32 * 3)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("nev", C.c_int32),
                ("svqb_steps", C.c_int32), ("eigenvalues", C.c_double * MAX_NEV),
                ("resnorm", C.c_double * MAX_NEV), ("ms_total", C.c_double), ("ms_setup", C.c_double),
                ("ms_lobpcg", C.c_double), ("ms_mj", C.c_double), ("ms_eval", C.c_double),
                ("ms_spmm", C.c_double), ("spmm_launches", C.c_int64), ("spmm_bytes", C.c_double),
                ("kernel_launches", C.c_int64), ("cut", C.c_double), ("cut_twice", C.c_double),
                ("imbalance", C.c_double),
                ("ms_spmm_by_dt", C.c_double * 3), ("spmm_bytes_by_dt", C.c_double * 3),
                ("spmm_launches_by_dt", C.c_int64 * 3), ("fp64_finished", C.c_int32), ("refine_moves", C.c_int32),
                ("ms_phase", C.c_double * 2), ("loop_iters", C.c_int32 * 2)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_
             if f not in ("reserved", "eigenvalues", "resnorm")}
        d["eigenvalues"] = list(self.eigenvalues[: self.nev])
        d["resnorm"] = list(self.resnorm[: self.nev])
        d["ms_phase"] = list(self.ms_phase)
        d["loop_iters"] = list(self.loop_iters)
        return d


class GraphInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("max_degree", C.c_int64), ("max_wdegree", C.c_double),
                ("total_vweight", C.c_int64), ("long_rows", C.c_int64), ("weighted", C.c_int32),
                ("spmm_variant", C.c_int32), ("tuned_us_csr", C.c_float), ("tuned_us_sell", C.c_float),
                ("sell_slices", C.c_int64), ("sell_narrow_slices", C.c_int64), ("spmm_graph_bytes", C.c_double),
                ("regular", C.c_int32), ("spmm_med_max", C.c_int32), ("sell_stride", C.c_int32),
                ("tuned_us_pattern", C.c_float), ("sell_pattern_slices", C.c_int64)]


class AmgLevelInfo(C.Structure):
    _fields_ = [("levels", C.c_int32), ("reserved", C.c_int32), ("n", C.c_int64), ("nnz", C.c_int64),
                ("n_next", C.c_int64), ("lambda_max", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2105_00578_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, u32, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
    pd, pi32 = C.POINTER(C.c_double), C.POINTER(C.c_int32)
    sig = {
        "sphynx_default_options": (None, [C.POINTER(Options)]),
        "sphynx_last_error": (C.c_char_p, []),
        "sphynx_create": (C.c_int, [vp, vp, vp, vp, i64, i64, u32, vp, C.POINTER(vp)]),
        "sphynx_destroy": (None, [vp]),
        "sphynx_get_info": (C.c_int, [vp, C.POINTER(GraphInfo)]),
        "sphynx_set_spmm_variant": (C.c_int, [vp, i32]),
        "sphynx_set_spmm_sell_stride": (C.c_int, [vp, i32]),
        "sphynx_degrees": (C.c_int, [vp, vp]),
        "sphynx_laplacian_apply": (C.c_int, [vp, i32, i32, vp, i32, vp, i32, i32]),
        "sphynx_precond_setup": (C.c_int, [vp, C.POINTER(Options), pd]),
        "sphynx_poly_step": (C.c_int, [vp, i32, i32, vp, i32, vp, vp, i32, i32, dbl, dbl, i32, i32]),
        "sphynx_precond_apply": (C.c_int, [vp, C.POINTER(Options), vp, vp, i32, i32]),
        "sphynx_gram": (C.c_int, [i32, C.POINTER(vp), C.POINTER(vp), i32, i32, i64, vp, pd, pd, vp]),
        "sphynx_rayleigh_ritz": (C.c_int, [pd, pd, pi32, i32, i32, dbl, pd, pd, pi32, vp]),
        "sphynx_eigensolve": (C.c_int, [vp, C.POINTER(Options), i32, pd, vp, i32, pd, pd, C.POINTER(Stats)]),
        "sphynx_mj": (C.c_int, [i32, vp, i32, i32, i64, vp, i32, vp, vp]),
        "sphynx_mj_noalloc": (C.c_int, [i32, vp, i32, i32, i64, vp, i32, vp, vp]),
        "sphynx_set_spmm_med_max": (C.c_int, [vp, i32]),
        "sphynx_amg_level": (C.c_int, [vp, i32, C.POINTER(AmgLevelInfo), vp, vp, vp, vp]),
        "sphynx_default_options_for": (C.c_int, [vp, i32, C.POINTER(Options)]),
        "sphynx_create_batch": (C.c_int, [vp, vp, vp, vp, vp, i32, i64, i64, C.c_uint32, vp, C.POINTER(vp)]),
        "sphynx_partition_batch": (C.c_int, [vp, i32, C.POINTER(Options), vp, vp, vp, vp, vp, vp, C.POINTER(Stats)]),
        "sphynx_eval": (C.c_int, [vp, vp, i32, pd, pd, pd]),
        "sphynx_refine": (C.c_int, [vp, vp, i32, dbl, i32, pd, pd, pi32, pi32]),
        "sphynx_partition": (C.c_int, [vp, i32, C.POINTER(Options), vp, pd, pd, C.POINTER(Stats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


class SphynxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sphynx error {code}: {msg}")
        self.code = code


def last_error() -> str:
    return (LIB.sphynx_last_error() or b"").decode()


def check(code: int, allow=()) -> int:
    if code != OK and code not in allow:
        raise SphynxError(code, last_error())
    return code


def ptr(x) -> int | None:
    """Address of a torch tensor / numpy array / integer pointer (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return x.ctypes.data
    raise TypeError(type(x))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def options(laplacian="combinatorial", precond="jacobi", poly_degree=25, precision="fp64", init="random",
            max_iter=1000, tol=1e-3, seed=1, out_device=False, sync_every=0, stall_window=0,
            conv="rel_theta", refine_rounds=0) -> Options:
    o = Options()
    LIB.sphynx_default_options(C.byref(o))
    o.laplacian = LAPLACIANS.get(laplacian, laplacian)
    o.precond = PRECONDS.get(precond, precond)
    o.poly_degree = poly_degree
    o.precision = PRECISIONS.get(precision, precision)
    o.init = INITS.get(init, init)
    o.max_iter = max_iter
    o.tol = tol
    o.seed = seed
    o.flags = OUT_DEVICE if out_device else 0
    o.sync_every = sync_every
    o.stall_window = stall_window
    o.conv = CONVS.get(conv, conv)
    o.refine_rounds = refine_rounds
    return o


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


# ---- thin wrappers, same names as the C ABI -----------------------------------

def sphynx_create(row_ptr, col, edge_w=None, vtx_w=None, n=None, nnz=None, flags=HOST_PTRS, stream=None) -> int:
    """Handle (an integer) for a CSR graph; host numpy arrays unless flags has DEVICE_PTRS."""
    if n is None:
        n = len(row_ptr) - 1
    if nnz is None:
        nnz = len(col)
    if not (flags & DEVICE_PTRS):
        def host(a, dt):
            return a if a is None or isinstance(a, int) or hasattr(a, "data_ptr") else np.ascontiguousarray(a, dt)
        row_ptr = host(row_ptr, np.int64)
        col = host(col, np.int32)
        edge_w = host(edge_w, np.float32)
        vtx_w = host(vtx_w, np.int64)
    h = C.c_void_p()
    check(LIB.sphynx_create(ptr(row_ptr), ptr(col), ptr(edge_w), ptr(vtx_w), int(n), int(nnz), int(flags),
                            _stream(stream), C.byref(h)))
    return h.value


def sphynx_destroy(h) -> None:
    LIB.sphynx_destroy(h)


def sphynx_get_info(h) -> dict:
    info = GraphInfo()
    check(LIB.sphynx_get_info(h, C.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def sphynx_set_spmm_variant(h, variant: int) -> None:
    check(LIB.sphynx_set_spmm_variant(h, variant))


def sphynx_set_spmm_sell_stride(h, stride: int) -> None:
    check(LIB.sphynx_set_spmm_sell_stride(h, stride))


def sphynx_set_spmm_med_max(h, med_max: int) -> None:
    check(LIB.sphynx_set_spmm_med_max(h, med_max))


def sphynx_degrees(h, deg_out) -> None:
    check(LIB.sphynx_degrees(h, ptr(deg_out)))


def sphynx_laplacian_apply(h, laplacian, dtype, x, ldx, y, ldy, ncols) -> None:
    check(LIB.sphynx_laplacian_apply(h, LAPLACIANS.get(laplacian, laplacian), dtype, ptr(x), ldx, ptr(y), ldy,
                                     ncols))


def sphynx_poly_step(h, laplacian, dtype_in, t, dtype_out, t_out, y, ld, ncols, theta_cur, theta_next, yterms,
                     first=0) -> None:
    check(LIB.sphynx_poly_step(h, LAPLACIANS.get(laplacian, laplacian), dtype_in, ptr(t), dtype_out, ptr(t_out),
                               ptr(y), ld, ncols, float(theta_cur), float(theta_next), yterms, first))


MAX_ADDED_ROOTS = 5


def sphynx_precond_setup(h, opt: Options) -> np.ndarray:
    """Set up the preconditioner; for the polynomial, its roots in application
    order (the degree plus any roots added to keep it positive)."""
    roots = np.zeros(max(1, opt.poly_degree) + MAX_ADDED_ROOTS)
    check(LIB.sphynx_precond_setup(h, C.byref(opt), _dptr(roots)))
    return roots[np.isfinite(roots)] if opt.precond == PRECOND_POLY else np.zeros(0)


def sphynx_precond_apply(h, opt: Options, r, hout, ld, ncols) -> None:
    check(LIB.sphynx_precond_apply(h, C.byref(opt), ptr(r), ptr(hout), ld, ncols))


def sphynx_amg_level(h, level: int, agg=None, row_ptr=None, col=None, w=None) -> dict:
    """Sizes of one multigrid level; fills the given device tensors (agg int32[n],
    row_ptr int64[n + 1], col int32[nnz], w float32[nnz])."""
    info = AmgLevelInfo()
    check(LIB.sphynx_amg_level(h, level, C.byref(info), ptr(agg), ptr(row_ptr), ptr(col), ptr(w)))
    return {f: getattr(info, f) for f, _ in info._fields_ if f != "reserved"}


def sphynx_gram(dtype, s_blocks, ls_blocks, ld, n, bdiag=None, stream=None):
    nblk = len(s_blocks)
    m = nblk * ld
    ga = np.zeros((m, m))
    gb = np.zeros((m, m))
    sp = (C.c_void_p * 3)(*[ptr(b) for b in s_blocks] + [None] * (3 - nblk))
    lp = (C.c_void_p * 3)(*[ptr(b) for b in ls_blocks] + [None] * (3 - nblk))
    check(LIB.sphynx_gram(dtype, sp, lp, nblk, ld, int(n), ptr(bdiag), _dptr(ga), _dptr(gb), _stream(stream)))
    return ga, gb


def sphynx_rayleigh_ritz(ga, gb, active, nev, u_work, stream=None):
    ga = np.ascontiguousarray(ga, dtype=np.float64)
    gb = np.ascontiguousarray(gb, dtype=np.float64)
    m = ga.shape[0]
    act = np.ascontiguousarray(active, dtype=np.int32)
    theta = np.zeros(nev)
    y = np.zeros((m, nev))
    sv = C.c_int32(0)
    check(LIB.sphynx_rayleigh_ritz(_dptr(ga), _dptr(gb), act.ctypes.data_as(C.POINTER(C.c_int32)), m, nev,
                                   float(u_work), _dptr(theta), _dptr(y), C.byref(sv), _stream(stream)))
    return theta, y, bool(sv.value)


def sphynx_eigensolve(h, opt: Options, nev, x_out, ldx, x0=None):
    theta = np.zeros(nev)
    res = np.zeros(nev)
    st = Stats()
    x0p = None
    if x0 is not None:
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        x0p = _dptr(x0)
    code = check(LIB.sphynx_eigensolve(h, C.byref(opt), nev, x0p, ptr(x_out), ldx, _dptr(theta), _dptr(res),
                                       C.byref(st)), allow=(ERR_NOCONV, ERR_BREAKDOWN))
    return code, theta, res, st.as_dict()


def sphynx_mj(dtype, coords, ldc, dims, n, vtx_w, K, part_out, stream=None) -> None:
    check(LIB.sphynx_mj(dtype, ptr(coords), ldc, dims, int(n), ptr(vtx_w), K, ptr(part_out), _stream(stream)))


def sphynx_mj_noalloc(dtype, coords, ldc, dims, n, vtx_w, K, part_out, stream=None) -> None:
    """sphynx_mj with its scratch in the library's fixed device array: for
    callers that cannot let the library allocate device memory."""
    check(LIB.sphynx_mj_noalloc(dtype, ptr(coords), ldc, dims, int(n), ptr(vtx_w), K, ptr(part_out),
                                _stream(stream)))


def sphynx_refine(h, part, K, eps=0.01, max_rounds=20):
    """Greedy refinement of the device partition `part` in place; returns
    (cut, imbalance, moves, rounds)."""
    cut, imb = C.c_double(), C.c_double()
    mv, rd = C.c_int32(), C.c_int32()
    check(LIB.sphynx_refine(h, ptr(part), K, float(eps), max_rounds, C.byref(cut), C.byref(imb), C.byref(mv),
                            C.byref(rd)))
    return cut.value, imb.value, mv.value, rd.value


def sphynx_eval(h, part, K):
    cut, cut2, imb = C.c_double(), C.c_double(), C.c_double()
    check(LIB.sphynx_eval(h, ptr(part), K, C.byref(cut), C.byref(cut2), C.byref(imb)))
    return cut.value, cut2.value, imb.value


def sphynx_partition(h, K, opt: Options, part_out):
    """Algorithm 2; part_out is a host int32 array (or a device tensor with OUT_DEVICE)."""
    cut, imb = C.c_double(), C.c_double()
    st = Stats()
    code = check(LIB.sphynx_partition(h, K, C.byref(opt), ptr(part_out), C.byref(cut), C.byref(imb), C.byref(st)),
                 allow=(ERR_NOCONV, ERR_BREAKDOWN))
    return code, cut.value, imb.value, st.as_dict()


def sphynx_default_options_for(h, precond: str = "jacobi") -> "Options":
    """Sphynx's defaults for this graph and preconditioner (Sec. 6.3.1)."""
    o = Options()
    check(LIB.sphynx_default_options_for(h, PRECONDS[precond], C.byref(o)))
    return o


def sphynx_create_batch(row_ptr, col, graph_ptr, edge_w=None, vtx_w=None, flags=HOST_PTRS, stream=None,
                        nnz=None) -> int:
    """Batch handle over a block-diagonal CSR; graph_ptr (host int64[count + 1])
    gives each graph's vertex range.  nnz is needed when the arrays are given
    as raw addresses."""
    graph_ptr = np.ascontiguousarray(graph_ptr, np.int64)
    n = int(graph_ptr[-1])
    if nnz is None:
        nnz = len(col)
    if not (flags & DEVICE_PTRS) and not isinstance(col, int):
        row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        col = np.ascontiguousarray(col, np.int32)
        edge_w = None if edge_w is None else np.ascontiguousarray(edge_w, np.float32)
        vtx_w = None if vtx_w is None else np.ascontiguousarray(vtx_w, np.int64)
    h = C.c_void_p()
    check(LIB.sphynx_create_batch(ptr(row_ptr), ptr(col), ptr(edge_w), ptr(vtx_w), ptr(graph_ptr),
                                  len(graph_ptr) - 1, n, int(nnz), int(flags), _stream(stream), C.byref(h)))
    return h.value


def sphynx_partition_batch(h, K, opt: Options, part_out, count):
    """Partition every graph of a batch handle; returns (code, cuts, imbalances,
    eigenvalues [count x d], iterations, status, stats) with per-graph numpy arrays."""
    d = int(K).bit_length()
    cuts = np.zeros(count)
    imbs = np.zeros(count)
    eigs = np.zeros((count, d))
    iters = np.zeros(count, dtype=np.int32)
    status = np.zeros(count, dtype=np.int32)
    st = Stats()
    code = check(LIB.sphynx_partition_batch(h, K, C.byref(opt), ptr(part_out), ptr(cuts), ptr(imbs), ptr(eigs),
                                            ptr(iters), ptr(status), C.byref(st)))
    return code, cuts, imbs, eigs, iters, status, st.as_dict()


class Graph:
    """Owning wrapper of a handle built from a workloads.CSRGraph (host arrays)."""

    def __init__(self, g, vtx_w=None, validate=False, stream=None):
        self.n = g.n
        self.nnz = g.nnz
        self.h = sphynx_create(g.row_ptr, g.col, g.w, vtx_w, g.n, g.nnz,
                               HOST_PTRS | (VALIDATE if validate else 0), stream)

    def close(self):
        if self.h:
            sphynx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def partition(self, K, **kw):
        parts = np.zeros(self.n, dtype=np.int32)
        code, cut, imb, st = sphynx_partition(self.h, K, options(**kw), parts)
        return parts, cut, imb, st, code
