"""Loader for the native generator helpers in ``_gen.c`` (built with gcc on
first use into ``workloads/_lib/``).  ``lib()`` returns None when no C
compiler is available; the numpy code in graphs.py then does the work."""

from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "_gen.c")
_LOCK = threading.Lock()
_LIB = None
_TRIED = False


def _build() -> str | None:
    out_dir = os.path.join(_HERE, "_lib")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, f"libgen_{platform.machine()}.so")
    if os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(_SRC):
        return so
    base = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", _SRC, "-o", so + ".tmp"]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:1] + extra + base[1:], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(so + ".tmp", so)
            return so
    return None


def lib():
    global _LIB, _TRIED
    with _LOCK:
        if _TRIED:
            return _LIB
        _TRIED = True
        try:
            so = _build()
        except OSError:
            so = None
        if so is None:
            return None
        L = C.CDLL(so)
        i64, u64, dbl, vp = C.c_int64, C.c_uint64, C.c_double, C.c_void_p
        L.gen_rmat_keys.argtypes = [C.c_int, i64, dbl, dbl, dbl, u64, vp]
        L.gen_rmat_keys.restype = None
        L.gen_sort_unique.argtypes = [vp, vp, i64, C.c_int]
        L.gen_sort_unique.restype = i64
        L.gen_csr_from_keys.argtypes = [i64, vp, i64, vp, vp]
        L.gen_csr_from_keys.restype = C.c_int
        L.gen_components.argtypes = [i64, vp, vp, vp]
        L.gen_components.restype = i64
        L.gen_induced.argtypes = [i64, vp, vp, vp, vp, i64, vp, vp, vp]
        L.gen_induced.restype = i64
        L.gen_edge_weights.argtypes = [i64, vp, vp, dbl, dbl, u64, vp]
        L.gen_edge_weights.restype = None
        L.gen_rgg_keys.argtypes = [i64, dbl, u64, vp, i64]
        L.gen_rgg_keys.restype = i64
        _LIB = L
        return _LIB
