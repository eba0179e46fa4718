"""Host-side checks of the C ABI: the library builds, loads, exports every
entry point include/sphynx.h declares, and its host-only calls behave.  No
call here touches a GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sphynx.h")


@pytest.fixture(scope="module", autouse=True)
def lib_path():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_sphynx_build", os.path.join(ROOT, "paper_2105_00578_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sphynx_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sphynx_create", "sphynx_partition", "sphynx_eval", "sphynx_destroy", "sphynx_last_error",
                     "sphynx_laplacian_apply", "sphynx_mj", "sphynx_gram", "sphynx_rayleigh_ritz",
                     "sphynx_eigensolve", "sphynx_precond_setup", "sphynx_precond_apply", "sphynx_poly_step",
                     "sphynx_mj_noalloc"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options_and_error_string(lib_path):
    import paper_2105_00578_gb300 as spx
    o = spx.Options()
    spx.LIB.sphynx_default_options(ctypes.byref(o))
    assert (o.laplacian, o.precond, o.poly_degree, o.precision, o.init, o.max_iter) == (
        spx.COMBINATORIAL, spx.PRECOND_JACOBI, 25, spx.FP64, spx.INIT_RANDOM, 1000)
    assert o.tol == 1e-3
    assert o.conv == spx.CONV_REL_THETA and o.stall_window == 0
    assert spx.last_error() == ""
    # struct layouts agree with the header's field order and sizes
    assert ctypes.sizeof(spx.Options) == 4 * 6 + 8 + 8 + 4 + 4 + 4 * 6
    assert spx.Stats.ms_total.offset == 16 + 16 * 8 * 2


def test_options_helper_maps_names():
    import paper_2105_00578_gb300 as spx
    o = spx.options(laplacian="generalized", precond="poly", precision="mixed_bf16", init="piecewise", tol=1e-2)
    assert (o.laplacian, o.precond, o.precision, o.init) == (spx.GENERALIZED, spx.PRECOND_POLY, spx.MIXED_BF16,
                                                           spx.INIT_PIECEWISE)


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every field offset and the size of the public structs, as the C
    compiler lays them out from the header, equal the Python binding's."""
    import shutil
    import subprocess
    import paper_2105_00578_gb300 as spx
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sphynx_options": spx.Options, "sphynx_stats": spx.Stats, "sphynx_graph_info": spx.GraphInfo,
               "sphynx_amg_level_info": spx.AmgLevelInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sphynx.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
