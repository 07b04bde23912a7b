"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/*.h declares; no compute call is made."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith(("spmv_", "ffspmv_", "polymat_", "sigma_")) and not name.endswith("_t"):
                names.add(name)
    return names


def test_headers_declare_the_boundary():
    names = declared_functions()
    for want in ("spmv_create_hybrid", "spmv_apply", "spmv_apply_transpose",
                 "spmv_block_sequence", "spmv_batch_apply", "spmv_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol():
    import paper_1004_3719_gb300 as ff
    path = ff.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_host_side_argument_errors_without_gpu():
    # these return before any CUDA call is made
    import paper_1004_3719_gb300 as ff
    ff.build()
    L = ff.lib()
    h = ctypes.c_void_p()
    assert L.spmv_create_hybrid(None, 1, 1, 0, None, None, None, 7, None, None) == 1
    assert L.spmv_create_hybrid(ctypes.byref(h), -1, 1, 0, None, None, None, 7, None, None) == 1
    assert L.spmv_apply(None, None, 1, None, 1, 1, 1, 0, None) == 1
    assert L.spmv_block_sequence(None, None, None, 16, 0, 10, None, None, None) == 1
    assert L.spmv_batch_apply(-1, None, None, None, None, None) == 1
    assert L.spmv_apply_gf2(None, 0, None, None, 1, 0, None) == 1
    assert L.spmv_check_status(None, None) == 1
    n = ctypes.c_int64()
    assert L.polymat_mul_workspace(0, 1, 1, ctypes.byref(n)) == 1          # s >= 1
    assert L.polymat_mul_workspace(33, 1, 1, ctypes.byref(n)) == 1         # s <= 32
    assert L.polymat_mul_workspace(4, -1, 1, ctypes.byref(n)) == 1         # degrees >= 0
    assert L.polymat_mul_workspace(4, 2**14, 2**14, ctypes.byref(n)) == 5  # length past 2^15
    assert L.polymat_mul_workspace(16, 6250, 6250, ctypes.byref(n)) == 0
    assert n.value == 3 * 3 * 256 * 16384 * 4 + 3 * 16384 * 8 + 256
    assert L.polymat_mul(1, 4, 1, 1, None, None, None, None, 0, None) == 1  # p >= 2, pointers
    assert L.sigma_basis_workspace(33, 16, 10, 0, ctypes.byref(n)) == 1      # m <= 32
    assert L.sigma_basis_workspace(8, 9, 10, 0, ctypes.byref(n)) == 1        # n <= m
    assert L.sigma_basis_workspace(32, 32, 10, 33, ctypes.byref(n)) == 1     # leaf order <= 32
    assert L.sigma_basis_workspace(32, 32, 10, 32, ctypes.byref(n)) == 0     # a cluster holds any order-32 leaf
    assert L.sigma_basis_workspace(32, 16, 30000, 0, ctypes.byref(n)) == 5   # products past 2^15 points
    assert L.sigma_basis_workspace(32, 16, 12502, 0, ctypes.byref(n)) == 0
    d = ctypes.c_int32(0)
    assert L.sigma_basis(65521 * 3, 2, 1, 4, 0, 8, None, 8, ctypes.byref(d), None, 16, 1 << 20, None) == 1  # p prime
    assert L.sigma_basis(65521, 2, 1, 4, 0, None, None, 8, ctypes.byref(d), None, 16, 1 << 20, None) == 1   # pointers
    assert L.sigma_wiedemann_input(65521, 17, 4, 8, 8, None) == 1           # s <= 16
    dg, cd = ctypes.c_int64(), ctypes.c_int64()
    dl = (ctypes.c_int32 * 4)(0, 0, 0, 0)
    gd = L.sigma_generator_degrees
    assert gd(65521 * 3, 4, 2, 3, 8, dl, 0, ctypes.byref(dg), ctypes.byref(cd), None) == 1   # p prime
    assert gd(65521, 4, 5, 3, 8, dl, 0, ctypes.byref(dg), ctypes.byref(cd), None) == 1       # n <= m
    assert gd(65521, 33, 2, 3, 8, dl, 0, ctypes.byref(dg), ctypes.byref(cd), None) == 1      # m <= 32
    assert gd(65521, 4, 2, 3, None, dl, 0, ctypes.byref(dg), ctypes.byref(cd), None) == 1    # pointers
    assert gd(65521, 4, 2, 3, 8, dl, 1 << 17, ctypes.byref(dg), ctypes.byref(cd), None) == 1  # precision <= 2^16
    assert ff.status_string(6) == "device wait timed out"
    o = ff.options_default()
    assert o.use_pm1 == -1 and o.ell_width == -1 and o.transpose_mode == 0


def test_options_layout_matches_header():
    import paper_1004_3719_gb300 as ff
    text = open(os.path.join(ROOT, "include", "ffspmv.h")).read()
    body = text[text.index("typedef struct {"):text.index("} ffspmv_options;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:int32_t|uint32_t|int64_t)\s+([a-z_0-9]+)\s*;", body)
    assert fields == [f for f, _ in ff.Options._fields_]
