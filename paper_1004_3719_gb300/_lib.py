"""ctypes declarations of the C ABI in include/ffspmv.h."""
from __future__ import annotations

import ctypes
import os

from . import _build


class FFSPMVError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        msg = status_string(self.status) if _lib_handle is not None else str(status)
        super().__init__(f"{where}: {msg} (status {self.status})" if where else msg)


class FMT:
    AUTO, CSR, ELLR, COO, COOS, DIA, HYBRID, BINNED, PANEL = range(9)


class SEL:
    HEURISTIC, LEARNED, EXHAUSTIVE, FIXED = range(4)


class TRANSPOSE:
    EXPLICIT, ATOMIC, NONE = range(3)


class Options(ctypes.Structure):
    _fields_ = [
        ("selector", ctypes.c_int32),
        ("use_pm1", ctypes.c_int32),
        ("priority_format", ctypes.c_int32),
        ("transpose_mode", ctypes.c_int32),
        ("value_check", ctypes.c_int32),
        ("group_width", ctypes.c_int32),
        ("ell_width", ctypes.c_int32),
        ("barrier_spin_limit", ctypes.c_uint32),
        ("guard_bytes", ctypes.c_int64),
        ("sequence_mode", ctypes.c_int32),
        ("test_hooks", ctypes.c_int32),
        ("panel_cluster", ctypes.c_int32),
    ]


_lib_handle = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_U32 = ctypes.c_uint32


def _declare(L):
    L.ffspmv_options_default.argtypes = [ctypes.POINTER(Options)]
    L.ffspmv_options_default.restype = None
    L.ffspmv_status_string.argtypes = [ctypes.c_int]
    L.ffspmv_status_string.restype = ctypes.c_char_p
    L.ffspmv_last_error.argtypes = []
    L.ffspmv_last_error.restype = ctypes.c_char_p
    L.spmv_create_hybrid.argtypes = [ctypes.POINTER(_P), _I64, _I64, _I64, _P, _P, _P,
                                     _U32, ctypes.POINTER(Options), _P]
    L.spmv_create_hybrid.restype = ctypes.c_int
    for f in (L.spmv_apply, L.spmv_apply_transpose):
        f.argtypes = [_P, _P, _I64, _P, _I64, _I32, _U32, _U32, _P]
        f.restype = ctypes.c_int
    L.spmv_block_sequence.argtypes = [_P, _P, _P, _I32, _I64, _I64, _P, _P, _P]
    L.spmv_block_sequence.restype = ctypes.c_int
    L.spmv_batch_apply.argtypes = [_I32, _P, _P, _P, _P, _P]
    L.spmv_batch_apply.restype = ctypes.c_int
    L.spmv_destroy.argtypes = [_P]
    L.spmv_destroy.restype = ctypes.c_int
    L.spmv_describe_plan.argtypes = [_P, ctypes.c_char_p, ctypes.c_size_t]
    L.spmv_describe_plan.restype = ctypes.c_int
    L.spmv_get_info.argtypes = [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                ctypes.POINTER(_I64), ctypes.POINTER(_U32),
                                ctypes.POINTER(_I64)]
    L.spmv_get_info.restype = ctypes.c_int
    L.spmv_apply_transpose_noalloc.argtypes = [_P, _P, _I64, _P, _I64, _I32, _U32, _U32, _P]
    L.spmv_apply_transpose_noalloc.restype = ctypes.c_int
    L.spmv_count_launches.argtypes = [_P, _I32, _I32, ctypes.POINTER(_I64)]
    L.spmv_count_launches.restype = ctypes.c_int
    L.ffspmv_panel_decode.argtypes = [_I64, _I64, _P, _P, _P, _U32, _I32, _I32, _I32, _I32, _I64, _P, _P, _P,
                                      ctypes.POINTER(_I64), _P]
    L.ffspmv_panel_decode.restype = ctypes.c_int
    L.spmv_check_status.argtypes = [_P, _P]
    L.spmv_check_status.restype = ctypes.c_int
    L.spmv_apply_gf2.argtypes = [_P, _I32, _P, _P, _I32, _I32, _P]
    L.spmv_apply_gf2.restype = ctypes.c_int
    L.polymat_mul_workspace.argtypes = [_I32, _I64, _I64, ctypes.POINTER(_I64)]
    L.polymat_mul_workspace.restype = ctypes.c_int
    L.polymat_mul.argtypes = [_U32, _I32, _I64, _I64, _P, _P, _P, _P, _I64, _P]
    L.polymat_mul.restype = ctypes.c_int
    L.sigma_basis_workspace.argtypes = [_I32, _I32, _I64, _I32, ctypes.POINTER(_I64)]
    L.sigma_basis_workspace.restype = ctypes.c_int
    L.sigma_basis.argtypes = [_U32, _I32, _I32, _I64, _I32, _P, _P, _P, _P, _P, _P, _I64, _P]
    L.sigma_basis.restype = ctypes.c_int
    L.sigma_wiedemann_input.argtypes = [_U32, _I32, _I64, _P, _P, _P]
    L.sigma_wiedemann_input.restype = ctypes.c_int
    L.sigma_generator_degrees.argtypes = [_U32, _I32, _I32, _I64, _P, _P, _I32, ctypes.POINTER(_I64),
                                          ctypes.POINTER(_I64), _P]
    L.sigma_generator_degrees.restype = ctypes.c_int
    L.spmv_block_project.argtypes = [_U32, _I64, _I32, _P, _P, _P, _P]
    L.spmv_block_project.restype = ctypes.c_int
    L.spmv_block_project_finish.argtypes = [_U32, _I32, _P, _P, _P]
    L.spmv_block_project_finish.restype = ctypes.c_int
    for name, args, res in EXTRA_SIGNATURES:
        if hasattr(L, name):
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res


_F = ctypes.c_float
# Entry points declared in include/ffspmv_select.h.
EXTRA_SIGNATURES = [
    ("ffspmv_matrix_features", [_I64, _I64, _P, _P, _P, _U32, _P, _P, _P], ctypes.c_int),
    ("ffspmv_tune_bins", [_I64, _I64, _I64, _P, _P, _P, _U32, _I32, _I64, _I32, _P, _P, _P, _P],
     ctypes.c_int),
    ("ffspmv_mlp_forward", [_P, _P, _I32, _P, _P, _P], ctypes.c_int),
    ("ffspmv_mlp_loss", [_P, _P, _P, _I32, _P, _P, _P], ctypes.c_int),
    ("ffspmv_mlp_backward", [_P, _P, _I32, _P, _P, _P, _P], ctypes.c_int),
    ("ffspmv_mlp_adam", [_P, _P, _P, _P, _I32, _F, _F, _F, _F, _P], ctypes.c_int),
    ("ffspmv_selector_load", [_P, _I64], ctypes.c_int),
    ("ffspmv_heuristic_choose", [_I64, _P, _P, _U32, _I32, _P], ctypes.c_int),
    ("ffspmv_selector_choose", [_I64, _I64, _I64, _P, _P, _P, _U32, _P, _P], ctypes.c_int),
    ("spmv_create_binned", [ctypes.POINTER(_P), _I64, _I64, _I64, _P, _P, _P, _U32, _P,
                            ctypes.POINTER(Options), _P], ctypes.c_int),
]

# Sizes of the selector network (include/ffspmv_select.h).
NUM_BINS = 17
NUM_FORMATS = 10
NUM_FEATURES = 16
NUM_BIN_FEATURES = 6
MLP_IN = NUM_FEATURES + NUM_BIN_FEATURES
MLP_HIDDEN = 64
MLP_OUT = NUM_FORMATS + 5
OUT_PM = NUM_FORMATS            # log(t_pm / t_nopm) of a bin
OUT_NETBINS = NUM_FORMATS + 1   # whole plan: log(t_binned_network / t_binned)
OUT_PANEL = NUM_FORMATS + 2     # whole plan: log(t_panel_q / t_binned), q = 1, 2, 4
MATRIX_INPUT = -1.0             # every bin feature of the matrix-level input
LAYOUT_BINNED, LAYOUT_NETBINS, LAYOUT_PANEL_Q1, LAYOUT_PANEL_Q2, LAYOUT_PANEL_Q4, LAYOUT_PANEL = range(6)
SEL_Q_MARGIN, SEL_NET_MARGIN = 0.05, 0.15   # log-ratio margins of the layout rule
SEL_VERIFY_MARGIN = 0.15                    # closer families are timed (FFSPMV_SEL_VERIFY_MARGIN)
MLP_PARAMS = (MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN
              + MLP_OUT * MLP_HIDDEN + MLP_OUT)
SELECTOR_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.npy")


def lib():
    """The loaded CUDA library.  Raises if it has not been built."""
    global _lib_handle
    if _lib_handle is None:
        path = _build.OUT
        if not os.path.exists(path):
            raise FFSPMVError(4, f"{os.path.basename(path)} is not built "
                              "(call paper_1004_3719_gb300.build())")
        L = ctypes.CDLL(path)
        _declare(L)
        _lib_handle = L
        _install_default_selector(L)
    return _lib_handle


def _install_default_selector(L):
    """Install the committed selector weights (written by train_selector.py)
    for FFSPMV_SEL_LEARNED, if the file exists."""
    if not os.path.exists(SELECTOR_WEIGHTS):
        return
    import numpy as np
    w = np.ascontiguousarray(np.load(SELECTOR_WEIGHTS), dtype=np.float32)
    if w.size == MLP_PARAMS:
        L.ffspmv_selector_load(w.ctypes.data, w.size)


def status_string(s):
    return lib().ffspmv_status_string(int(s)).decode()


def check(status, where):
    if status != 0:
        if status == 4:
            where = f"{where} [{lib().ffspmv_last_error().decode()}]"
        raise FFSPMVError(status, where)


def options_default(**kw):
    o = Options()
    lib().ffspmv_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o
