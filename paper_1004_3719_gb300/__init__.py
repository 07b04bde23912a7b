"""Exact sparse matrix x vector / block products over Z/mZ on GB300.

A thin Python binding of ``libffspmv.so`` (declared in ``include/ffspmv.h``):
it marshals arguments only.  Every step of the computation runs in the CUDA
kernels behind the C ABI; PyTorch provides device memory and streams.  There
is no CPU fallback: if the library is missing or no CUDA device is present,
the calls raise.

    import paper_1004_3719_gb300 as ff
    ff.build()                                    # compile libffspmv.so (sm_103a)
    A = ff.Matrix(nrows, ncols, row_ptr, col, val, m)
    y = A.apply(x)                                # y = A x mod m
    z = A.apply_transpose(y)                      # z = A^T y mod m
    S = A.block_sequence(X, Y, nsteps)            # S_i = X^T A^i Y mod m
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _build
from ._lib import (FMT, SEL, TRANSPOSE, FFSPMVError, Options, lib,  # noqa: F401
                   options_default, status_string)
from ._api import (Matrix, spmv_apply, spmv_apply_transpose,  # noqa: F401
                   spmv_apply_transpose_noalloc,
                   spmv_batch_apply, spmv_block_project, spmv_block_project_finish,
                   spmv_block_sequence, spmv_create_hybrid,
                   polymat_mul, sigma_basis, sigma_generator_degrees, sigma_wiedemann_input,
                   spmv_apply_gf2, spmv_check_status,
                   spmv_count_launches, spmv_describe_plan,
                   spmv_destroy, spmv_get_info, stream_ptr, to_numpy_u32)

__all__ = ["build", "Matrix", "Options", "FMT", "SEL", "TRANSPOSE", "FFSPMVError",
           "spmv_create_hybrid", "spmv_apply", "spmv_apply_transpose",
           "spmv_apply_transpose_noalloc",
           "spmv_block_sequence", "spmv_block_project", "spmv_block_project_finish",
           "spmv_batch_apply", "spmv_destroy",
           "spmv_describe_plan", "spmv_get_info", "spmv_count_launches",
           "spmv_check_status", "spmv_apply_gf2", "polymat_mul", "sigma_basis", "sigma_generator_degrees",
           "sigma_wiedemann_input",
           "options_default", "to_numpy_u32",
           "status_string", "library_path"]


def build(force=False):
    """Compile libffspmv.so for sm_103a if it is missing or stale."""
    return _build.build(force=force)


def library_path():
    return _build.OUT
