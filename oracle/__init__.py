"""CPU oracle for the exact sparse products over Z/mZ.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library neither
imports nor links anything here, and nothing here imports the library.

``oracle.c`` holds the plain definitions (128-bit exact sums, one ``%`` per
output); this module compiles it with gcc on first use and marshals numpy
arrays into it.  ``linalg`` (rank, Berlekamp-Massey), ``mlp`` (the selector
network in fp64) and ``features`` are further oracle pieces in pure numpy /
Python.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile ``oracle.c`` into ``liboracle.so`` (plain gcc, -O2)."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                            "-o", tmp, _SRC], check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        i64, i32, u32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        sig = [i64, i64, p, p, p, u32, p, i64, p, i64, i32, u32, u32]
        lib.oracle_spmv.argtypes = sig
        lib.oracle_spmv.restype = ctypes.c_int
        lib.oracle_spmv_transpose.argtypes = sig
        lib.oracle_spmv_transpose.restype = ctypes.c_int
        lib.oracle_block_sequence.argtypes = [i64, p, p, p, u32, p, p, i32,
                                              i64, p, p]
        lib.oracle_block_sequence.restype = ctypes.c_int
        for f in (lib.oracle_spmv_threads, lib.oracle_spmv_transpose_threads):
            f.argtypes = [i32] + sig
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _csr_arrays(row_ptr, col, val):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.uint32)
    return row_ptr, col, val


def _block(x, rows):
    x = np.ascontiguousarray(x, dtype=np.uint32)
    if x.ndim == 1:
        x = x.reshape(rows, 1)
    return x


def spmv(nrows, ncols, row_ptr, col, val, m, x, y=None, alpha=1, beta=0, threads=1):
    """y <- alpha*A*x + beta*y mod m (Sec. 2).  ``x`` is ncols or
    ncols x nvec; returns a new array shaped like ``x`` with nrows rows.
    ``threads`` > 1 splits the rows over that many host threads (timing)."""
    row_ptr, col, val = _csr_arrays(row_ptr, col, val)
    flat = np.asarray(x).ndim == 1
    xb = _block(x, ncols)
    nvec = xb.shape[1]
    out = (np.zeros((nrows, nvec), dtype=np.uint32) if y is None else
           _block(np.array(y, dtype=np.uint32, copy=True), nrows))
    args = (nrows, ncols, _ptr(row_ptr), _ptr(col), _ptr(val), m, _ptr(xb), nvec,
            _ptr(out), nvec, nvec, alpha % m, beta % m)
    rc = (_load().oracle_spmv(*args) if threads <= 1 else
          _load().oracle_spmv_threads(int(threads), *args))
    if rc != 0:
        raise ValueError(f"oracle_spmv failed ({rc})")
    return out.reshape(nrows) if flat else out


def spmv_transpose(nrows, ncols, row_ptr, col, val, m, x, y=None, alpha=1,
                   beta=0, threads=1):
    """y <- alpha*A^T*x + beta*y mod m.  ``x`` has nrows rows, the result
    ncols rows."""
    row_ptr, col, val = _csr_arrays(row_ptr, col, val)
    flat = np.asarray(x).ndim == 1
    xb = _block(x, nrows)
    nvec = xb.shape[1]
    out = (np.zeros((ncols, nvec), dtype=np.uint32) if y is None else
           _block(np.array(y, dtype=np.uint32, copy=True), ncols))
    args = (nrows, ncols, _ptr(row_ptr), _ptr(col), _ptr(val), m, _ptr(xb), nvec,
            _ptr(out), nvec, nvec, alpha % m, beta % m)
    rc = (_load().oracle_spmv_transpose(*args) if threads <= 1 else
          _load().oracle_spmv_transpose_threads(int(threads), *args))
    if rc != 0:
        raise ValueError(f"oracle_spmv_transpose failed ({rc})")
    return out.reshape(ncols) if flat else out


def block_sequence(n, row_ptr, col, val, p, X, Y, nsteps, want_next=False):
    """S_i = X^T A^i Y mod p for 0 <= i < nsteps (Sec. 3, step 1).  Returns
    S (nsteps x s x s) and, with ``want_next``, A^nsteps Y."""
    row_ptr, col, val = _csr_arrays(row_ptr, col, val)
    X = _block(X, n)
    Y = _block(Y, n)
    s = X.shape[1]
    if Y.shape != X.shape:
        raise ValueError("X and Y must both be n x s")
    S = np.zeros((nsteps, s, s), dtype=np.uint32)
    Vn = np.zeros((n, s), dtype=np.uint32) if want_next else None
    rc = _load().oracle_block_sequence(
        n, _ptr(row_ptr), _ptr(col), _ptr(val), p, _ptr(X), _ptr(Y), s, nsteps,
        _ptr(S), _ptr(Vn) if want_next else ctypes.c_void_p(0))
    if rc != 0:
        raise ValueError(f"oracle_block_sequence failed ({rc})")
    return (S, Vn) if want_next else S


def csr_spmv(A, x, **kw):
    """``spmv`` on an object with nrows/ncols/row_ptr/col/val/modulus."""
    m = kw.pop("m", A.modulus)
    return spmv(A.nrows, A.ncols, A.row_ptr, A.col, A.val, m, x, **kw)


def csr_spmv_transpose(A, x, **kw):
    m = kw.pop("m", A.modulus)
    return spmv_transpose(A.nrows, A.ncols, A.row_ptr, A.col, A.val, m, x,
                          **kw)


def csr_block_sequence(A, X, Y, nsteps, **kw):
    p = kw.pop("p", A.modulus)
    return block_sequence(A.nrows, A.row_ptr, A.col, A.val, p, X, Y, nsteps,
                          **kw)
