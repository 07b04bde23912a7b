"""Oracle for the products over GF(2) (Z/2Z) with bit-packed vectors.

TEST INFRASTRUCTURE ONLY (see the package docstring): the tests and the
benchmark's CPU-baseline leg are the only callers.

Over Z/2Z a block of vectors packs into machine words, 64 components per
64-bit word -- the bit-packed x and y that Sec. 2.5 and the conclusion list
for the binary case.  X is an ncols x w array of uint64, bit b of word k of
row j being component 64k + b of x_j; Y = A X has nrows x w words.  The
definition is Sec. 2's y_i = sum_j A_ij x_j with m = 2: a sum mod 2 is an
exclusive or, and A_ij is its residue mod 2, so entry (i, j) contributes x_j
exactly when its value is odd.  Repeated (i, j) pairs add up, as everywhere
in this library: an even number of odd copies cancels.
"""
from __future__ import annotations

import numpy as np


def _entries(nrows, row_ptr, col, val):
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    rows = np.repeat(np.arange(nrows, dtype=np.int64), np.diff(row_ptr))
    keep = (np.asarray(val, dtype=np.uint64) & np.uint64(1)) == 1
    return rows[keep], np.asarray(col, dtype=np.int64)[keep]


def spmv_gf2(nrows, ncols, row_ptr, col, val, X):
    """Y = A X over GF(2); X: (ncols, w) or (ncols,) uint64 words."""
    X = np.asarray(X, dtype=np.uint64)
    flat = X.ndim == 1
    X = X.reshape(ncols, -1)
    rows, cols = _entries(nrows, row_ptr, col, val)
    Y = np.zeros((nrows, X.shape[1]), dtype=np.uint64)
    np.bitwise_xor.at(Y, rows, X[cols])      # y_i ^= x_j for every odd entry
    return Y.reshape(-1) if flat else Y


def spmv_gf2_transpose(nrows, ncols, row_ptr, col, val, X):
    """Y = A^T X over GF(2); X: (nrows, w) words, Y: (ncols, w)."""
    X = np.asarray(X, dtype=np.uint64)
    flat = X.ndim == 1
    X = X.reshape(nrows, -1)
    rows, cols = _entries(nrows, row_ptr, col, val)
    Y = np.zeros((ncols, X.shape[1]), dtype=np.uint64)
    np.bitwise_xor.at(Y, cols, X[rows])      # y_j ^= x_i
    return Y.reshape(-1) if flat else Y


def csr_gf2(A, X, transpose=False):
    f = spmv_gf2_transpose if transpose else spmv_gf2
    return f(A.nrows, A.ncols, A.row_ptr, A.col, A.val, X)


def unpack_bits(X):
    """(rows, w) uint64 words -> (rows, 64 w) array of 0/1 (component 64k + b)."""
    X = np.asarray(X, dtype=np.uint64).reshape(X.shape[0], -1)
    b = (X[:, :, None] >> np.arange(64, dtype=np.uint64)[None, None, :]) & np.uint64(1)
    return b.reshape(X.shape[0], -1).astype(np.uint8)


def pack_bits(B):
    """Inverse of unpack_bits: (rows, 64 w) of 0/1 -> (rows, w) uint64."""
    B = np.asarray(B, dtype=np.uint64).reshape(B.shape[0], -1, 64)
    return (B << np.arange(64, dtype=np.uint64)[None, None, :]).sum(axis=2, dtype=np.uint64)
