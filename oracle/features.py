"""Features of a sparse matrix for the format selector, in float64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).  These are the
definitions the device feature kernel must reproduce.

Matrix features f[0..15] (n = rows, N = columns, L_i = row lengths, nnz = sum
L_i, mean = nnz / n, "+-1" = value mod m equal to 1 or m-1):
  0 log2(n)/32              1 log2(N)/32             2 log2(1+mean)/16
  3 min(std(L)/mean, 10)/10 4 log2(1+max L)/32       5 share of empty rows
  6 share of rows with 1 <= L <= 4                   7 share of rows with L >= 64
  8 share of +-1 entries    9 log2(m)/32             10 share with |j-i| <= 64
 11 share with j == i      12 share with |j-i| <= max(1, max(n,N)//64)
 13 mean |j-i| / max(n,N)  14 skewness of L clipped to [-10,10], /10
 15 share of entries on diagonals holding at least half their length
Bin features g[b][0..5] for the 17 row-length bins of the binned layout
(bin 0: L = 0; bin b: 2^(b-2) < L <= 2^(b-1), bin 16 also the longer rows):
  0 b/16  1 rows share  2 nnz share  3 +-1 share in the bin
  4 (nnz_b/rows_b)/2^(b-1)  5 log2(1+rows_b)/32
"""
from __future__ import annotations

import numpy as np

NUM_BINS = 17


def bin_of_length(L):
    L = np.asarray(L, dtype=np.int64)
    b = np.zeros(L.shape, dtype=np.int64)
    pos = L > 0
    # smallest b >= 1 with 2^(b-1) >= L, capped at 16
    b[pos] = 1 + np.ceil(np.log2(L[pos].astype(np.float64))).astype(np.int64)
    # guard against log2 rounding at exact powers of two
    u = np.where(pos, 2 ** np.maximum(b - 1, 0), 0)
    b = np.where(pos & (u < L), b + 1, b)
    b = np.where(pos & (b > 1) & (2 ** np.maximum(b - 2, 0) >= L), b - 1, b)
    return np.minimum(b, NUM_BINS - 1)


def features(nrows, ncols, row_ptr, col, val, m):
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.uint64) % np.uint64(m)
    L = np.diff(row_ptr)
    nnz = int(L.sum())
    n = max(nrows, 1)
    nz = max(nnz, 1)
    mean = nnz / n
    ex2 = float((L.astype(np.float64) ** 2).sum()) / n
    ex3 = float((L.astype(np.float64) ** 3).sum()) / n
    var = max(ex2 - mean * mean, 0.0)
    sd = np.sqrt(var)
    cv = min(sd / mean, 10.0) if mean > 0 else 0.0
    sk = 0.0
    if sd > 0:
        sk = (ex3 - 3 * mean * ex2 + 2 * mean ** 3) / sd ** 3
        sk = float(np.clip(sk, -10, 10))
    rows = np.repeat(np.arange(nrows, dtype=np.int64), L)
    d = col - rows
    ad = np.abs(d)
    pm = (val == 1) | ((m > 2) & (val == np.uint64(m - 1)))
    big = max(nrows, ncols, 1)
    local = max(1, max(nrows, ncols) // 64)
    half = 0
    if nnz:
        cnt = np.bincount(d + nrows - 1, minlength=nrows + ncols - 1)
        off = np.arange(cnt.size) - (nrows - 1)
        length = np.where(off >= 0, np.minimum(nrows, ncols - off), np.minimum(nrows + off, ncols))
        half = int(cnt[(cnt > 0) & (2 * cnt >= length)].sum())
    f = np.array([
        np.log2(n) / 32, np.log2(max(ncols, 1)) / 32, np.log2(1 + mean) / 16, cv / 10,
        np.log2(1 + (L.max() if nrows else 0)) / 32, (L == 0).sum() / n,
        ((L > 0) & (L <= 4)).sum() / n, (L >= 64).sum() / n, pm.sum() / nz, np.log2(m) / 32,
        (ad <= 64).sum() / nz, (d == 0).sum() / nz, (ad <= local).sum() / nz,
        (ad.sum() / nz) / big, sk / 10, half / nz], dtype=np.float64)
    b = bin_of_length(L)
    g = np.zeros((NUM_BINS, 6), dtype=np.float64)
    pm_row = np.zeros(nrows, dtype=np.int64)
    if nnz:
        np.add.at(pm_row, rows, pm.astype(np.int64))
    for k in range(NUM_BINS):
        sel = b == k
        r = int(sel.sum())
        z = int(L[sel].sum())
        g[k] = [k / 16, r / n, z / nz, (pm_row[sel].sum() / z) if z else 0.0,
                ((z / r) / 2 ** (k - 1)) if (k > 0 and r > 0) else 0.0, np.log2(1 + r) / 32]
    return f, g
