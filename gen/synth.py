"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random structure and residues.  It holds none of the
arithmetic of the method (no products, no reductions of sums, no formats): the
CPU oracle and the CUDA library both receive the arrays made here, unchanged.

The paper's own test matrices (Table "Matrices overview", Sec. 2.2) are not
available, so these generators stand in for them:

* ``tiny_matrix``       2000 x 2000, 10 distinct uniform columns per row,
                        values in Z/65521 with 20% forced to +-1.
* ``powerlaw_matrix``   1M x 1M, Zipf row lengths (mean 16, max 10 000),
                        distinct uniform columns; moduli 65521, 2^31-1, 3.
* ``wiedemann_matrix``  100k x 100k, 4 nonzero diagonals {0, +1, -1, +n/2}
                        plus 6 random entries per row (Sec. 3.1 workload).
* ``batch_problems``    256 square matrices of uneven size, structure and
                        prime modulus, each with 1-32 right-hand sides.
* ``selector_matrix``   the generated family used to train and evaluate the
                        format selector (banded, block-diagonal, uniform,
                        power-law; +-1 fraction 0-100%).

Every generator is keyed by an explicit seed; numpy's PCG64 stream is the
same on every platform, so the same seed gives the same matrix everywhere.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

M65521 = 65521
M31 = 2**31 - 1


@dataclasses.dataclass
class CSR:
    """A sparse matrix in compressed-row form (Sec. 2.1, CSR).

    ``row_ptr`` int64[nrows+1], ``col`` int32[nnz], ``val`` uint32[nnz];
    row i holds entries ``row_ptr[i] <= k < row_ptr[i+1]``.  Values are the
    residues in [0, modulus) the matrix is defined with.
    """

    nrows: int
    ncols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    modulus: int
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def rng_for(seed: int, *keys: int) -> np.random.Generator:
    """A PCG64 stream keyed by (seed, *keys)."""
    return np.random.default_rng([int(seed), *[int(k) for k in keys]])


def _csr_from_lengths(lengths: np.ndarray) -> np.ndarray:
    row_ptr = np.zeros(lengths.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    return row_ptr


def distinct_columns(rng, lengths, ncols, forbid=None, window=None):
    """Per row, ``lengths[i]`` distinct column indices, sorted ascending.

    ``window(rows)`` may return (lo, hi) arrays restricting row i's columns to
    [lo, hi); ``forbid(rows, cols)`` flags columns a row must not use.
    Collisions are redrawn until none remain.
    """
    lengths = np.asarray(lengths, dtype=np.int64)
    nrows = lengths.size
    if window is None and forbid is None and nrows:
        dense = lengths * 4 > ncols
        if dense.any():
            # rows filling a large share of the columns: sample them without
            # replacement directly, the rest by drawing and redrawing
            sparse_len = np.where(dense, 0, lengths)
            r_s, c_s = distinct_columns(rng, sparse_len, ncols)
            rows_d, cols_d = [r_s], [c_s.astype(np.int64)]
            for i in np.nonzero(dense)[0]:
                c = np.sort(rng.choice(ncols, int(lengths[i]), replace=False))
                rows_d.append(np.full(c.size, i, dtype=np.int64))
                cols_d.append(c.astype(np.int64))
            rows = np.concatenate(rows_d)
            cols = np.concatenate(cols_d)
            order = np.lexsort((cols, rows))
            return rows[order], cols[order].astype(np.int32)
    nnz = int(lengths.sum())
    rows = np.repeat(np.arange(nrows, dtype=np.int64), lengths)
    if window is None:
        lo = np.zeros(nnz, dtype=np.int64)
        span = np.full(nnz, ncols, dtype=np.int64)
    else:
        wlo, whi = window(np.arange(nrows, dtype=np.int64))
        lo = np.repeat(wlo, lengths)
        span = np.repeat(whi - wlo, lengths)
    if nnz and np.any(np.repeat(lengths, lengths) > span):
        raise ValueError("a row asks for more distinct columns than it may use")
    cols = lo + (rng.random(nnz) * span).astype(np.int64)
    cols = np.minimum(cols, lo + span - 1)
    for _ in range(10_000):
        key = rows * np.int64(ncols) + cols
        order = np.argsort(key, kind="stable")
        rows = rows[order]
        cols = cols[order]
        lo = lo[order]
        span = span[order]
        bad = np.zeros(nnz, dtype=bool)
        if nnz > 1:
            bad[1:] = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if forbid is not None:
            bad |= forbid(rows, cols)
        nb = int(bad.sum())
        if nb == 0:
            return rows, cols.astype(np.int32)
        cols[bad] = lo[bad] + np.minimum(
            (rng.random(nb) * span[bad]).astype(np.int64), span[bad] - 1)
    raise RuntimeError("could not draw distinct columns")


def residues(rng, count, m, pm_fraction=0.0):
    """Nonzero residues in [1, m-1]; a fraction ``pm_fraction`` is forced to
    +1 or -1 (= m-1) by a fair coin.  For m = 3 every nonzero is +-1."""
    count = int(count)
    if m < 2:
        raise ValueError("modulus must be >= 2")
    if m == 2:
        return np.ones(count, dtype=np.uint32)
    v = 1 + (rng.random(count) * (m - 1)).astype(np.uint64)
    v = np.minimum(v, m - 1)
    if pm_fraction > 0:
        forced = rng.random(count) < pm_fraction
        sign = rng.random(count) < 0.5
        v = np.where(forced, np.where(sign, 1, m - 1), v)
    return v.astype(np.uint32)


def uniform_block(seed, n, s, m, key=0):
    """Dense n x s block of residues uniform in [0, m), row-major (row k's s
    residues contiguous)."""
    rng = rng_for(seed, 77, key)
    v = (rng.random(int(n) * int(s)) * m).astype(np.uint64)
    v = np.minimum(v, m - 1).astype(np.uint32)
    return v.reshape(int(n), int(s)) if s > 1 else v


def zipf_exponent(mean, lmax, lmin=1):
    """Exponent a with E[L] = mean for P(L = k) proportional to k^-a on
    [lmin, lmax]."""
    k = np.arange(lmin, lmax + 1, dtype=np.float64)

    def f(a):
        w = k ** -a
        return float((k * w).sum() / w.sum()) - mean

    lo, hi = 0.0, 8.0
    if f(lo) < 0:
        return 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def zipf_lengths(rng, nrows, mean, lmax, lmin=1, force_max=True):
    a = zipf_exponent(mean, lmax, lmin)
    k = np.arange(lmin, lmax + 1, dtype=np.float64)
    cdf = np.cumsum(k ** -a)
    cdf /= cdf[-1]
    lengths = lmin + np.searchsorted(cdf, rng.random(nrows), side="right")
    lengths = np.minimum(lengths, lmax).astype(np.int64)
    if force_max and nrows > 0:
        lengths[int(rng.integers(0, nrows))] = lmax
    return lengths


def _assemble(nrows, ncols, lengths, rows, cols, vals, m, name):
    return CSR(nrows, ncols, _csr_from_lengths(lengths), cols.astype(np.int32),
               vals.astype(np.uint32), int(m), name)


def uniform_matrix(seed, nrows, ncols, lengths, m, pm_fraction=0.0, name="uniform"):
    rng = rng_for(seed, 1)
    lengths = np.asarray(lengths, dtype=np.int64)
    rows, cols = distinct_columns(rng, lengths, ncols)
    vals = residues(rng, rows.size, m, pm_fraction)
    return _assemble(nrows, ncols, lengths, rows, cols, vals, m, name)


def tiny_matrix(seed=1001, n=2000, per_row=10, m=M65521, pm_fraction=0.2):
    """2000 x 2000, 10 distinct uniform columns per row, 20% of the values
    forced to +-1, the rest uniform in [1, m-1]."""
    return uniform_matrix(seed, n, n, np.full(n, per_row), m, pm_fraction,
                          name=f"tiny{n}")


def powerlaw_matrix(seed=1002, n=1_000_000, mean=16.0, lmax=10_000, m=M65521,
                    pm_fraction=0.0, ncols=None):
    """Zipf row lengths on [1, lmax] with mean ``mean`` (one row forced to
    lmax), distinct uniform columns, nonzero residues mod m."""
    ncols = n if ncols is None else ncols
    rng = rng_for(seed, 2)
    lengths = zipf_lengths(rng, n, mean, min(lmax, ncols))
    rows, cols = distinct_columns(rng, lengths, ncols)
    vals = residues(rng_for(seed, 3, m), rows.size, m, pm_fraction)
    return _assemble(n, ncols, lengths, rows, cols, vals, m, f"powerlaw{n}")


def wiedemann_offsets(n):
    return (0, 1, -1, n // 2)


def wiedemann_matrix(seed=1003, n=100_000, p=M65521, n_random=6):
    """Square matrix with the four diagonals {0, +1, -1, +n/2} (entries that
    fall outside the matrix are dropped) plus ``n_random`` uniform entries per
    row off those diagonals; every stored value is uniform in [1, p-1]."""
    rng = rng_for(seed, 4)
    offs = wiedemann_offsets(n)

    def forbid(rows, cols):
        d = cols.astype(np.int64) - rows
        bad = np.zeros(rows.size, dtype=bool)
        for o in offs:
            bad |= d == o
        return bad

    rr, rc = distinct_columns(rng, np.full(n, n_random), n, forbid=forbid)
    drows, dcols = [], []
    for o in offs:
        i = np.arange(n, dtype=np.int64)
        j = i + o
        ok = (j >= 0) & (j < n)
        drows.append(i[ok])
        dcols.append(j[ok])
    rows = np.concatenate([rr] + drows)
    cols = np.concatenate([rc.astype(np.int64)] + dcols)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    lengths = np.bincount(rows, minlength=n).astype(np.int64)
    vals = residues(rng_for(seed, 5), rows.size, p)
    return _assemble(n, n, lengths, rows, cols, vals, p, f"wiedemann{n}")


def windowed_distinct(rng, lengths, lo, hi, chunk=1 << 16):
    """Row i gets ``lengths[i]`` distinct sorted columns from [lo[i], hi[i])
    (windows of at most a few hundred columns): the first ``lengths[i]``
    positions of a random permutation of the window, row by row in chunks."""
    lengths = np.asarray(lengths, dtype=np.int64)
    width = int((hi - lo).max()) if lengths.size else 0
    rows_out, cols_out = [], []
    for a in range(0, lengths.size, chunk):
        b = min(lengths.size, a + chunk)
        keys = rng.random((b - a, width))
        off = np.arange(width)[None, :]
        keys[off >= (hi[a:b] - lo[a:b])[:, None]] = 2.0     # outside the window
        order = np.argsort(keys, axis=1)
        take = off < lengths[a:b, None]
        picked = np.sort(np.where(take, order, width + 1), axis=1)
        r, k = np.nonzero(picked <= width)
        rows_out.append(r + a)
        cols_out.append(lo[a:b][r] + picked[r, k])
    if not rows_out:
        return np.zeros(0, np.int64), np.zeros(0, np.int32)
    return np.concatenate(rows_out), np.concatenate(cols_out).astype(np.int32)


def banded_matrix(seed, n, lengths, m, bandwidth=64, pm_fraction=0.0):
    rng = rng_for(seed, 6)
    half = bandwidth // 2
    i = np.arange(n, dtype=np.int64)
    lo = np.maximum(i - half, 0)
    hi = np.minimum(i + half + 1, n)
    lengths = np.minimum(np.asarray(lengths, dtype=np.int64), hi - lo)
    rows, cols = windowed_distinct(rng, lengths, lo, hi)
    vals = residues(rng, rows.size, m, pm_fraction)
    return _assemble(n, n, lengths, rows, cols, vals, m, f"banded{n}")


def block_diagonal_matrix(seed, n, block, lengths, m, pm_fraction=0.0):
    rng = rng_for(seed, 7)
    i = np.arange(n, dtype=np.int64)
    lo = (i // block) * block
    hi = np.minimum(lo + block, n)
    lengths = np.minimum(np.asarray(lengths, dtype=np.int64), hi - lo)
    rows, cols = windowed_distinct(rng, lengths, lo, hi, chunk=max(1, (1 << 22) // block))
    vals = residues(rng, rows.size, m, pm_fraction)
    return _assemble(n, n, lengths, rows, cols, vals, m, f"blockdiag{n}")


def is_prime(q: int) -> bool:
    """Deterministic Miller-Rabin for q < 3.2e9 (bases 2, 3, 5, 7)."""
    if q < 2:
        return False
    for sp in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if q % sp == 0:
            return q == sp
    d, r = q - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in (2, 3, 5, 7):
        x = pow(a, d, q)
        if x in (1, q - 1):
            continue
        for _ in range(r - 1):
            x = x * x % q
            if x == q - 1:
                break
        else:
            return False
    return True


def random_prime(rng, lo=2**30, hi=2**31):
    while True:
        q = int(rng.integers(lo, hi)) | 1
        if q < hi and is_prime(q):
            return q


BATCH_STRUCTURES = ("uniform", "banded", "powerlaw")


def batch_problems(seed=1004, count=256, rows_lo=1_000, rows_hi=200_000,
                   len_lo=4, len_hi=40, s_lo=1, s_hi=32):
    """``count`` independent square problems of uneven size: rows
    log-uniform in [rows_lo, rows_hi], row lengths uniform in
    [len_lo, len_hi] (power-law members: Zipf with the same mean), structure
    uniform over {uniform, banded (bandwidth 64), power-law}, a random prime
    modulus in [2^30, 2^31) and a block of s_j in [s_lo, s_hi] right-hand
    sides.  Returns a list of (CSR, s_j)."""
    rng = rng_for(seed, 8)
    out = []
    for j in range(count):
        n = int(round(math.exp(rng.uniform(math.log(rows_lo), math.log(rows_hi)))))
        kind = BATCH_STRUCTURES[int(rng.integers(0, 3))]
        p = random_prime(rng)
        s = int(rng.integers(s_lo, s_hi + 1))
        sub = int(rng.integers(0, 2**31))
        lrng = rng_for(sub, 9)
        if kind == "uniform":
            lengths = np.minimum(lrng.integers(len_lo, len_hi + 1, n), n)
            A = uniform_matrix(sub, n, n, lengths, p, name=f"b{j}-uniform")
        elif kind == "banded":
            lengths = lrng.integers(len_lo, len_hi + 1, n)
            A = banded_matrix(sub, n, lengths, p)
            A.name = f"b{j}-banded"
        else:
            mean = 0.5 * (len_lo + len_hi)
            lengths = zipf_lengths(lrng, n, mean, min(10_000, n))
            rows, cols = distinct_columns(lrng, lengths, n)
            vals = residues(lrng, rows.size, p)
            A = _assemble(n, n, lengths, rows, cols, vals, p, f"b{j}-powerlaw")
        out.append((A, s))
    return out


SELECTOR_STRUCTURES = ("banded", "blockdiag", "uniform", "powerlaw")
SELECTOR_MODULI = (3, M65521, M31)


def selector_matrix(seed, index, rows_lo=10_000, rows_hi=2_000_000):
    """Matrix ``index`` of the format-selector family: rows log-uniform in
    [rows_lo, rows_hi], row lengths uniform in [4, 40] (power-law: Zipf with
    that mean), structure uniform over {banded, block-diagonal (block
    32-512), uniform, power-law}, +-1 fraction uniform in [0, 1], modulus
    uniform over {3, 65521, 2^31-1}."""
    rng = rng_for(seed, 10, index)
    n = int(round(math.exp(rng.uniform(math.log(rows_lo), math.log(rows_hi)))))
    kind = SELECTOR_STRUCTURES[int(rng.integers(0, 4))]
    m = SELECTOR_MODULI[int(rng.integers(0, 3))]
    pm = float(rng.random())
    d = int(rng.integers(4, 41))
    sub = int(rng.integers(0, 2**31))
    lrng = rng_for(sub, 11)
    if kind == "banded":
        lengths = lrng.integers(max(1, d // 2), d + d // 2 + 1, n)
        A = banded_matrix(sub, n, lengths, m, pm_fraction=pm)
    elif kind == "blockdiag":
        block = int(lrng.integers(32, 513))
        lengths = lrng.integers(max(1, d // 2), d + d // 2 + 1, n)
        A = block_diagonal_matrix(sub, n, block, lengths, m, pm_fraction=pm)
    elif kind == "uniform":
        lengths = lrng.integers(max(1, d // 2), d + d // 2 + 1, n)
        A = uniform_matrix(sub, n, n, lengths, m, pm_fraction=pm)
    else:
        lengths = zipf_lengths(lrng, n, float(d), min(10_000, n))
        rows, cols = distinct_columns(lrng, lengths, n)
        vals = residues(lrng, rows.size, m, pm)
        A = _assemble(n, n, lengths, rows, cols, vals, m, "powerlaw")
    A.name = f"sel{index}-{kind}-m{m}"
    return A


def dense_to_csr(dense, m, name="dense"):
    """CSR of the nonzero entries of a small dense integer matrix."""
    dense = np.asarray(dense)
    nrows, ncols = dense.shape
    rows, cols = np.nonzero(dense)
    lengths = np.bincount(rows, minlength=nrows).astype(np.int64)
    return CSR(nrows, ncols, _csr_from_lengths(lengths), cols.astype(np.int32),
               dense[rows, cols].astype(np.uint32), int(m), name)


def random_small(seed, nrows, ncols, density, m, pm_fraction=0.0, dup=False):
    """Small random matrix for brute-force checks.  With ``dup`` some
    entries are repeated inside a row (duplicates are summed)."""
    rng = rng_for(seed, 12)
    mask = rng.random((nrows, ncols)) < density
    rows, cols = np.nonzero(mask)
    vals = residues(rng, rows.size, m, pm_fraction)
    if dup and rows.size:
        extra = rng.integers(0, rows.size, max(1, rows.size // 4))
        rows = np.concatenate([rows, rows[extra]])
        cols = np.concatenate([cols, cols[extra]])
        vals = np.concatenate([vals, residues(rng, extra.size, m)])
        order = np.argsort(rows, kind="stable")
        rows, cols, vals = rows[order], cols[order], vals[order]
    lengths = np.bincount(rows, minlength=nrows).astype(np.int64)
    return CSR(nrows, ncols, _csr_from_lengths(lengths), cols.astype(np.int32),
               vals.astype(np.uint32), int(m), f"small{nrows}x{ncols}")
