"""The host half of the x-panel layout, on the CPU: every stored entry
decodes back to the matrix's (row, column, value) triples exactly once,
packs hold eight entries of one row, the +-1 sections carry the right signs,
and the bank ordering keeps a warp's shared-memory accesses spread (the
model the layout is built for).  The device kernel that consumes the layout
is checked against the oracle in test_gpu_spmv.py."""
import ctypes

import numpy as np
import pytest

import gen
from helpers import with_modulus


def decode(A, m, use_pm1, q, clusters, nv=1):
    import paper_1004_3719_gb300 as ff
    ff.build()
    L = ff.lib()
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(A.col, dtype=np.int32)
    val = np.ascontiguousarray(A.val, dtype=np.uint32)
    cap = int(A.nnz)
    r = np.zeros(cap, np.int64)
    c = np.zeros(cap, np.int64)
    v = np.zeros(cap, np.uint32)
    n = ctypes.c_int64()
    st = (ctypes.c_double * 10)()
    rc = L.ffspmv_panel_decode(A.nrows, A.ncols, rp.ctypes.data, col.ctypes.data, val.ctypes.data, m,
                               use_pm1, q, nv, clusters, cap, r.ctypes.data, c.ctypes.data, v.ctypes.data,
                               ctypes.byref(n), st)
    assert rc == 0
    return r[:n.value], c[:n.value], v[:n.value], list(st)


def expected(A, m):
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    lens = np.diff(A.row_ptr)
    keep = np.repeat(lens <= 32768, lens)
    v = (np.asarray(A.val, np.uint64) % m).astype(np.uint32)
    keep &= v != 0
    return rows[keep], np.asarray(A.col, np.int64)[keep], v[keep]


def same_triples(a, b):
    ka = np.lexsort((a[2], a[1], a[0]))
    kb = np.lexsort((b[2], b[1], b[0]))
    return all(np.array_equal(x[ka], y[kb]) for x, y in zip(a, b))


@pytest.mark.parametrize("m,use_pm1,q", [(65521, 0, 2), (65521, 1, 2), (3, 1, 2), (3, 0, 4),
                                         (2**31 - 1, 1, 2), (2**31 - 1, 0, 1), (65536, 1, 4),
                                         (2**20, 1, 2), (4294967291, 0, 1)])
def test_layout_decodes_to_the_matrix(m, use_pm1, q):
    # odd 2^16 < m < 2^31 stores values in Montgomery form (v 2^32 mod m);
    # the decoder maps them back, so every modulus decodes to the matrix
    A = with_modulus(gen.powerlaw_matrix(seed=41, n=60_000, lmax=6000), m, pm_fraction=0.3, seed=3)
    r, c, v, st = decode(A, m, use_pm1, q, 12)
    assert st[8] == 0                                   # every pack is one row
    assert same_triples((r, c, v), expected(A, m))
    if use_pm1 and m > 3:
        assert st[4] > 0                                # +-1 sections in use
    if m == 3 and use_pm1:
        assert st[4] >= 0.99 * A.nnz                    # all +-1 (up to the odd few per stage)


@pytest.mark.parametrize("m,use_pm1,q,nv", [(65521, 1, 2, 2), (3, 1, 1, 4), (65521, 0, 4, 4),
                                            (2**31 - 1, 1, 2, 2)])
def test_multi_vector_layout_decodes_to_the_matrix(m, use_pm1, q, nv):
    """The layouts of 2- and 4-vector passes (x and row sums interleaved by
    vector, so smaller panels and row groups) hold the same entries, with
    panel bytes a multiple of the interleaved column width."""
    A = with_modulus(gen.powerlaw_matrix(seed=43, n=50_000, lmax=5000), m, pm_fraction=0.3, seed=5)
    r, c, v, st = decode(A, m, use_pm1, q, 12, nv=nv)
    assert st[8] == 0
    assert same_triples((r, c, v), expected(A, m))
    xb = (2 if m <= 65536 else 4) * nv
    assert st[6] % 128 == 0 and st[6] % xb == 0
    _, _, _, st1 = decode(A, m, use_pm1, q, 12, nv=1)
    assert st[6] / xb <= st1[6] / (xb // nv)            # no more columns per panel than one vector's


def test_multi_vector_layout_limits():
    """Four vectors per pass only with 16-bit residues; nv outside 1, 2, 4 is
    an argument error."""
    import paper_1004_3719_gb300 as ff
    A = with_modulus(gen.powerlaw_matrix(seed=44, n=5_000, lmax=500), 2**31 - 1, seed=1)
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(A.col, dtype=np.int32)
    val = np.ascontiguousarray(A.val, dtype=np.uint32)
    n = ctypes.c_int64()
    L = ff.lib()
    for nv, want in ((4, 5), (3, 1), (0, 1)):
        rc = L.ffspmv_panel_decode(A.nrows, A.ncols, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                   2**31 - 1, 0, 1, nv, 8, 0, None, None, None, ctypes.byref(n), None)
        assert rc == want, (nv, rc)


def test_builder_cluster_size_rule():
    """The builder's choice between one and two CTAs per cluster (q = 0,
    152 SMs): one for local structure (a band: each row group's entries fall
    in one column half) and where the entries outweigh x in what a CTA
    streams; two for spread columns with x at least twice the entries."""
    n = 300_000
    band = gen.banded_matrix(3, n, np.full(n, 12), 65521)
    assert decode(band, 65521, 0, 0, 152)[3][9] == 1
    sparse = gen.uniform_matrix(4, n, n, np.full(n, 4), 65521)          # x/e = 300k*2*152 / (1.2M*6) = 12.7
    assert decode(sparse, 65521, 0, 0, 152)[3][9] == 2
    dense = gen.uniform_matrix(5, 60_000, 60_000, np.full(60_000, 40), 65521)   # x/e = 60k*2*152 / (2.4M*6) = 1.3
    assert decode(dense, 65521, 0, 0, 152)[3][9] == 1


def test_layout_with_duplicates_zeros_and_long_rows():
    # repeated (i, j) pairs, explicit zeros, a row past the panel cap, empty rows
    rng = np.random.default_rng(5)
    n = 5000
    lens = rng.integers(0, 30, n)
    lens[17] = 40_000                                   # stays out of the panels
    lens[100:200] = 0
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = rng.integers(0, n, rp[-1]).astype(np.int32)
    col[rp[300]:rp[300] + 5] = 7                        # five copies of (300, 7)
    val = rng.integers(0, 65521, rp[-1]).astype(np.uint32)
    val[::97] = 0
    A = gen.CSR(n, n, rp, col, val, 65521)
    r, c, v, st = decode(A, 65521, 1, 1, 8)
    assert st[8] == 0
    assert same_triples((r, c, v), expected(A, 65521))


def test_packs_of_one_row_in_both_sections():
    # rows with eight general and eight +-1 entries in one stage give a
    # general pack and a +-1 pack of the same row in one warp, with single
    # lanes between them: the segmented sum must keep them apart
    rng = np.random.default_rng(9)
    n, m = 300, 65521
    cols, vals, rp = [], [], [0]
    for i in range(n):
        k = 16 if i % 7 == 0 else int(rng.integers(1, 12))
        c = np.sort(rng.choice(n, k, replace=False))
        v = rng.integers(2, m - 1, k)
        if i % 7 == 0:
            v[::2] = np.where(rng.random(8) < 0.5, 1, m - 1)
        cols.append(c); vals.append(v); rp.append(rp[-1] + k)
    A = gen.CSR(n, n, np.array(rp, np.int64), np.concatenate(cols).astype(np.int32),
                np.concatenate(vals).astype(np.uint32), m)
    r, c, v, st = decode(A, m, 1, 1, 8)
    assert st[8] == 0
    assert same_triples((r, c, v), expected(A, m))


def test_bank_order_spreads_a_warps_accesses():
    # the power-law shape of the benchmark at 1/5 size: random x gathers and
    # row-sum atomics would need about 3.5 wavefronts per warp instruction
    A = gen.powerlaw_matrix(seed=1002, n=200_000)
    _, _, _, st = decode(A, 65521, -1, 2, 76)
    assert st[8] == 0
    assert st[2] < 2.3, st                              # x gathers per slot
    assert st[3] < 2.0, st                              # single-lane atomics per slot
