"""Pins of the GF(2) oracle (oracle/gf2.py) to things other than itself: a
dense integer product reduced mod 2, the C oracle of the mod-m products at
m = 2 bit-plane by bit-plane, cancellation of repeated pairs, linearity and
the transpose identity."""
import numpy as np

import gen
import oracle
from oracle import gf2


def _rand_words(seed, rows, w):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2**63, (rows, w), dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, (rows, w), dtype=np.uint64)


def test_dense_product_mod_2():
    # every entry value 0..5 (even ones vanish mod 2), dense integer matmul
    rng = np.random.default_rng(1)
    D = rng.integers(0, 6, (37, 29))
    A = gen.dense_to_csr(D, 1 << 20)      # keep the raw values, parity decides
    X = _rand_words(2, 29, 2)
    Y = gf2.csr_gf2(A, X)
    want = (D % 2) @ gf2.unpack_bits(X).astype(np.int64) % 2
    assert np.array_equal(gf2.unpack_bits(Y), want)
    YT = gf2.csr_gf2(A, _rand_words(3, 37, 1), transpose=True)
    wantT = (D % 2).T @ gf2.unpack_bits(_rand_words(3, 37, 1)).astype(np.int64) % 2
    assert np.array_equal(gf2.unpack_bits(YT), wantT)


def test_c_oracle_at_m_2_bit_planes():
    A = gen.random_small(5, 2000, 1500, 0.01, 2, dup=True)
    X = _rand_words(6, A.ncols, 1)
    Y = gf2.unpack_bits(gf2.csr_gf2(A, X))
    bits = gf2.unpack_bits(X)
    for b in (0, 1, 31, 63):
        y = oracle.csr_spmv(A, bits[:, b].astype(np.uint32))
        assert np.array_equal(Y[:, b], y), b


def test_repeated_pairs_cancel_and_linearity():
    ptr = np.array([0, 3, 5, 5], dtype=np.int64)
    col = np.array([1, 1, 2, 0, 0], dtype=np.int32)
    val = np.array([1, 3, 1, 1, 1], dtype=np.uint32)   # (0,1) twice odd: cancels
    X = np.array([[7], [9], [12]], dtype=np.uint64)
    Y = gf2.spmv_gf2(3, 3, ptr, col, val, X)
    assert Y.reshape(-1).tolist() == [12, 0, 0]
    A = gen.random_small(7, 300, 400, 0.05, 2)
    X1, X2 = _rand_words(8, 400, 3), _rand_words(9, 400, 3)
    assert np.array_equal(gf2.csr_gf2(A, X1 ^ X2), gf2.csr_gf2(A, X1) ^ gf2.csr_gf2(A, X2))


def test_transpose_identity():
    # <A x_b, z_b> = <x_b, A^T z_b> over GF(2) for every component b: the
    # exclusive or over rows of (A x) & z, bit b, is that inner product
    A = gen.random_small(10, 250, 180, 0.04, 2)
    x, z = _rand_words(11, 180, 2), _rand_words(12, 250, 2)
    lhs = np.bitwise_xor.reduce(gf2.csr_gf2(A, x) & z, axis=0)
    rhs = np.bitwise_xor.reduce(x & gf2.csr_gf2(A, z, transpose=True), axis=0)
    assert np.array_equal(lhs, rhs)
    assert lhs.any()  # a non-trivial check
