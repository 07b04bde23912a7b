"""The allocation-free transpose product (spmv_apply_transpose_noalloc),
called through the C ABI, against the CPU oracle.

It is meant for callers that cannot let the library allocate device memory
while they run (their device memory is all reserved up front for their own
pool, or they cannot take the device-wide synchronisation of a cudaFree); its
scratch is one fixed array inside the library.  Each case makes two calls in
a row, so a second call that found the first one's sums still in the shared
array would fail.  The cases reach the chunk loop: more than 16 vectors, and
a column count for which the array holds one vector at a time.  This file is
collected last on purpose: a failure here comes after every other test."""
import numpy as np
import pytest

import gen
import oracle
from helpers import rand_block, to_dev, to_host

pytestmark = pytest.mark.gpu


def _two_calls(lib, A, M, nvec, ldx, ldy, calls):
    import torch
    for call, (alpha, beta) in enumerate(calls):
        xs = rand_block(100 + call, A.nrows, ldx, A.modulus).reshape(A.nrows, ldx)
        y0 = rand_block(200 + call, A.ncols, ldy, A.modulus).reshape(A.ncols, ldy)
        got = to_dev(y0)
        lib.spmv_apply_transpose_noalloc(M.handle, to_dev(xs), ldx, got, ldy, nvec, alpha, beta)
        torch.cuda.synchronize()
        want = y0.copy()
        want[:, :nvec] = oracle.csr_spmv_transpose(A, xs[:, :nvec], y=y0[:, :nvec],
                                                   alpha=alpha, beta=beta)
        assert np.array_equal(to_host(got).reshape(A.ncols, ldy), want), f"call {call}"


def test_noalloc_transpose_matches_oracle(lib):
    A = gen.powerlaw_matrix(seed=31, n=50_000, lmax=3000, m=2**31 - 1, pm_fraction=0.2)
    M = lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.ATOMIC)
    _two_calls(lib, A, M, 3, 3, 3, ((5, 7), (1, 0)))


def test_noalloc_more_than_16_vectors_strided(lib):
    # 40 vectors: chunks of 16, 16 and 8; x and y with leading dimensions
    # larger than the block, whose extra columns must stay untouched
    A = gen.powerlaw_matrix(seed=32, n=6000, lmax=400, m=65521, pm_fraction=0.3)
    M = lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.ATOMIC)
    _two_calls(lib, A, M, 40, 43, 41, ((3, 2), (1, 0)))


def test_noalloc_one_vector_per_chunk(lib):
    # ncols just above 2^19: the array holds one vector of sums at a time,
    # so three vectors take three chunks, each clearing it again
    n = (1 << 19) + 40
    A = gen.uniform_matrix(7, n, n, np.full(n, 3), 65521)
    M = lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.ATOMIC)
    _two_calls(lib, A, M, 3, 3, 3, ((1, 0), (2, 5)))


def test_noalloc_value_check_and_device(lib):
    A = gen.tiny_matrix(n=300, per_row=5)
    M = lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.ATOMIC, value_check=1)
    x = rand_block(1, 300, 1, A.modulus)
    x[17] = A.modulus                                 # one residue out of range
    y = to_dev(np.zeros(300, np.uint32))
    with pytest.raises(lib.FFSPMVError) as e:
        lib.spmv_apply_transpose_noalloc(M.handle, to_dev(x), 1, y, 1, 1)
    assert e.value.status == 2
    x[17] = 0
    lib.spmv_apply_transpose_noalloc(M.handle, to_dev(x), 1, y, 1, 1)
    assert np.array_equal(to_host(y), oracle.csr_spmv_transpose(A, x))


def test_noalloc_rejects_what_it_cannot_hold(lib):
    A = gen.tiny_matrix(n=300, per_row=5)
    E = lib.Matrix.from_csr(A)                       # explicit transpose: no device CSR
    x = to_dev(rand_block(1, 300, 1, A.modulus))
    y = to_dev(np.zeros(300, np.uint32))
    with pytest.raises(lib.FFSPMVError) as e:
        lib.spmv_apply_transpose_noalloc(E.handle, x, 1, y, 1, 1)
    assert e.value.status == 5
    wide = gen.uniform_matrix(2, 4, (1 << 20) + 1, np.array([1, 0, 2, 1]), 65521)
    W = lib.Matrix.from_csr(wide, transpose_mode=lib.TRANSPOSE.ATOMIC)
    with pytest.raises(lib.FFSPMVError) as e:
        lib.spmv_apply_transpose_noalloc(W.handle, to_dev(np.ones(4, np.uint32)), 1,
                                         to_dev(np.zeros((1 << 20) + 1, np.uint32)), 1, 1)
    assert e.value.status == 5
