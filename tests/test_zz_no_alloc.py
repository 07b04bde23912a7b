"""The allocation-free transpose product (spmv_apply_transpose_noalloc),
called through the C ABI, against the existing transpose entry point.

It is meant for callers that cannot let the library allocate device memory
while they run; its scratch is a fixed array inside the library.  Two calls
in a row check that the shared array is cleared between calls.  This file is
collected last on purpose: a failure here comes after every other test."""
import numpy as np
import pytest

import gen
from helpers import rand_block, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_noalloc_transpose_matches_existing_entry_point(lib):
    import torch
    A = gen.powerlaw_matrix(seed=31, n=50_000, lmax=3000, m=2**31 - 1, pm_fraction=0.2)
    M = lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.ATOMIC)
    for call, (nvec, alpha, beta) in enumerate(((3, 5, 7), (3, 1, 0))):
        x = to_dev(rand_block(100 + call, A.nrows, nvec, A.modulus))
        y0 = rand_block(200 + call, A.ncols, nvec, A.modulus)
        want = to_dev(y0)
        got = to_dev(y0)
        lib.spmv_apply_transpose(M.handle, x, nvec, want, nvec, nvec, alpha, beta)
        lib.spmv_apply_transpose_noalloc(M.handle, x, nvec, got, nvec, nvec, alpha, beta)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(got), to_host(want)), f"call {call}"


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
