"""GPU parity of the GF(2) products with bit-packed vectors (Y = A X, A^T X,
Y ^= A X; 64 components per word) against the oracle in oracle/gf2.py,
bit-exact."""
import numpy as np
import pytest

import gen
from oracle import gf2

pytestmark = pytest.mark.gpu


def _words(seed, rows, w):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2**63, (rows, w), dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, (rows, w), dtype=np.uint64)


def _host(t):
    return t.detach().cpu().numpy().view(np.uint64)


def _check(lib, A, w, seed, transpose=False, accumulate=False):
    M = lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.NONE)
    in_rows, out_rows = (A.nrows, A.ncols) if transpose else (A.ncols, A.nrows)
    X = _words(seed, in_rows, w)
    want = gf2.csr_gf2(A, X, transpose=transpose)
    if accumulate:
        import torch
        Y0 = _words(seed + 1, out_rows, w)
        y = torch.from_numpy(Y0.view(np.int64)).cuda()
        M.apply_gf2(X, y, transpose=transpose, accumulate=True)
        want = want ^ Y0
    else:
        y = M.apply_gf2(X, transpose=transpose)
    got = _host(y).reshape(out_rows, w)
    assert np.array_equal(got, want), (A.name, w, transpose, accumulate)


def test_tiny_words_and_modes(lib):
    A = gen.tiny_matrix(m=2)
    for w in (1, 2, 3, 4, 5, 9):
        _check(lib, A, w, seed=w)
    _check(lib, A, 2, seed=20, transpose=True)
    _check(lib, A, 3, seed=21, accumulate=True)
    _check(lib, A, 1, seed=22, transpose=True, accumulate=True)


def test_powerlaw_long_rows(lib):
    # Zipf rows up to 3000 entries: rows over 32 entries go to warps, in chunks of 1024
    A = gen.powerlaw_matrix(seed=7, n=30_011, lmax=3000, m=2)
    for w in (1, 2, 4, 5):
        _check(lib, A, w, seed=30 + w)
    _check(lib, A, 2, seed=40, transpose=True)


def test_rectangular_duplicates_empty_rows(lib):
    A = gen.random_small(3, 517, 1283, 0.01, 2, dup=True)
    _check(lib, A, 1, seed=50)
    _check(lib, A, 3, seed=51, transpose=True)
    # every value even: the product is zero
    Z = gen.CSR(A.nrows, A.ncols, A.row_ptr, A.col, np.zeros_like(A.val), 2)
    _check(lib, Z, 2, seed=52)
    E = gen.CSR(6, 4, np.zeros(7, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint32), 2)
    _check(lib, E, 1, seed=53)


def test_full_size_powerlaw(lib):
    A = gen.powerlaw_matrix(seed=1002, m=2)
    _check(lib, A, 1, seed=60)
    _check(lib, A, 1, seed=61, transpose=True)


def test_errors(lib):
    A = gen.tiny_matrix(m=3)
    M = lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.NONE)
    with pytest.raises(lib.FFSPMVError) as e:
        M.apply_gf2(_words(1, A.ncols, 1))
    assert e.value.status == 5            # modulus must be 2
    B = lib.Matrix.from_csr(gen.tiny_matrix(m=2), transpose_mode=lib.TRANSPOSE.NONE)
    import torch
    x = torch.zeros((B.ncols, 1), dtype=torch.int64, device="cuda")
    y = torch.zeros((B.nrows, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(lib.FFSPMVError) as e:
        lib.spmv_apply_gf2(B.handle, 0, x, y, 0)
    assert e.value.status == 1            # words >= 1
    with pytest.raises(lib.FFSPMVError) as e:
        lib.spmv_apply_gf2(B.handle, 2, x, y, 1)
    assert e.value.status == 1            # transpose is 0 or 1
