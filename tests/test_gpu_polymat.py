"""GPU parity of the polynomial-matrix product (NTT over three primes and the
Chinese remainder theorem) against oracle/polymat.py: element by element at
sizes the oracle finishes quickly, and at the sigma-basis top-level size
(s = 16, degree 6250 each) through evaluation at random points."""
import numpy as np
import pytest

from oracle import polymat

pytestmark = pytest.mark.gpu


def _rand(seed, d, s, p):
    rng = np.random.default_rng(seed)
    return rng.integers(0, p, (d + 1, s, s), dtype=np.int64).astype(np.uint32)


def _run(lib, p, A, B):
    return lib.polymat_mul(p, A, B).cpu().numpy().view(np.uint32).astype(np.int64)


@pytest.mark.parametrize("p,s,da,db", [(3, 1, 0, 0), (65521, 4, 1, 3), (65521, 16, 100, 157),
                                       (2**31 - 1, 16, 300, 300), (2**31, 8, 50, 0),
                                       (1000003, 32, 63, 64), (65537, 5, 1000, 17)])
def test_parity(lib, p, s, da, db):
    A, B = _rand(p % 1000 + da, da, s, p), _rand(p % 1000 + db + 1, db, s, p)
    got = _run(lib, p, A, B)
    assert np.array_equal(got, polymat.polymat_mul(A, B, p)), (p, s, da, db)


def test_all_maximal_coefficients(lib):
    # every coefficient p - 1: the exact sums are as large as the bound allows
    p, s, d = 2**31, 32, 2**13 - 1
    A = np.full((d + 1, s, s), p - 1, dtype=np.uint32)
    B = np.full((d + 1, s, s), p - 1, dtype=np.uint32)
    got = _run(lib, p, A, B)
    k = np.arange(2 * d + 1)
    terms = np.minimum(k, 2 * d - k) + 1                    # pairs (a, b) with a + b = k
    want = (terms.astype(object) * s * (p - 1) * (p - 1)) % p
    assert np.array_equal(got[:, 0, 0], want.astype(np.int64))
    assert np.all(got == got[:, :1, :1])


def test_sigma_basis_size_by_evaluation(lib):
    p, s, d = 65521, 16, 6250
    A, B = _rand(11, d, s, p), _rand(12, d, s, p)
    C = _run(lib, p, A, B)
    assert C.shape == (2 * d + 1, s, s)
    for x0 in (0, 1, 12345, p - 1):
        lhs = polymat.polymat_eval(C, x0, p)
        rhs = np.dot(polymat.polymat_eval(A, x0, p), polymat.polymat_eval(B, x0, p)) % p
        assert np.array_equal(lhs, rhs), x0


def test_errors(lib):
    import ctypes
    L = lib.lib()
    n = ctypes.c_int64()
    assert L.polymat_mul_workspace(33, 1, 1, ctypes.byref(n)) == 1       # s <= 32
    assert L.polymat_mul_workspace(4, 2**14, 2**14, ctypes.byref(n)) == 5  # length over 2^15
    assert L.polymat_mul_workspace(4, 2**14 - 1, 2**14, ctypes.byref(n)) == 0
    with pytest.raises(lib.FFSPMVError) as e:
        lib.polymat_mul(1, _rand(1, 2, 2, 1), _rand(2, 2, 2, 1))        # p >= 2
    assert e.value.status == 1
