"""Pins of the polynomial-matrix product oracle (oracle/polymat.py): exact
big-integer convolution for 1 x 1 matrices, evaluation at random points
(C(x0) = A(x0) B(x0) mod p, computed with Python integers), and the degree /
identity special cases."""
import numpy as np

from oracle import polymat


def _rand(seed, d, s, p):
    return np.random.default_rng(seed).integers(0, p, (d + 1, s, s), dtype=np.int64)


def test_scalar_is_exact_convolution():
    for p in (3, 65521, 2**31 - 1):
        a, b = _rand(1, 40, 1, p), _rand(2, 57, 1, p)
        want = np.convolve(a[:, 0, 0].astype(object), b[:, 0, 0].astype(object)) % p
        assert np.array_equal(polymat.polymat_mul(a, b, p)[:, 0, 0], want.astype(np.int64))


def test_evaluation_at_random_points():
    rng = np.random.default_rng(3)
    for p, s, da, db in ((65521, 4, 9, 13), (2**31 - 1, 16, 6, 3), (7, 3, 20, 0)):
        A, B = _rand(4, da, s, p), _rand(5, db, s, p)
        C = polymat.polymat_mul(A, B, p)
        assert C.shape == (da + db + 1, s, s)
        for x0 in rng.integers(0, p, 3).tolist():
            lhs = polymat.polymat_eval(C, int(x0), p)
            rhs = np.dot(polymat.polymat_eval(A, int(x0), p), polymat.polymat_eval(B, int(x0), p)) % p
            assert np.array_equal(lhs, rhs)


def test_identity_and_constants():
    p, s = 65521, 5
    A = _rand(6, 11, s, p)
    I = np.eye(s, dtype=np.int64)[None, :, :]
    assert np.array_equal(polymat.polymat_mul(A, I, p), A)
    assert np.array_equal(polymat.polymat_mul(I, A, p), A)
    c = _rand(7, 0, s, p)
    assert np.array_equal(polymat.polymat_mul(c, A, p), np.matmul(c[0].astype(object), A.astype(object)) % p)
