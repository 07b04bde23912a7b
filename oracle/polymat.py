"""Oracle for products of polynomial matrices over Z/pZ.

TEST INFRASTRUCTURE ONLY (see the package docstring): the tests and the
benchmark's CPU-baseline leg are the only callers.

The sigma-basis / PM-Basis step of block Wiedemann (Sec. 3) multiplies s x s
matrices whose entries are polynomials over F_p: C(x) = A(x) B(x), i.e.
C_k = sum_{a+b=k} A_a B_b mod p with A_a, B_b the s x s coefficient matrices.
Arrays are coefficient-major: A[k, i, j] is the coefficient of x^k in entry
(i, j).  The sum is taken exactly: each coefficient matrix of A is split into
16-bit limbs so that the int64 matrix products cannot overflow (s <= 64,
p <= 2^31), then reduced mod p.
"""
from __future__ import annotations

import numpy as np


def polymat_mul(A, B, p):
    """C = A B mod p; A: (da+1, s, s), B: (db+1, s, s) -> (da+db+1, s, s)."""
    A = np.asarray(A, dtype=np.int64) % p
    B = np.asarray(B, dtype=np.int64) % p
    da, db = A.shape[0] - 1, B.shape[0] - 1
    s = A.shape[1]
    assert A.shape[1:] == (s, s) and B.shape[1:] == (s, s) and s <= 64 and p <= 2**31
    C = np.zeros((da + db + 1, s, s), dtype=np.int64)
    for a in range(da + 1):
        hi, lo = A[a] >> 16, A[a] & 0xFFFF
        # (hi 2^16 + lo) B_b for every b at once; each int64 product sum < 2^58
        ph = np.matmul(hi[None, :, :], B) % p
        pl = np.matmul(lo[None, :, :], B) % p
        C[a:a + db + 1] = (C[a:a + db + 1] + ph * 65536 % p + pl) % p
    return C


def polymat_eval(A, x0, p):
    """A(x0) mod p by Horner's rule (an s x s matrix)."""
    A = np.asarray(A, dtype=object)
    r = np.zeros(A.shape[1:], dtype=object)
    for k in range(A.shape[0] - 1, -1, -1):
        r = (r * x0 + A[k]) % p
    return r
