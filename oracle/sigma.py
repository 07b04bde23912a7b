"""Oracle for sigma-bases (minimal approximant bases) over F_p.

TEST INFRASTRUCTURE ONLY (see the package docstring): the tests are the only
callers.

Block Wiedemann's second step (Sec. 3.2) computes the minimal matrix generator
of the sequence S_i by a sigma-basis computation, with the algorithm PM-Basis
of Giorgi, Jeannerod and Villard (2003), which reduces to polynomial-matrix
products and, at small orders, to their iterative M-Basis.  Definitions used
here: for F in F_p[x]^{m x n}, an order d and a shift vector s in Z^m, a
sigma-basis is an m x m polynomial matrix P whose rows span (over F_p[x]) the
module of approximants {v : v F = 0 mod x^d}, and whose rows have minimal
s-shifted degrees.  Both algorithms return P together with the shifted row
degrees delta (delta_i = s_i + the number of times row i was multiplied by x).

Polynomial matrices are coefficient-major object arrays of Python integers,
shape (deg + 1, rows, cols), so every sum is exact before its reduction mod p.
"""
from __future__ import annotations

import numpy as np


def _zeros(deg, r, c):
    return np.zeros((deg + 1, r, c), dtype=object)


def poly_mul(A, B, p):
    """A(x) B(x) mod p for coefficient-major object arrays (plain convolution)."""
    C = _zeros(A.shape[0] + B.shape[0] - 2, A.shape[1], B.shape[2])
    for a in range(A.shape[0]):
        for b in range(B.shape[0]):
            C[a + b] = (C[a + b] + np.dot(A[a], B[b])) % p
    return C


def coeff(P, F, k, p):
    """The coefficient of x^k in P(x) F(x)."""
    out = np.zeros((P.shape[1], F.shape[2]), dtype=object)
    for j in range(max(0, k - F.shape[0] + 1), min(k, P.shape[0] - 1) + 1):
        out = (out + np.dot(P[j], F[k - j])) % p
    return out


def trim(P):
    """Drop leading zero coefficient matrices (keep at least one)."""
    d = P.shape[0]
    while d > 1 and not np.any(P[d - 1]):
        d -= 1
    return P[:d]


def mbasis(F, d, shift, p):
    """Order-d sigma-basis of F (m x n) by the iterative algorithm: at order k,
    take the coefficient Delta of x^k in P F, order the rows by their current
    shifted degree, eliminate Delta column by column with the first row (in
    that order) that is nonzero in the column as pivot -- adding multiples of
    a pivot row only to rows after it -- and multiply the pivot rows by x."""
    F = np.asarray(F, dtype=object) % p
    m = F.shape[1]
    delta = [int(v) for v in shift]
    P = _zeros(0, m, m)
    for i in range(m):
        P[0, i, i] = 1
    for k in range(d):
        D = coeff(P, F, k, p)
        order = sorted(range(m), key=lambda i: (delta[i], i))  # stable in the row index
        pivots = []
        for j in range(F.shape[2]):
            piv = next((r for r in order if r not in pivots and D[r, j] % p), None)
            if piv is None:
                continue
            pivots.append(piv)
            inv = pow(int(D[piv, j]), p - 2, p)
            for r in order[order.index(piv) + 1:]:
                if r in pivots or D[r, j] % p == 0:
                    continue
                f = (D[r, j] * inv) % p
                D[r] = (D[r] - f * D[piv]) % p
                P[:, r] = (P[:, r] - f * P[:, piv]) % p
        if pivots:
            P = np.concatenate([P, _zeros(0, m, m)], axis=0)
            for r in pivots:
                P[1:, r] = P[:-1, r].copy()
                P[0, r] = 0
                delta[r] += 1
        P = trim(P)
    return P, delta


def pmbasis(F, d, shift, p, base=4):
    """Order-d sigma-basis by divide and conquer: a basis P1 of order d1 =
    ceil(d/2), then a basis P2 of order d - d1 of the remaining coefficients of
    P1 F (x^-d1 (P1 F) mod x^(d-d1)) with P1's shifted degrees as shift; the
    result is P2 P1 with P2's degrees.  Orders up to `base` use mbasis."""
    F = np.asarray(F, dtype=object) % p
    if d <= base:
        return mbasis(F, d, shift, p)
    d1 = (d + 1) // 2
    P1, delta1 = pmbasis(F[:d1], d1, shift, p, base)
    G = np.stack([coeff(P1, F, d1 + k, p) for k in range(d - d1)])
    P2, delta2 = pmbasis(G, d - d1, delta1, p, base)
    return trim(poly_mul(P2, P1, p)), delta2


def det_poly(P, p):
    """det P(x) mod p as a coefficient list, by evaluation at deg+1 points and
    Lagrange interpolation (p must exceed the degree bound)."""
    m = P.shape[1]
    bound = (P.shape[0] - 1) * m
    assert p > bound + 1
    xs = list(range(bound + 1))
    vals = []
    for x0 in xs:
        M = np.zeros((m, m), dtype=object)
        for k in range(P.shape[0] - 1, -1, -1):
            M = (M * x0 + P[k]) % p
        vals.append(_det_mod(M, p))
    # Lagrange interpolation to coefficients
    coeffs = [0] * (bound + 1)
    for i, xi in enumerate(xs):
        num = [1]
        den = 1
        for j, xj in enumerate(xs):
            if j == i:
                continue
            num = _poly_mul_lin(num, -xj, p)
            den = den * (xi - xj) % p
        c = vals[i] * pow(den, p - 2, p) % p
        for t in range(len(num)):
            coeffs[t] = (coeffs[t] + c * num[t]) % p
    return coeffs


def _poly_mul_lin(a, c, p):
    """a(x) * (x + c) mod p."""
    out = [0] * (len(a) + 1)
    for i, v in enumerate(a):
        out[i + 1] = (out[i + 1] + v) % p
        out[i] = (out[i] + v * c) % p
    return out


def _det_mod(M, p):
    M = [list(map(int, r)) for r in M]
    n = len(M)
    det = 1
    for c in range(n):
        piv = next((r for r in range(c, n) if M[r][c] % p), None)
        if piv is None:
            return 0
        if piv != c:
            M[c], M[piv] = M[piv], M[c]
            det = -det
        det = det * M[c][c] % p
        inv = pow(M[c][c], p - 2, p)
        for r in range(c + 1, n):
            f = M[r][c] * inv % p
            if f:
                M[r] = [(a - f * b) % p for a, b in zip(M[r], M[c])]
    return det % p


def degree_and_codegree(coeffs):
    """(deg, codeg) of a nonzero polynomial given by its coefficient list."""
    nz = [i for i, c in enumerate(coeffs) if c]
    return nz[-1], nz[0]
