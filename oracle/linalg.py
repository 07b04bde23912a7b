"""Dense linear algebra mod p used to pin the sequence oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Pure Python integers:
slow, exact, and independent of ``oracle.c``.

* ``rank_mod_p``        Gaussian elimination over Z/pZ (p prime).
* ``berlekamp_massey``  the minimal polynomial of a scalar linearly recurrent
                        sequence (the scalar case of block Wiedemann's second
                        step, Sec. 3, step 2).
* ``rank_from_minpoly`` deg f - codeg f: the rank read off the generator
                        (Sec. 3, step 3, scalar case).
* ``dense_*``           brute-force dense products over Python integers.
"""
from __future__ import annotations


def rank_mod_p(rows, p):
    """Rank of a matrix (list of lists of ints) over Z/pZ, p prime."""
    a = [[int(v) % p for v in r] for r in rows]
    if not a:
        return 0
    nr, nc = len(a), len(a[0])
    rank = 0
    for c in range(nc):
        piv = None
        for r in range(rank, nr):
            if a[r][c]:
                piv = r
                break
        if piv is None:
            continue
        a[rank], a[piv] = a[piv], a[rank]
        inv = pow(a[rank][c], p - 2, p)
        a[rank] = [(v * inv) % p for v in a[rank]]
        for r in range(nr):
            if r != rank and a[r][c]:
                f = a[r][c]
                a[r] = [(v - f * w) % p for v, w in zip(a[r], a[rank])]
        rank += 1
        if rank == nr:
            break
    return rank


def berlekamp_massey(seq, p):
    """Connection polynomial C (C[0] = 1) and length L of the shortest linear
    recurrence sum_{j=0..L} C[j] * seq[i-j] = 0 (mod p) for i >= L.

    The minimal polynomial of the sequence is the reverse x^L C(1/x)."""
    s = [int(v) % p for v in seq]
    C, B = [1], [1]
    L, m, b = 0, 1, 1
    for n in range(len(s)):
        d = s[n]
        for j in range(1, L + 1):
            d = (d + C[j] * s[n - j]) % p
        if d == 0:
            m += 1
            continue
        coef = d * pow(b, p - 2, p) % p
        T = list(C)
        if len(C) < len(B) + m:
            C = C + [0] * (len(B) + m - len(C))
        for j, bj in enumerate(B):
            C[j + m] = (C[j + m] - coef * bj) % p
        if 2 * L <= n:
            L = n + 1 - L
            B, b, m = T, d, 1
        else:
            m += 1
    C = C + [0] * max(0, L + 1 - len(C))
    return C[:L + 1], L


def minpoly_from_bm(C, L):
    """Coefficients (low degree first) of the minimal polynomial x^L C(1/x)."""
    return [C[L - i] if L - i < len(C) else 0 for i in range(L + 1)]


def rank_from_minpoly(f):
    """deg f - codeg f, codeg f being the multiplicity of x as a factor."""
    deg = len(f) - 1
    while deg > 0 and f[deg] == 0:
        deg -= 1
    codeg = 0
    while codeg < deg and f[codeg] == 0:
        codeg += 1
    return deg - codeg


def dense_from_csr(nrows, ncols, row_ptr, col, val):
    """Dense list-of-lists of Python ints; repeated (i, j) entries add up."""
    a = [[0] * ncols for _ in range(nrows)]
    for i in range(nrows):
        for k in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            a[i][int(col[k])] += int(val[k])
    return a


def dense_matvec(a, x, m):
    return [sum(aij * int(xj) for aij, xj in zip(row, x)) % m for row in a]


def dense_transpose(a):
    return [list(r) for r in zip(*a)] if a else []


def dense_matmul(a, b, m):
    bt = dense_transpose(b)
    return [[sum(x * y for x, y in zip(r, c)) % m for c in bt] for r in a]
