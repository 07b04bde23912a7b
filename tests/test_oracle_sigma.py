"""Pins of the sigma-basis oracle (oracle/sigma.py) to things other than
itself: the approximant property and the determinant x^(sum of degree
increases) for random inputs; the scalar case against Berlekamp-Massey
(oracle/linalg.py); block Wiedemann's rank (deg det - codeg det of the
minimal generator) against Gaussian elimination mod p on matrices of known
rank; and M-Basis against PM-Basis."""
import numpy as np
import pytest

from oracle import linalg, sigma

P65521 = 65521


def _rand_F(seed, d, m, n, p):
    return np.random.default_rng(seed).integers(0, p, (d, m, n)).astype(object)


@pytest.mark.parametrize("shift", [[0, 0, 0, 0], [2, 0, 1, 0]])
def test_approximant_property_and_determinant(shift):
    p, d = P65521, 9
    F = _rand_F(1, d, 4, 2, p)
    results = [sigma.mbasis(F, d, shift, p), sigma.pmbasis(F, d, shift, p, base=2)]
    for P, delta in results:
        for k in range(d):
            assert not np.any(sigma.coeff(P, F, k, p)), k
        grow = sum(a - b for a, b in zip(delta, shift))
        assert grow == d * 2                  # generic F: two pivots at every order
        dp = sigma.det_poly(P, p)
        assert sigma.degree_and_codegree(dp) == (grow, grow)
    assert sorted(results[0][1]) == sorted(results[1][1])


@pytest.mark.parametrize("L", [1, 3, 6])
def test_scalar_case_is_berlekamp_massey(L):
    p = P65521
    rng = np.random.default_rng(L)
    c = [int(v) for v in rng.integers(1, p, L)]
    s = [int(v) for v in rng.integers(0, p, L)]
    N = 2 * L + 2
    while len(s) < N:
        s.append(sum(c[i] * s[-1 - i] for i in range(L)) % p)
    C, LL = linalg.berlekamp_massey(s, p)
    assert LL == L
    F = np.zeros((N, 2, 1), dtype=object)
    F[:, 0, 0] = s
    F[0, 1, 0] = p - 1                                  # rows (u, v): u S - v = 0 mod x^N
    for P, delta in (sigma.mbasis(F, N, [0, 0], p), sigma.pmbasis(F, N, [0, 0], p, base=2)):
        r = int(np.argmin(delta))
        assert delta[r] == L
        u = [int(P[k, r, 0]) for k in range(P.shape[0])]
        inv = pow(u[0], p - 2, p)
        u = [v * inv % p for v in u]
        while len(u) > 1 and u[-1] == 0:
            u.pop()
        assert u == list(C)


def _inverse_mod(P, p):
    n = len(P)
    aug = [list(row) + [int(i == j) for j in range(n)] for i, row in enumerate(P)]
    for c in range(n):
        piv = next(i for i in range(c, n) if aug[i][c] % p)
        aug[c], aug[piv] = aug[piv], aug[c]
        inv = pow(aug[c][c], p - 2, p)
        aug[c] = [(t * inv) % p for t in aug[c]]
        for i in range(n):
            if i != c and aug[i][c]:
                f = aug[i][c]
                aug[i] = [(t - f * w) % p for t, w in zip(aug[i], aug[c])]
    return [row[n:] for row in aug]


@pytest.mark.parametrize("p", [P65521, 2**31 - 1])
def test_block_wiedemann_rank(p):
    # A = Q diag(d_1..d_r, 0..0) Q^-1; S_i = X^T A^i Y; the s rows of least
    # degree of an order-L sigma-basis of [S(x); -I] give the generator, and
    # deg det - codeg det is the rank
    n, s = 12, 3
    rng = np.random.default_rng(5)
    for r in (0, 4, 7, 11, 12):
        while True:
            Q = rng.integers(0, p, (n, n)).tolist()
            if linalg.rank_mod_p(Q, p) == n:
                break
        dvals = rng.choice(np.arange(1, 10**4), r, replace=False).tolist() + [0] * (n - r)
        D = [[dvals[i] if i == j else 0 for j in range(n)] for i in range(n)]
        A = linalg.dense_matmul(linalg.dense_matmul(Q, D, p), _inverse_mod(Q, p), p)
        assert linalg.rank_mod_p(A, p) == r
        X = rng.integers(0, p, (n, s)).tolist()
        V = rng.integers(0, p, (n, s)).tolist()
        L = 2 * (n // s) + 4
        F = np.zeros((L, 2 * s, s), dtype=object)
        for i in range(L):
            F[i, :s, :] = np.array([[sum(X[k][a] * V[k][b] for k in range(n)) % p for b in range(s)]
                                    for a in range(s)], dtype=object)
            V = linalg.dense_matmul(A, V, p)
        for i in range(s):
            F[0, s + i, i] = p - 1
        P, delta = sigma.pmbasis(F, L, [0] * (2 * s), p, base=3)
        rows = sorted(range(2 * s), key=lambda i: (delta[i], i))[:s]
        dg, cdg = sigma.degree_and_codegree(sigma.det_poly(sigma.trim(P[:, rows, :s]), p))
        assert dg - cdg == r, (r, delta)
        assert dg == sum(delta[i] for i in rows)    # the generator is row reduced


def _count_approximants(F, d, shift, D, p):
    """Brute force: how many row vectors v with deg v_i <= D - s_i satisfy
    v F = 0 mod x^d (every vector enumerated, no algebra)."""
    import itertools
    m, n = F.shape[1], F.shape[2]
    sizes = [max(0, D - s + 1) for s in shift]
    count = 0
    for flat in itertools.product(range(p), repeat=sum(sizes)):
        coeffs, pos = [], 0
        for sz in sizes:
            coeffs.append(flat[pos:pos + sz])
            pos += sz
        ok = True
        for k in range(d):
            for j in range(n):
                acc = 0
                for i in range(m):
                    for t, c in enumerate(coeffs[i]):
                        if c and k - t >= 0 and k - t < F.shape[0]:
                            acc += c * int(F[k - t, i, j])
                if acc % p:
                    ok = False
                    break
            if not ok:
                break
        count += ok
    return count


@pytest.mark.parametrize("p,m,n,d,shift,seed", [(3, 2, 1, 5, [0, 0], 1), (2, 3, 1, 4, [0, 1, 0], 2),
                                                (2, 3, 2, 3, [0, 0, 0], 3), (3, 3, 2, 2, [1, 0, 0], 4)])
def test_degrees_are_minimal_by_enumeration(p, m, n, d, shift, seed):
    # a reduced basis has the predictable-degree property: the approximants of
    # shifted degree <= D form a space of dimension sum_i max(0, D - delta_i + 1);
    # counting them one by one pins the degrees without the algorithm
    F = np.random.default_rng(seed).integers(0, p, (d, m, n)).astype(object)
    for P, delta in (sigma.mbasis(F, d, shift, p), sigma.pmbasis(F, d, shift, p, base=1)):
        for D in range(0, 3):
            want = p ** sum(max(0, D - dl + 1) for dl in delta)
            assert _count_approximants(F, d, shift, D, p) == want, (D, delta)


def _pmul(a, b, p):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] = (out[i + j] + x * y) % p
    return out


@pytest.mark.parametrize("n,e,seed", [(1, 4, 1), (3, 2, 2), (4, 3, 3)])
def test_det_poly_of_triangular_matrices(n, e, seed):
    # det of a triangular polynomial matrix is the product of its diagonal
    # (by plain polynomial multiplication); rows shifted by powers of x give
    # a nonzero codegree
    p = 10007
    rng = np.random.default_rng(seed)
    P = np.zeros((e + 1, n, n), dtype=object)
    for i in range(n):
        for j in range(i, n):
            P[:, i, j] = [int(v) for v in rng.integers(0, p, e + 1)]
    P[0, 0, 0] = 0                       # x divides the first diagonal entry
    want = [1]
    for i in range(n):
        want = _pmul(want, [int(P[k, i, i]) for k in range(e + 1)], p)
    got = sigma.det_poly(P, p)
    assert got[:len(want)] == want and not any(got[len(want):])
    dg, cdg = sigma.degree_and_codegree(got)
    assert cdg >= 1


def test_det_poly_2x2_closed_form():
    # det [[a, b], [c, d]] = a d - b c, by plain polynomial multiplication
    p = 65521
    rng = np.random.default_rng(7)
    a, b, c, d = ([int(v) for v in rng.integers(0, p, 4)] for _ in range(4))
    P = np.zeros((4, 2, 2), dtype=object)
    for k in range(4):
        P[k] = [[a[k], b[k]], [c[k], d[k]]]
    ad, bc = _pmul(a, d, p), _pmul(b, c, p)
    want = [(x - y) % p for x, y in zip(ad, bc)]
    got = sigma.det_poly(P, p)
    assert got[:len(want)] == want and not any(got[len(want):])
