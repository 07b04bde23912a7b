"""The σ-basis library's schedule, restated step by step on the CPU and
compared with oracle/sigma.py (no GPU): the M-Basis leaf eliminates fraction
free (row r becomes a r - b q) and divides each row by the product of its
multipliers at the end, in the order the CUDA leaf uses (a column
elimination first, then the same operations applied position by position,
then the pivot rows times x); PM-Basis sizes its products by the degree
bound max(delta) - min(shift), which must never drop a nonzero coefficient."""
import numpy as np
import pytest

from oracle import sigma


def _leaf(F, d, shift, p):
    m, n = F.shape[1], F.shape[2]
    R = [[[int(F[t][r][c]) % p for c in range(n)] for r in range(m)] for t in range(d)]
    P = [[[int(r == c) if t == 0 else 0 for c in range(m)] for r in range(m)] for t in range(d + 1)]
    delta, scale = list(shift), [1] * m
    for k in range(d):
        rank = [sum(1 for j in range(m) if (delta[j], j) < (delta[r], r)) for r in range(m)]
        col = [[R[k][r][c] for r in range(m)] for c in range(n)]
        pivots, ops = set(), []
        for j in range(n):
            cands = [r for r in range(m) if r not in pivots and col[j][r]]
            if not cands:
                continue
            q = min(cands, key=lambda r: rank[r])
            a = col[j][q]
            upd = [r for r in cands if rank[r] > rank[q]]
            g = {r: p - col[j][r] for r in upd}
            for c in range(j + 1, n):
                for r in upd:
                    col[c][r] = (a * col[c][r] + g[r] * col[c][q]) % p
            for r in upd:
                scale[r] = scale[r] * a % p
            ops.append((q, a, g))
            pivots.add(q)
        for r in pivots:
            delta[r] += 1

        def apply(vec):
            for q, a, g in ops:
                vq = vec[q]
                for r, gr in g.items():
                    vec[r] = (a * vec[r] + gr * vq) % p
            return vec
        for t in range(k, d):
            for c in range(n):
                v = apply([R[t][r][c] for r in range(m)])
                for r in range(m):
                    R[t][r][c] = v[r]
        for t in range(k + 1):
            for c in range(m):
                v = apply([P[t][r][c] for r in range(m)])
                for r in range(m):
                    P[t][r][c] = v[r]
        for q in pivots:
            for c in range(n):
                for t in range(d - 1, k, -1):
                    R[t][q][c] = R[t - 1][q][c]
                R[k][q][c] = 0
            for c in range(m):
                for t in range(k + 1, 0, -1):
                    P[t][q][c] = P[t - 1][q][c]
                P[0][q][c] = 0
    inv = [pow(c, p - 2, p) for c in scale]
    out = np.array([[[P[t][r][c] * inv[r] % p for c in range(m)] for r in range(m)] for t in range(d + 1)],
                   dtype=object)
    return out, delta


def _bound(delta, shift, d):
    return max(0, min(d, max(delta) - min(shift)))


def _pmbasis(F, d, shift, p, base):
    m = F.shape[1]
    if d <= base:
        P, delta = _leaf(F, d, shift, p)
        e = _bound(delta, shift, d)
        assert not np.any(P[e + 1:])
        return P, delta, e
    d1 = (d + 1) // 2
    P1, delta1, e1 = _pmbasis(F[:d1], d1, shift, p, base)
    C = sigma.poly_mul(P1[:e1 + 1], F[:d], p)          # e1 + d coefficients, as the library allocates
    P2, delta2, e2 = _pmbasis(C[d1:d], d - d1, delta1, p, base)
    P = np.zeros((d + 1, m, m), dtype=object)
    P[:e1 + e2 + 1] = sigma.poly_mul(P2[:e2 + 1], P1[:e1 + 1], p)
    e = min(e1 + e2, _bound(delta2, shift, d))
    assert not np.any(P[e + 1:])
    return P, delta2, e


@pytest.mark.parametrize("p,m,n,d,base,shift,sparse", [
    (65521, 2, 1, 14, 4, [0, 0], False),
    (65521, 8, 4, 50, 8, [0] * 8, False),
    (2**31 - 1, 6, 3, 37, 16, [2, 0, 1, 0, 3, 0], False),
    (7, 8, 4, 30, 4, [0] * 8, True),
    (65521, 5, 3, 23, 3, [1, 0, 0, 2, 0], False),
    (65521, 4, 1, 9, 32, [0, 5, 0, 1], False),
])
def test_schedule_equals_oracle(p, m, n, d, base, shift, sparse):
    rng = np.random.default_rng(d * 7 + m)
    F = rng.integers(0, p, (d, m, n))
    if sparse:
        F = F * (rng.random((d, m, n)) < 0.3)
        F[:, :, 1] = 0
    F = F.astype(object)
    P, delta, e = _pmbasis(F, d, shift, p, base)
    Po, do = sigma.pmbasis(F, d, shift, p, base=base)
    want = np.zeros((d + 1, m, m), dtype=object)
    want[:Po.shape[0]] = Po
    assert delta == do and np.array_equal(P, want)


def test_schedule_on_a_rank_deficient_wiedemann_input():
    p, s, L = 65521, 3, 20
    rng = np.random.default_rng(4)
    F = np.zeros((L, 2 * s, s), dtype=object)
    F[:, :s, :] = rng.integers(0, p, (L, s, s))
    F[:, :s, 2] = 0
    for i in range(s):
        F[0, s + i, i] = p - 1
    P, delta, _ = _pmbasis(F, L, [0] * (2 * s), p, 4)
    Po, do = sigma.pmbasis(F, L, [0] * (2 * s), p, base=4)
    want = np.zeros((L + 1, 2 * s, 2 * s), dtype=object)
    want[:Po.shape[0]] = Po
    assert delta == do and np.array_equal(P, want)
