"""The sequence's purpose (Sec. 3): the rank read off the minimal polynomial
of a GPU-produced scalar sequence S_i = u^T A^i v (s = 1), with
Berlekamp-Massey and deg f - codeg f on the CPU (oracle side), against
Gaussian elimination mod p.  Matrices are built with a known rank:
A = P diag(d_1..d_r, 0..0) P^-1 with distinct nonzero d, whose minimal
polynomial is x * prod(x - d_i) when r < n."""
import numpy as np
import pytest

import gen
from helpers import to_dev, to_host
from oracle import linalg

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("p", [65521, 2**31 - 1])
def test_rank_from_gpu_sequence(lib, p):
    n = 40
    rng = np.random.default_rng(17)
    for r in (0, 9, 25, 39, 40):
        while True:
            P = rng.integers(0, p, (n, n)).tolist()
            if linalg.rank_mod_p(P, p) == n:
                break
        d = rng.choice(np.arange(1, min(p, 10**6)), r, replace=False).tolist() + [0] * (n - r)
        D = [[d[i] if i == j else 0 for j in range(n)] for i in range(n)]
        Ad = linalg.dense_matmul(linalg.dense_matmul(P, D, p), _inverse_mod(P, p), p)
        assert linalg.rank_mod_p(Ad, p) == r
        A = gen.dense_to_csr(np.array(Ad, dtype=np.int64), p)
        M = lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.NONE)
        u = gen.uniform_block(50 + r, n, 1, p).reshape(n, 1)
        v = gen.uniform_block(51 + r, n, 1, p, key=2).reshape(n, 1)
        S = to_host(M.block_sequence(to_dev(u), to_dev(v), 2 * n + 4)).reshape(-1)
        C, L = linalg.berlekamp_massey(S.tolist(), p)
        f = linalg.minpoly_from_bm(C, L)
        assert linalg.rank_from_minpoly(f) == r, (r, L)
