"""Pins for the CPU oracle: it is checked against what the paper and the
mathematics fix, never against itself.

* the worked example of Sec. 2.4.1 (A = [[2,1],[0,3]] over Z/27Z), golden file;
* dense brute force over Python integers (tiny inputs, every modulus class);
* exhaustive inputs over (Z/3Z)^8;
* closed forms: all-(m-1) rows, identity and permutation matrices, diagonal
  sequences by fast exponentiation, Fermat periodicity;
* invariants: linearity, the transpose identity y^T(Ax) = (A^T y)^T x;
* the sequence's purpose (Sec. 3): Berlekamp-Massey on the scalar sequence
  recovers the Krylov dimension and the rank of a matrix built with a known
  rank, cross-checked by Gaussian elimination.
"""
import os

import numpy as np
import pytest

import gen
import oracle
from oracle import linalg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODULI = [2, 3, 27, 65521, 2**31 - 1, 4294967291]


def test_worked_example_mod27():
    rows = np.loadtxt(os.path.join(GOLDEN, "jit_example_mod27.txt"),
                      dtype=np.int64, ndmin=2)
    A = gen.dense_to_csr([[2, 1], [0, 3]], 27)
    for x0, x1, y0, y1, e0, e1 in rows:
        y = oracle.csr_spmv(A, np.array([x0, x1]), y=np.array([y0, y1]),
                            alpha=1, beta=1)
        assert list(y) == [e0, e1]


@pytest.mark.parametrize("m", MODULI)
@pytest.mark.parametrize("nvec", [1, 3])
def test_dense_brute_force(m, nvec):
    for seed in range(4):
        A = gen.random_small(seed + 10 * nvec, 13, 9, 0.3, m, pm_fraction=0.3,
                             dup=(seed % 2 == 1))
        rng = np.random.default_rng(seed)
        x = (rng.random((A.ncols, nvec)) * m).astype(np.uint64).astype(np.uint32)
        y0 = (rng.random((A.nrows, nvec)) * m).astype(np.uint64).astype(np.uint32)
        alpha, beta = int(rng.integers(0, m)), int(rng.integers(0, m))
        got = oracle.csr_spmv(A, x, y=y0, alpha=alpha, beta=beta)
        d = linalg.dense_from_csr(A.nrows, A.ncols, A.row_ptr, A.col, A.val)
        for v in range(nvec):
            ax = linalg.dense_matvec(d, x[:, v], m)
            want = [(alpha * a + beta * int(b)) % m for a, b in zip(ax, y0[:, v])]
            assert list(got[:, v]) == want
        gotT = oracle.csr_spmv_transpose(A, y0, alpha=alpha)
        dt = linalg.dense_transpose(d)
        for v in range(nvec):
            want = [(alpha * a) % m for a in linalg.dense_matvec(dt, y0[:, v], m)]
            assert list(gotT[:, v]) == want


def test_exhaustive_z3():
    m = 3
    A = gen.random_small(5, 8, 8, 0.5, m)
    grid = np.array(np.meshgrid(*[range(3)] * 8, indexing="ij")).reshape(8, -1)
    X = grid.astype(np.uint32)                      # 8 x 6561, every x
    Y = oracle.csr_spmv(A, X)
    d = linalg.dense_from_csr(8, 8, A.row_ptr, A.col, A.val)
    for v in range(0, X.shape[1], 37):
        assert list(Y[:, v]) == linalg.dense_matvec(d, X[:, v], m)
    # all 3^8 images agree with the dense product computed in numpy int64
    D = np.array(d, dtype=np.int64)
    assert np.array_equal(Y.astype(np.int64), (D @ X.astype(np.int64)) % 3)


@pytest.mark.parametrize("m", [65521, 2**31 - 1, 4294967291])
def test_all_max_closed_form(m):
    # rows of L entries all equal to m-1 against x = m-1: each product is
    # (m-1)^2 = 1 (mod m), so y_i = L_i mod m, far past 64-bit range.
    lengths = np.array([0, 1, 2, 5, 4000, 10_000])
    n = lengths.size
    A = gen.CSR(n, 10_000, np.concatenate([[0], np.cumsum(lengths)]),
                np.concatenate([np.arange(L) for L in lengths]).astype(np.int32),
                np.full(lengths.sum(), m - 1, dtype=np.uint32), m)
    x = np.full(10_000, m - 1, dtype=np.uint32)
    y = oracle.csr_spmv(A, x)
    assert list(y) == [int(L) % m for L in lengths]
    yT = oracle.csr_spmv_transpose(A, np.full(n, m - 1, dtype=np.uint32))
    counts = np.zeros(10_000, dtype=np.int64)
    for L in lengths:
        counts[:L] += 1
    assert list(yT) == [int(c) % m for c in counts]


def test_identity_and_permutation():
    n, m = 500, 65521
    rng = np.random.default_rng(3)
    x = rng.integers(0, m, n).astype(np.uint32)
    I = gen.dense_to_csr(np.eye(n, dtype=np.int64), m)
    assert np.array_equal(oracle.csr_spmv(I, x), x)
    perm = rng.permutation(n)
    P = gen.CSR(n, n, np.arange(n + 1, dtype=np.int64), perm.astype(np.int32),
                np.ones(n, dtype=np.uint32), m)
    assert np.array_equal(oracle.csr_spmv(P, x), x[perm])
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    assert np.array_equal(oracle.csr_spmv_transpose(P, x), x[inv])
    # -1 entries: (m-1) * x = -x
    Pm = gen.CSR(n, n, P.row_ptr, P.col, np.full(n, m - 1, dtype=np.uint32), m)
    assert np.array_equal(oracle.csr_spmv(Pm, x), (m - x[perm].astype(np.int64)) % m)


@pytest.mark.parametrize("m", [3, 65521, 2**31 - 1])
def test_linearity_and_transpose_identity(m):
    A = gen.tiny_matrix(m=m)
    rng = np.random.default_rng(11)
    x1 = rng.integers(0, m, A.ncols).astype(np.uint32)
    x2 = rng.integers(0, m, A.ncols).astype(np.uint32)
    a, b = int(rng.integers(1, m)), int(rng.integers(1, m))
    comb = ((a * x1.astype(object) + b * x2.astype(object)) % m).astype(np.uint32)
    lhs = oracle.csr_spmv(A, comb)
    y1 = oracle.csr_spmv(A, x1)
    y2 = oracle.csr_spmv(A, x2)
    rhs = ((a * y1.astype(object) + b * y2.astype(object)) % m).astype(np.uint32)
    assert np.array_equal(lhs, rhs)
    # alpha/beta form equals the same combination
    ab = oracle.csr_spmv(A, x1, y=y2, alpha=a, beta=b)
    assert np.array_equal(ab, ((a * y1.astype(object) + b * y2.astype(object)) % m).astype(np.uint32))
    # y^T (A x) == (A^T y)^T x  (mod m)
    y = rng.integers(0, m, A.nrows).astype(np.uint32)
    Ax = oracle.csr_spmv(A, x1)
    ATy = oracle.csr_spmv_transpose(A, y)
    lhs = sum(int(u) * int(v) for u, v in zip(y, Ax)) % m
    rhs = sum(int(u) * int(v) for u, v in zip(ATy, x1)) % m
    assert lhs == rhs


def test_empty_shapes():
    m = 65521
    E = gen.CSR(0, 5, np.zeros(1, dtype=np.int64), np.zeros(0, np.int32),
                np.zeros(0, np.uint32), m)
    assert oracle.csr_spmv(E, np.arange(5, dtype=np.uint32)).size == 0
    assert list(oracle.csr_spmv_transpose(E, np.zeros(0, np.uint32))) == [0] * 5
    Z = gen.CSR(4, 4, np.zeros(5, dtype=np.int64), np.zeros(0, np.int32),
                np.zeros(0, np.uint32), m)
    y = oracle.csr_spmv(Z, np.arange(4, dtype=np.uint32),
                        y=np.array([1, 2, 3, 4], dtype=np.uint32), alpha=5, beta=2)
    assert list(y) == [2, 4, 6, 8]


def test_sequence_dense_powers():
    p, n, s, L = 65521, 12, 3, 9
    A = gen.random_small(21, n, n, 0.3, p, pm_fraction=0.2)
    X = gen.uniform_block(1, n, s, p)
    Y = gen.uniform_block(2, n, s, p, key=1)
    S, Vn = oracle.csr_block_sequence(A, X, Y, L, want_next=True)
    d = linalg.dense_from_csr(n, n, A.row_ptr, A.col, A.val)
    Xt = linalg.dense_transpose(X.tolist())
    V = Y.tolist()
    for i in range(L):
        assert S[i].tolist() == linalg.dense_matmul(Xt, V, p)
        V = linalg.dense_matmul(d, V, p)
    assert Vn.tolist() == V


def test_sequence_diagonal_closed_form():
    # A = diag(d): S_i[a][b] = sum_k X[k][a] d_k^i Y[k][b]  (mod p)
    p, n, s, L = 65521, 40, 4, 300
    rng = np.random.default_rng(5)
    d = rng.integers(0, p, n)
    A = gen.CSR(n, n, np.arange(n + 1, dtype=np.int64),
                np.arange(n, dtype=np.int32), d.astype(np.uint32), p)
    X = gen.uniform_block(3, n, s, p)
    Y = gen.uniform_block(4, n, s, p)
    S = oracle.csr_block_sequence(A, X, Y, L)
    for i in (0, 1, 2, 17, 150, L - 1):
        di = [pow(int(v), i, p) for v in d]
        want = [[sum(int(X[k, a]) * di[k] * int(Y[k, b]) for k in range(n)) % p
                 for b in range(s)] for a in range(s)]
        assert S[i].tolist() == want


def test_sequence_fermat_period():
    # diag with nonzero entries mod 13: d^12 = 1, so S_{i+12} = S_i
    p, n, s = 13, 30, 2
    rng = np.random.default_rng(9)
    d = rng.integers(1, p, n)
    A = gen.CSR(n, n, np.arange(n + 1, dtype=np.int64),
                np.arange(n, dtype=np.int32), d.astype(np.uint32), p)
    X = gen.uniform_block(5, n, s, p)
    Y = gen.uniform_block(6, n, s, p)
    S = oracle.csr_block_sequence(A, X, Y, 40)
    assert np.array_equal(S[12:40], S[0:28])


def test_sequence_permutation_closed_form():
    p, n, s, L = 65521, 50, 2, 25
    rng = np.random.default_rng(2)
    perm = rng.permutation(n)
    P = gen.CSR(n, n, np.arange(n + 1, dtype=np.int64), perm.astype(np.int32),
                np.ones(n, dtype=np.uint32), p)
    X = gen.uniform_block(7, n, s, p)
    Y = gen.uniform_block(8, n, s, p)
    S = oracle.csr_block_sequence(P, X, Y, L)
    idx = np.arange(n)
    for i in range(L):
        Vi = Y[idx]                      # (P^i Y)[k] = Y[perm^i(k)]
        want = (X.astype(object).T.dot(Vi.astype(object))) % p
        assert S[i].tolist() == want.tolist()
        idx = perm[idx]


def test_sequence_two_sided_and_resume():
    p, s = 65521, 4
    A = gen.wiedemann_matrix(n=300)
    X = gen.uniform_block(9, 300, s, p)
    Y = gen.uniform_block(10, 300, s, p)
    S = oracle.csr_block_sequence(A, X, Y, 12)
    # S_i = ((A^T)^j X)^T (A^(i-j) Y)
    Xj = X.copy()
    for _ in range(3):
        Xj = oracle.csr_spmv_transpose(A, Xj)
    S2 = oracle.csr_block_sequence(A, Xj, Y, 9)
    assert np.array_equal(S2, S[3:12])
    # resuming from A^5 Y continues the sequence
    S5, V5 = oracle.csr_block_sequence(A, X, Y, 5, want_next=True)
    Sr = oracle.csr_block_sequence(A, X, V5, 7)
    assert np.array_equal(np.concatenate([S5, Sr]), S)


def _krylov_dim(d, v, p):
    n = len(v)
    K, w = [], [int(t) for t in v]
    for _ in range(n + 1):
        K.append(w)
        w = linalg.dense_matvec(d, w, p)
    return linalg.rank_mod_p(K, p)


def test_scalar_sequence_minpoly_matches_krylov():
    p, n = 65521, 24
    for seed in range(3):
        A = gen.random_small(40 + seed, n, n, 0.15, p, pm_fraction=0.5)
        u = gen.uniform_block(11 + seed, n, 1, p)
        v = gen.uniform_block(12 + seed, n, 1, p, key=3)
        S = oracle.csr_block_sequence(A, u, v, 2 * n + 2)
        C, L = linalg.berlekamp_massey(S.reshape(-1).tolist(), p)
        d = linalg.dense_from_csr(n, n, A.row_ptr, A.col, A.val)
        assert L == _krylov_dim(d, v, p)


def test_rank_from_sequence_known_rank():
    # A = P diag(d_1..d_r, 0..0) P^-1 with distinct nonzero d: minimal
    # polynomial x * prod(x - d_i), so deg - codeg = r = rank(A).
    p, n = 65521, 20
    rng = np.random.default_rng(1)
    for r in (0, 7, 19, 20):
        while True:
            P = rng.integers(0, p, (n, n)).tolist()
            if linalg.rank_mod_p(P, p) == n:
                break
        # inverse of P by Gauss-Jordan on [P | I]
        aug = [row + [int(i == j) for j in range(n)] for i, row in enumerate(P)]
        for c in range(n):
            piv = next(i for i in range(c, n) if aug[i][c] % p)
            aug[c], aug[piv] = aug[piv], aug[c]
            inv = pow(aug[c][c], p - 2, p)
            aug[c] = [(t * inv) % p for t in aug[c]]
            for i in range(n):
                if i != c and aug[i][c]:
                    f = aug[i][c]
                    aug[i] = [(t - f * w) % p for t, w in zip(aug[i], aug[c])]
        Pinv = [row[n:] for row in aug]
        dvals = rng.choice(np.arange(1, p), r, replace=False).tolist() + [0] * (n - r)
        D = [[dvals[i] if i == j else 0 for j in range(n)] for i in range(n)]
        Ad = linalg.dense_matmul(linalg.dense_matmul(P, D, p), Pinv, p)
        assert linalg.rank_mod_p(Ad, p) == r
        A = gen.dense_to_csr(np.array(Ad, dtype=np.int64), p)
        u = gen.uniform_block(30 + r, n, 1, p)
        v = gen.uniform_block(31 + r, n, 1, p, key=5)
        S = oracle.csr_block_sequence(A, u, v, 2 * n + 4)
        C, L = linalg.berlekamp_massey(S.reshape(-1).tolist(), p)
        f = linalg.minpoly_from_bm(C, L)
        assert linalg.rank_from_minpoly(f) == r


def test_generators_shapes():
    A = gen.tiny_matrix()
    assert A.nrows == 2000 and A.nnz == 20_000
    assert np.all(np.diff(A.row_ptr) == 10)
    pm = np.mean((A.val == 1) | (A.val == A.modulus - 1))
    assert 0.15 < pm < 0.25
    W = gen.wiedemann_matrix(n=1000)
    L = W.row_lengths()
    assert L.min() >= 8 and L.max() <= 10
    for i in range(W.nrows):
        c = W.col[W.row_ptr[i]:W.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_threaded_oracle_equals_single_thread():
    # the all-core timing form splits rows over threads; its results are the
    # single-thread definition's, for both products, alpha/beta and blocks
    A = gen.powerlaw_matrix(seed=5, n=3000, lmax=300, m=2**31 - 1, pm_fraction=0.3)
    x = gen.uniform_block(3, A.ncols, 3, A.modulus).reshape(-1, 3)
    y0 = gen.uniform_block(4, A.nrows, 3, A.modulus).reshape(-1, 3)
    for t in (2, 5, 16):
        assert np.array_equal(oracle.csr_spmv(A, x, y=y0, alpha=5, beta=7, threads=t),
                              oracle.csr_spmv(A, x, y=y0, alpha=5, beta=7))
        assert np.array_equal(oracle.csr_spmv_transpose(A, x, y=y0, alpha=5, beta=7, threads=t),
                              oracle.csr_spmv_transpose(A, x, y=y0, alpha=5, beta=7))
