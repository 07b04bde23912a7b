"""GPU parity of the block Wiedemann sequence S_i = X^T A^i Y mod p (Sec. 3,
step 1) against the CPU oracle, on the persistent-kernel path and the
per-launch path, plus resume, closed forms and the bounded barrier wait."""
import numpy as np
import pytest

import gen
import oracle
from helpers import to_dev, to_host, with_modulus

pytestmark = pytest.mark.gpu


def run(ff, A, X, Y, nsteps, mode=0, want_next=False, **kw):
    M = ff.Matrix.from_csr(A, sequence_mode=mode, **kw)
    out = M.block_sequence(to_dev(X), to_dev(Y), nsteps, want_next=want_next)
    if want_next:
        return to_host(out[0]), to_host(out[1])
    return to_host(out)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("s", [1, 3, 16])
def test_small_sequence(lib, mode, s):
    p = 65521
    A = gen.wiedemann_matrix(seed=5, n=1003)
    X = gen.uniform_block(1, A.nrows, s, p).reshape(A.nrows, s)
    Y = gen.uniform_block(2, A.nrows, s, p, key=1).reshape(A.nrows, s)
    S = run(lib, A, X, Y, 41, mode).reshape(41, s, s)
    want = oracle.csr_block_sequence(A, X, Y, 41)
    assert np.array_equal(S, want)


@pytest.mark.parametrize("mode", [0, 1])
def test_resume_from_checkpoint(lib, mode):
    p, s = 65521, 16
    A = gen.wiedemann_matrix(seed=6, n=2500)
    X = gen.uniform_block(3, A.nrows, s, p)
    Y = gen.uniform_block(4, A.nrows, s, p, key=2)
    S1, V = run(lib, A, X, Y, 13, mode, want_next=True)
    S2 = run(lib, A, X, V, 17, mode)
    want, Vw = oracle.csr_block_sequence(A, X, Y, 13, want_next=True)
    assert np.array_equal(V, Vw)
    full = oracle.csr_block_sequence(A, X, Y, 30)
    assert np.array_equal(np.concatenate([S1, S2]), full)


def test_general_matrix_and_large_prime(lib):
    # power-law rows do not fit the DIA + ELL_R layout; 2^31-1 needs 4 limbs:
    # both go through the per-launch path
    for A in (gen.powerlaw_matrix(seed=3, n=4000, lmax=800, m=65521),
              with_modulus(gen.wiedemann_matrix(seed=8, n=1500), 2**31 - 1)):
        s, p = 8, A.modulus
        X = gen.uniform_block(5, A.nrows, s, p)
        Y = gen.uniform_block(6, A.nrows, s, p, key=3)
        S = run(lib, A, X, Y, 20)
        assert np.array_equal(S, oracle.csr_block_sequence(A, X, Y, 20))


def test_diagonal_closed_form_long(lib):
    # diag(d): S_i[a][b] = sum_k X[k][a] d_k^i Y[k][b]; far steps checked
    p, n, s, L = 65521, 5000, 16, 3000
    rng = np.random.default_rng(3)
    d = rng.integers(1, p, n)
    A = gen.CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32),
                d.astype(np.uint32), p)
    X = gen.uniform_block(7, n, s, p)
    Y = gen.uniform_block(8, n, s, p, key=4)
    S = run(lib, A, X, Y, L)
    for i in (0, 1, 999, L - 1):
        di = np.array([pow(int(v), i, p) for v in d], dtype=object)
        want = (X.astype(object).T.dot(Y.astype(object) * di[:, None])) % p
        assert np.array_equal(S[i].astype(object), want), i


def test_timeout_hook_returns_status_and_handle_survives(lib):
    p, s = 65521, 16
    A = gen.wiedemann_matrix(seed=9, n=4000)
    X = gen.uniform_block(9, A.nrows, s, p)
    Y = gen.uniform_block(10, A.nrows, s, p, key=5)
    M = lib.Matrix.from_csr(A, test_hooks=1, barrier_spin_limit=20_000)
    with pytest.raises(lib.FFSPMVError) as e:
        M.block_sequence(to_dev(X), to_dev(Y), 5)
    assert e.value.status == 6
    # the same device stays usable: a normal handle still matches the oracle
    S = run(lib, A, X, Y, 5)
    assert np.array_equal(S, oracle.csr_block_sequence(A, X, Y, 5))


def test_full_size_wiedemann(lib):
    # 100k x 100k, s = 16, the benchmark's 12 502 steps; the oracle checks
    # the first 24 steps whole and one (a, b) entry over every step.
    p, s = 65521, 16
    A = gen.wiedemann_matrix(seed=1003)
    n = A.nrows
    L = 2 * n // s + 2
    X = gen.uniform_block(1003, n, s, p)
    Y = gen.uniform_block(1003, n, s, p, key=1)
    S = run(lib, A, X, Y, L)
    assert S.shape == (L, s, s)
    assert np.array_equal(S[:24], oracle.csr_block_sequence(A, X, Y, 24))
    a, b = 5, 11
    col = oracle.csr_block_sequence(A, X[:, a:a + 1], Y[:, b:b + 1], L).reshape(L)
    assert np.array_equal(S[:, a, b], col)
