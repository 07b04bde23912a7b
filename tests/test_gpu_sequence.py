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


@pytest.mark.parametrize("mode", [0, 1])
def test_resume_with_start_step_and_state(lib, mode):
    # the boundary's resume form: start_step > 0 continues from d_V_state,
    # which is advanced in place; d_Y is not read
    import torch
    p, s = 65521, 8
    A = gen.wiedemann_matrix(seed=16, n=3000)
    X = gen.uniform_block(13, A.nrows, s, p)
    Y = gen.uniform_block(14, A.nrows, s, p, key=6)
    M = lib.Matrix.from_csr(A, sequence_mode=mode)
    Xd = to_dev(X)
    S1, V = M.block_sequence(Xd, to_dev(Y), 11, want_next=True)
    S2 = M.resume_sequence(Xd, V, 11, 9)
    S3 = M.resume_sequence(Xd, V, 20, 6)
    torch.cuda.synchronize()
    full, Vw = oracle.csr_block_sequence(A, X, Y, 26, want_next=True)
    got = np.concatenate([to_host(S1), to_host(S2), to_host(S3)]).reshape(26, s, s)
    assert np.array_equal(got, full)
    assert np.array_equal(to_host(V).reshape(A.nrows, s), Vw)
    with pytest.raises(lib.FFSPMVError) as e:      # start_step > 0 needs the state
        lib.spmv_block_sequence(M.handle, Xd, to_dev(Y), s, 3, 2,
                                torch.empty((2, s, s), dtype=torch.int32, device="cuda"), None)
    assert e.value.status == 1


def test_one_handle_new_blocks_each_call(lib):
    # the captured graph of the persistent kernel reads X and Y: a later call
    # on the same handle with other blocks (same sizes) must use them
    import torch
    p, s, L = 65521, 16, 15
    A = gen.wiedemann_matrix(seed=17, n=4000)
    M = lib.Matrix.from_csr(A)
    blocks = [(gen.uniform_block(20 + k, A.nrows, s, p), gen.uniform_block(30 + k, A.nrows, s, p, key=k))
              for k in range(3)]
    S = torch.empty((L, s, s), dtype=torch.int32, device="cuda")
    dev = [(to_dev(X), to_dev(Y)) for X, Y in blocks]   # all alive: distinct addresses
    for k in (0, 1, 2, 0):
        X, Y = blocks[k]
        lib.spmv_block_sequence(M.handle, dev[k][0], dev[k][1], s, 0, L, S, None)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(S).reshape(L, s, s), oracle.csr_block_sequence(A, X, Y, L)), k
    # and a resume on the same handle whose state buffer is the previous Y
    X, Y = blocks[1]
    S1, V = M.block_sequence(to_dev(X), to_dev(Y), 7, want_next=True)
    S2 = M.block_sequence(to_dev(X), V, 8)
    torch.cuda.synchronize()
    assert np.array_equal(np.concatenate([to_host(S1), to_host(S2)]).reshape(15, s, s),
                          oracle.csr_block_sequence(A, X, Y, 15))


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
    # 100k x 100k, s = 16, the benchmark's 12 502 steps.  The oracle checks
    # the first 24 steps whole, one (a, b) entry over every step, and every
    # entry of every step through random fingerprints: for u, w uniform in
    # (Z/pZ)^s, u^T S_i w = (X u)^T A^i (Y w) mod p is the scalar sequence of
    # the projected blocks X u and Y w, which the oracle computes with one
    # column each.  A wrong block E != 0 has u^T E w = 0 with probability at
    # most 2/p for one (u, w) (a nonzero bilinear form of degree 2), so two
    # fingerprints miss a wrong S_i with probability below 1e-9.
    from concurrent.futures import ThreadPoolExecutor
    p, s = 65521, 16
    A = gen.wiedemann_matrix(seed=1003)
    n = A.nrows
    L = 2 * n // s + 2
    X = gen.uniform_block(1003, n, s, p)
    Y = gen.uniform_block(1003, n, s, p, key=1)
    S = run(lib, A, X, Y, L)
    assert S.shape == (L, s, s)
    rng = np.random.default_rng(77)
    fps = [(rng.integers(0, p, s, dtype=np.uint64), rng.integers(0, p, s, dtype=np.uint64))
           for _ in range(2)]
    a, b = 5, 11
    jobs = [(X, Y, 24), (X[:, a:a + 1], Y[:, b:b + 1], L)]
    for u, w in fps:
        # inputs below 2^16, so these u64 sums of 16 products are exact
        xu = ((X.astype(np.uint64) @ u) % p).astype(np.uint32).reshape(n, 1)
        yw = ((Y.astype(np.uint64) @ w) % p).astype(np.uint32).reshape(n, 1)
        jobs.append((xu, yw, L))
    with ThreadPoolExecutor(len(jobs)) as ex:       # the oracle releases the GIL
        res = list(ex.map(lambda j: oracle.csr_block_sequence(A, *j), jobs))
    assert np.array_equal(S[:24], res[0])
    assert np.array_equal(S[:, a, b], res[1].reshape(L))
    S64 = S.astype(np.uint64)
    for (u, w), want in zip(fps, res[2:]):
        # u^T S_i w: terms below 2^48, 256 of them, exact in u64
        got = ((S64 * u[None, :, None]) % p * w[None, None, :]).sum(axis=(1, 2)) % p
        assert np.array_equal(got.astype(np.uint32), want.reshape(L))
