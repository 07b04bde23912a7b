"""GPU parity of the sigma-basis (PM-Basis over polynomial-matrix products,
M-Basis leaves) against oracle/sigma.py, bit for bit with the same leaf
order: several leaves, a shift, p = 2^31 - 1, sparse rank-deficient input,
the full width of 32 rows, one leaf at the largest order; the block-Wiedemann
pipeline (GPU sequence, [S; -I], sigma-basis) on a matrix of known rank; and
at the size of the 100k Wiedemann workload (s = 16, 12 502 terms) the
properties that hold at any size."""
import time

import numpy as np
import pytest

import gen
import oracle
from oracle import linalg, sigma

pytestmark = pytest.mark.gpu


def _full(P, d):
    m = P.shape[1]
    out = np.zeros((d + 1, m, m), dtype=np.int64)
    out[:P.shape[0]] = np.asarray(P, dtype=np.int64)
    return out


def _gpu(lib, p, F, shift=None, base=0):
    P, delta, e = lib.sigma_basis(p, np.ascontiguousarray(F, dtype=np.uint32), shift=shift, base=base)
    return P.cpu().numpy().view(np.uint32).astype(np.int64), delta, e


@pytest.mark.parametrize("p,m,n,d,base,shift,density", [
    (65521, 2, 1, 14, 4, None, 1.0),                  # the scalar case, several leaves
    (65521, 8, 4, 50, 8, None, 1.0),
    (2**31 - 1, 6, 3, 37, 16, [2, 0, 1, 0, 3, 0], 1.0),
    (7, 8, 4, 30, 4, None, 0.3),                      # sparse, one zero column: orders without pivots
    (65521, 6, 6, 20, 4, None, 1.0),                  # n = m
    (65521, 5, 3, 23, 3, [1, 0, 0, 2, 0], 1.0),       # odd m, n and leaf orders
    (65521, 32, 16, 20, 8, None, 1.0),                # the width of s = 16 block Wiedemann
    (65521, 32, 16, 32, 32, None, 1.0),               # one leaf of the largest order
    (1000003, 32, 32, 18, 16, None, 1.0),             # square
    (1000003, 32, 32, 40, 32, None, 1.0),             # square, order-32 leaves over a cluster of 8 CTAs
    (65521, 3, 1, 9, 0, [0, 4, 1], 1.0),              # four columns: a cluster of four CTAs
])
def test_parity_with_oracle(lib, p, m, n, d, base, shift, density):
    rng = np.random.default_rng(d * 131 + m)
    F = rng.integers(0, p, (d, m, n))
    if density < 1.0:
        F = F * (rng.random((d, m, n)) < density)
        F[:, :, 1] = 0
    P, delta, e = _gpu(lib, p, F, shift, base)
    Po, do = sigma.pmbasis(F.astype(object), d, shift or [0] * m, p, base=base or 16)
    assert delta == do
    assert np.array_equal(P, _full(Po, d))
    assert Po.shape[0] - 1 <= e <= d
    assert not np.any(P[e + 1:])


def test_default_base_matches_oracle_leaf_order(lib):
    # m = 8, n = 4: the default leaf order is 32, so d = 40 splits once
    p, m, n, d = 65521, 8, 4, 40
    F = np.random.default_rng(3).integers(0, p, (d, m, n))
    P, delta, _ = _gpu(lib, p, F)
    Po, do = sigma.pmbasis(F.astype(object), d, [0] * m, p, base=32)
    assert delta == do and np.array_equal(P, _full(Po, d))


def _block_diagonal(seed, nb, zero_blocks, p):
    """2 x 2 blocks, invertible except the last `zero_blocks` (all zero):
    rank 2 (nb - zero_blocks), and 0 is a semisimple eigenvalue."""
    rng = np.random.default_rng(seed)
    dense = np.zeros((2 * nb, 2 * nb), dtype=np.int64)
    for b in range(nb - zero_blocks):
        while True:
            B = rng.integers(0, p, (2, 2))
            if (int(B[0, 0]) * int(B[1, 1]) - int(B[0, 1]) * int(B[1, 0])) % p:
                break
        dense[2 * b:2 * b + 2, 2 * b:2 * b + 2] = B
    return dense


def test_block_wiedemann_pipeline_rank(lib):
    # GPU sequence -> [S; -I] -> GPU sigma-basis; the generator's
    # deg det - codeg det equals the rank from Gaussian elimination
    p, s, nb, z = 65521, 4, 30, 3
    dense = _block_diagonal(9, nb, z, p)
    n = dense.shape[0]
    A = gen.dense_to_csr(dense, p)
    assert linalg.rank_mod_p(dense.tolist(), p) == n - 2 * z
    X = gen.uniform_block(21, n, s, p)
    Y = gen.uniform_block(22, n, s, p, key=1)
    L = 2 * n // s + 4
    M = lib.Matrix.from_csr(A)
    import torch
    S = M.block_sequence(torch.from_numpy(X.view(np.int32)).cuda(), torch.from_numpy(Y.view(np.int32)).cuda(), L)
    assert np.array_equal(lib.to_numpy_u32(S), oracle.csr_block_sequence(A, X, Y, L))
    F = lib.sigma_wiedemann_input(p, S)
    Fh = F.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(Fh[:, :s], lib.to_numpy_u32(S).astype(np.int64))
    assert np.array_equal(Fh[0, s:], (p - 1) * np.eye(s, dtype=np.int64))
    assert not np.any(Fh[1:, s:])
    P, delta, _ = _gpu(lib, p, Fh, base=8)
    Po, do = sigma.pmbasis(Fh.astype(object), L, [0] * (2 * s), p, base=8)
    assert delta == do and np.array_equal(P, _full(Po, L))
    rows = sorted(range(2 * s), key=lambda i: (delta[i], i))[:s]
    U = sigma.trim(P[:, rows, :s].astype(object))
    dg, cdg = sigma.degree_and_codegree(sigma.det_poly(U, p))
    assert dg - cdg == n - 2 * z
    # the library's own deg det and codeg det of the GPU generator
    assert lib.sigma_generator_degrees(p, P.astype(np.uint32), delta, s) == (dg, cdg)


def _coeff_np(P, F, k, e):
    """coefficient k of P F (int64 sums: entries below 2^16, at most 2^18 terms)."""
    lo, hi = max(0, k - F.shape[0] + 1), min(k, e)
    t = np.arange(lo, hi + 1)
    return np.einsum("tij,tjl->il", P[t], F[k - t])


def _det_mod(Mx, p):
    return sigma._det_mod(Mx.astype(object), p)


def test_wiedemann_100k_generator(lib):
    # diag(d_1..d_N) with every nonzero residue once or twice: rank N, and no
    # eigenvalue repeats more than s times, so the first s invariant factors
    # of xI - A multiply to its characteristic polynomial.  S from the GPU
    # sequence, L = 2N/s + 2 terms; the generator (the s rows of least
    # degree) has det of degree N (its leading row coefficients are
    # nonsingular, so deg det = the sum of its row degrees) and codegree 0
    # (U(0) nonsingular)
    import torch
    p, s, N = 65521, 16, 100_000
    rng = np.random.default_rng(100)
    once = np.arange(1, p, dtype=np.int64)
    dvals = rng.permutation(np.concatenate([once, rng.choice(once, N - (p - 1), replace=False)]))
    dvals = dvals.astype(np.uint32)
    A = gen.synth.CSR(N, N, np.arange(N + 1, dtype=np.int64), np.arange(N, dtype=np.int32), dvals, p, "diag")
    L = 2 * N // s + 2
    X = gen.uniform_block(31, N, s, p)
    Y = gen.uniform_block(32, N, s, p, key=1)
    M = lib.Matrix.from_csr(A)
    S = M.block_sequence(torch.from_numpy(X.view(np.int32)).cuda(), torch.from_numpy(Y.view(np.int32)).cuda(), L)
    F = lib.sigma_wiedemann_input(p, S)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Pd, delta, e = lib.sigma_basis(p, F)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    print(f"sigma-basis 32 x 16, order {L}, p = {p}: {secs * 1e3:.1f} ms, degree bound {e}")
    assert sum(delta) == s * L                      # det P = c x^(s L) for [S; -I]
    P = Pd[:e + 1].cpu().numpy().view(np.uint32).astype(np.int64)
    assert not np.any(Pd[e + 1:].cpu().numpy())
    Fh = F.cpu().numpy().view(np.uint32).astype(np.int64)
    for k in (0, 1, 2, 777, L // 2, L - 2, L - 1):   # P F = 0 mod x^L, sampled
        assert not np.any(_coeff_np(P, Fh, k, e) % p), k
    # every order through random fingerprints: u^T (P F)_k w = 0 for all k < L,
    # the coefficients of sum_j (u^T P)_j (F w)_j; a nonzero coefficient block
    # passes one fingerprint with probability at most 2/p
    for seed in (1, 2):
        fr = np.random.default_rng(seed)
        u = fr.integers(0, p, 2 * s, dtype=np.int64)
        w = fr.integers(0, p, s, dtype=np.int64)
        uP = np.einsum("i,kij->kj", u, P) % p       # (e+1) x 2s, sums below 2^42
        Fw = np.einsum("kjl,l->kj", Fh, w) % p      # L x 2s
        r = np.zeros(L, dtype=np.int64)
        for j in range(2 * s):                      # sums below 2^46 per j
            r = (r + np.convolve(uP[:, j], Fw[:, j])[:L]) % p
        assert not np.any(r), int(np.flatnonzero(r)[0])
    rows = sorted(range(2 * s), key=lambda i: (delta[i], i))[:s]
    assert sum(delta[i] for i in rows) == N
    lead = np.stack([P[delta[i], i, :s] for i in rows])
    assert _det_mod(lead, p) != 0                   # row reduced: deg det = N
    assert _det_mod(P[0][rows][:, :s], p) != 0      # codegree 0: rank N
    # the library reads the same rank off the device basis
    assert lib.sigma_generator_degrees(p, Pd, delta, s) == (N, 0)


def test_errors(lib):
    F = np.zeros((4, 2, 1), dtype=np.uint32)
    with pytest.raises(lib.FFSPMVError) as e:
        lib.sigma_basis(65520, F)                   # not a prime
    assert e.value.status == 1
    with pytest.raises(lib.FFSPMVError) as e:
        lib.sigma_basis(65521, np.zeros((4, 2, 3), dtype=np.uint32))   # n > m
    assert e.value.status == 1
