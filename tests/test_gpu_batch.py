"""GPU parity of the batched product Y_j = A_j X_j mod p_j (one launch over
uneven matrices with their own moduli) against the CPU oracle."""
import numpy as np
import pytest

import gen
import oracle
from helpers import rand_block, to_dev, to_host

pytestmark = pytest.mark.gpu


def run_batch(ff, probs, seed=0):
    mats = [ff.Matrix.from_csr(A, transpose_mode=ff.TRANSPOSE.NONE) for A, _ in probs]
    xs = [rand_block(seed + j, A.ncols, s, A.modulus) for j, (A, s) in enumerate(probs)]
    xd = [to_dev(x) for x in xs]
    import torch
    yd = [torch.empty((A.nrows, s) if s > 1 else (A.nrows,), dtype=torch.int32, device="cuda")
          for A, s in probs]
    ff.spmv_batch_apply([M.handle for M in mats], xd, yd, [s for _, s in probs])
    return mats, xs, [to_host(y) for y in yd]


def test_small_batch(lib):
    probs = gen.batch_problems(seed=77, count=40, rows_lo=50, rows_hi=3000)
    mats, xs, ys = run_batch(lib, probs, seed=3)
    for (A, s), x, y in zip(probs, xs, ys):
        assert np.array_equal(y, oracle.csr_spmv(A, x)), A.name


def test_batch_repeat_and_changed_pointers(lib):
    probs = gen.batch_problems(seed=78, count=12, rows_lo=100, rows_hi=2000)
    run_batch(lib, probs, seed=1)
    mats, xs, ys = run_batch(lib, probs, seed=9)
    for (A, s), x, y in zip(probs, xs, ys):
        assert np.array_equal(y, oracle.csr_spmv(A, x))


def test_full_batch_sampled(lib):
    # 256 problems, rows log-uniform in [1k, 200k]; every output checked for
    # a sample of 24 problems, plus the whole of the smallest and largest
    probs = gen.batch_problems(seed=1004)
    mats, xs, ys = run_batch(lib, probs, seed=5)
    rng = np.random.default_rng(0)
    pick = set(rng.choice(len(probs), 24, replace=False).tolist())
    sizes = [A.nrows for A, _ in probs]
    pick |= {int(np.argmin(sizes)), int(np.argmax(sizes))}
    for j in sorted(pick):
        A, s = probs[j]
        assert np.array_equal(ys[j], oracle.csr_spmv(A, xs[j])), A.name


def test_batch_widths_moduli_long_rows_and_offsets(lib):
    # block widths 1..32 (one, two or four components per lane), moduli on both
    # sides of 2^31 (64-bit partial sums of four products, or none), rows long
    # enough to get a whole CTA, and x starting 4 bytes past a 16-byte boundary
    import torch
    probs = []
    for j, (s, m) in enumerate([(1, 65521), (2, 2**31 - 1), (3, 2**31), (4, 4294967291), (8, 1000003),
                                (12, 4294967291), (16, 2**31 - 1), (32, 3), (6, 2147483659)]):
        n = 300 + 37 * j
        lengths = np.full(n, 7)
        lengths[5] = 2500          # long row
        lengths[9] = 0             # empty row
        probs.append((gen.uniform_matrix(100 + j, n, 4000, lengths, m), s))
    mats = [lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.NONE) for A, _ in probs]
    xs = [rand_block(200 + j, A.ncols, s, A.modulus) for j, (A, s) in enumerate(probs)]
    xd = []
    for (A, s), x in zip(probs, xs):
        if s % 2 == 0:
            buf = torch.empty(A.ncols * s + 1, dtype=torch.int32, device="cuda")
            v = buf[1:].view(A.ncols, s)             # misaligned for vector loads
            v.copy_(torch.from_numpy(x.view(np.int32).reshape(A.ncols, s)))
            xd.append(v)
        else:
            xd.append(to_dev(x))
    yd = [torch.empty((A.nrows, s) if s > 1 else (A.nrows,), dtype=torch.int32, device="cuda")
          for A, s in probs]
    lib.spmv_batch_apply([M.handle for M in mats], xd, yd, [s for _, s in probs])
    for (A, s), x, y in zip(probs, xs, yd):
        assert np.array_equal(to_host(y), oracle.csr_spmv(A, x)), (A.name, s, A.modulus)
    # the same with aligned x
    xd = [to_dev(x) for x in xs]
    lib.spmv_batch_apply([M.handle for M in mats], xd, yd, [s for _, s in probs])
    for (A, s), x, y in zip(probs, xs, yd):
        assert np.array_equal(to_host(y), oracle.csr_spmv(A, x)), (A.name, s, A.modulus)
