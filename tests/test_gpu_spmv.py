"""GPU parity of y = alpha*A*x + beta*y and of the transpose product (Sec. 2)
against the CPU oracle, element by element and bit-exact, for every storage
format, several moduli, block widths and edge cases."""
import numpy as np
import pytest

import gen
import oracle
from helpers import rand_block, to_dev, to_host, with_modulus

pytestmark = pytest.mark.gpu

FORMATS = ["CSR", "ELLR", "COO", "COOS", "DIA", "HYBRID", "BINNED", "PANEL"]
MODULI = [2, 3, 27, 65521, 2**31 - 1, 4294967291]


def make(ff, A, fmt, **kw):
    return ff.Matrix.from_csr(A, priority_format=getattr(ff.FMT, fmt), **kw)


def check_apply(ff, M, A, nvec=1, alpha=1, beta=0, seed=0, transpose=False):
    m = A.modulus
    in_rows, out_rows = (A.nrows, A.ncols) if transpose else (A.ncols, A.nrows)
    x = rand_block(seed, in_rows, nvec, m)
    y0 = rand_block(seed + 1, out_rows, nvec, m)
    yd = to_dev(y0)
    if transpose:
        M.apply_transpose(to_dev(x), yd, alpha=alpha, beta=beta)
        want = oracle.csr_spmv_transpose(A, x, y=y0, alpha=alpha, beta=beta)
    else:
        M.apply(to_dev(x), yd, alpha=alpha, beta=beta)
        want = oracle.csr_spmv(A, x, y=y0, alpha=alpha, beta=beta)
    M.check_status()  # no bounded device wait ran out
    got = to_host(yd)
    assert got.shape == want.shape
    bad = np.nonzero(got != want)
    assert bad[0].size == 0, f"{bad[0].size} mismatches, first at {bad[0][:5]}"


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("m", MODULI)
def test_tiny_all_formats(lib, fmt, m):
    A = gen.tiny_matrix() if m == 65521 else with_modulus(gen.tiny_matrix(), m)
    M = make(lib, A, fmt)
    for transpose in (False, True):
        check_apply(lib, M, A, transpose=transpose, seed=3)
        check_apply(lib, M, A, alpha=7 % m, beta=(m - 3) % m, transpose=transpose, seed=5)


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("nvec", [2, 3, 4, 16, 19, 32])
def test_block_vectors(lib, fmt, nvec):
    for m in (65521, 2**31 - 1):
        A = with_modulus(gen.tiny_matrix(n=700, per_row=9), m, seed=nvec)
        M = make(lib, A, fmt)
        check_apply(lib, M, A, nvec=nvec, alpha=3, beta=2, seed=nvec)
        check_apply(lib, M, A, nvec=nvec, transpose=True, seed=nvec + 1)


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("use_pm1", [0, 1])
def test_powerlaw_medium(lib, fmt, use_pm1):
    # Zipf rows (mean 16, max 3000) with a ragged tail; several tiles per bin
    for m, pm in ((65521, 0.3), (2**31 - 1, 0.0), (3, 0.0)):
        A = gen.powerlaw_matrix(seed=7, n=30_011, lmax=3000, m=m, pm_fraction=pm)
        if fmt == "DIA":
            # ~60k occupied diagonals x 30k rows: refused by the size guard
            with pytest.raises(lib.FFSPMVError) as e:
                make(lib, A, fmt, use_pm1=use_pm1, guard_bytes=1 << 30)
            assert e.value.status == 5
            continue
        M = make(lib, A, fmt, use_pm1=use_pm1, guard_bytes=1 << 30)
        check_apply(lib, M, A, seed=11)
        check_apply(lib, M, A, transpose=True, alpha=5, beta=1, seed=12)


@pytest.mark.parametrize("fmt", ["DIA", "HYBRID", "BINNED", "ELLR"])
def test_banded_and_block_diagonal(lib, fmt):
    for A in (gen.banded_matrix(4, 20_000, np.full(20_000, 12), 65521, pm_fraction=0.5),
              gen.block_diagonal_matrix(5, 9_000, 300, np.full(9_000, 30), 2**31 - 1)):
        M = make(lib, A, fmt, guard_bytes=1 << 30)
        check_apply(lib, M, A, seed=1)
        check_apply(lib, M, A, transpose=True, alpha=2, beta=3, seed=2)
        check_apply(lib, M, A, nvec=4, seed=3)


def test_split_long_rows(lib):
    # rows far longer than one CTA chunk, in every plan that splits them
    lengths = np.array([30_000, 1, 9000, 0, 4097, 4096, 4095, 70_000, 2], dtype=np.int64)
    A = gen.uniform_matrix(3, lengths.size, 100_000, lengths, 2**31 - 1, pm_fraction=0.3)
    for fmt in ("HYBRID", "BINNED", "COO", "CSR", "PANEL"):
        for pm in (0, 1):
            M = make(lib, A, fmt, use_pm1=pm)
            check_apply(lib, M, A, alpha=3, beta=4, seed=pm)
            check_apply(lib, M, A, nvec=3, seed=pm + 2)


@pytest.mark.parametrize("m,q", [(65521, 0), (65521, 1), (65521, 2), (65521, 4),
                                 (2**31 - 1, 0), (2**31 - 1, 1), (2**31 - 1, 2)])
def test_panel_column_groups(lib, m, q):
    # clusters of 1, 2 or 4 CTAs splitting the columns (0: the builder's
    # choice; with 8-byte row sums four column groups leave no room); the
    # transpose has the power-law skew on its columns instead of its rows
    A = gen.powerlaw_matrix(seed=8, n=150_001, lmax=20_000, m=m, pm_fraction=0.2)
    M = make(lib, A, "PANEL", panel_cluster=q)
    if q:
        assert f"x {q} column groups" in M.describe()
    for rep in range(2):  # the group counters carry over between calls
        check_apply(lib, M, A, alpha=7, beta=5, seed=31 + rep)
    check_apply(lib, M, A, transpose=True, seed=32)
    check_apply(lib, M, A, nvec=2, seed=33)
    M.check_status()  # no bounded wait ran out


def test_panel_packs_in_both_sections(lib):
    # rows with eight general and eight +-1 entries in one stage: a general
    # pack and a +-1 pack of one row in the same warp, single lanes between
    rng = np.random.default_rng(9)
    n, m = 300, 65521
    cols, vals, rp = [], [], [0]
    for i in range(n):
        k = 16 if i % 7 == 0 else int(rng.integers(1, 12))
        c = np.sort(rng.choice(n, k, replace=False))
        v = rng.integers(2, m - 1, k)
        if i % 7 == 0:
            v[::2] = np.where(rng.random(8) < 0.5, 1, m - 1)
        cols.append(c); vals.append(v); rp.append(rp[-1] + k)
    A = gen.CSR(n, n, np.array(rp, np.int64), np.concatenate(cols).astype(np.int32),
                np.concatenate(vals).astype(np.uint32), m)
    M = make(lib, A, "PANEL", use_pm1=1)
    check_apply(lib, M, A, seed=41)
    check_apply(lib, M, A, alpha=3, beta=5, transpose=True, seed=42)


def test_panel_timeout_hook_sets_status_and_handle_survives(lib):
    # the copies of each CTA's second stage are never issued: the bounded
    # waits for them run out, the kernel ends, and the status word says so
    A = gen.powerlaw_matrix(seed=8, n=150_001, lmax=20_000, m=65521)
    M = make(lib, A, "PANEL", test_hooks=2, transpose_mode=lib.TRANSPOSE.NONE)
    x = rand_block(1, A.ncols, 1, A.modulus)
    yd = to_dev(np.zeros(A.nrows, dtype=np.uint32))
    M.apply(to_dev(x), yd)
    with pytest.raises(lib.FFSPMVError) as e:
        M.check_status()
    assert e.value.status == 6
    M.check_status()  # read and cleared
    # the device and the library stay usable
    N = make(lib, A, "PANEL", transpose_mode=lib.TRANSPOSE.NONE)
    check_apply(lib, N, A, seed=4)


@pytest.mark.parametrize("m,pm", [(65521, 0.3), (3, 1.0), (2**31 - 1, 0.2)])
def test_panel_multi_vector_passes(lib, m, pm):
    """Blocks on an x-panel handle run in passes of 4 (m <= 2^16) or 2
    vectors, each reading the matrix once on a layout built for its width.
    Widths 2 to 16 cover contiguous blocks (ldx = pass width), strided ones
    (vector loads and scalar loads of x), and remainders of 2 and 1."""
    A = gen.powerlaw_matrix(seed=17, n=60_007, lmax=4000, m=m, pm_fraction=pm)
    # test hook 4: the wide passes are taken whether or not they are faster
    M = make(lib, A, "PANEL", use_pm1=1 if pm else 0, test_hooks=4)
    for nvec in (2, 3, 4, 6, 7, 16):
        check_apply(lib, M, A, nvec=nvec, alpha=5 % m, beta=(m - 2) % m, seed=nvec)
        check_apply(lib, M, A, nvec=nvec, transpose=True, seed=nvec + 50)
    width = 4 if m <= 65536 else 2
    assert M.launches(False, 16) == 16 // width     # one launch per pass


@pytest.mark.parametrize("m", [65521, 2**31 - 1])
def test_panel_one_vector_passes_stage_groups(lib, m):
    """One-vector passes over a block (test hook 8): the first launch of each
    group of four vectors stages all of them (vector loads when ldx is a
    multiple of four, scalar loads otherwise), the others read the staged
    copies; groups of 4, 3, 2 and 1 and the staging launch of plans whose
    row groups exceed the resident clusters."""
    A = gen.powerlaw_matrix(seed=19, n=50_021, lmax=3000, m=m, pm_fraction=0.2)
    M = make(lib, A, "PANEL", use_pm1=1, test_hooks=8)
    for nvec in (2, 3, 4, 5, 7, 16):
        check_apply(lib, M, A, nvec=nvec, alpha=3, beta=5, seed=40 + nvec)
        check_apply(lib, M, A, nvec=nvec, transpose=True, seed=60 + nvec)
    assert M.launches(False, 7) == 7
    n = 1_200_000
    B = gen.uniform_matrix(9, n, 200_000, np.full(n, 3), m, pm_fraction=0.2)
    q = 4 if m > 65536 else 2
    MB = make(lib, B, "PANEL", panel_cluster=q, transpose_mode=lib.TRANSPOSE.NONE, test_hooks=8)
    check_apply(lib, MB, B, nvec=6, seed=77)


@pytest.mark.parametrize("m", [2, 3, 251, 256])
def test_panel_u8_moduli(lib, m):
    """m <= 256: the x-panel layout stages x and stores values as u8 and adds
    the products v x < 2^16 unreduced; products, transposes, blocks (one
    staging launch per four vectors) and the longest panel rows at the worst
    values, against the oracle."""
    A = gen.powerlaw_matrix(seed=23, n=40_009, lmax=3000, m=m, pm_fraction=0.3)
    for pm in (0, 1):
        M = make(lib, A, "PANEL", use_pm1=pm)
        assert "x staged as u8" in M.describe()
        check_apply(lib, M, A, alpha=1 % m, beta=(m - 1) % m, seed=3 + pm)
        check_apply(lib, M, A, transpose=True, seed=5 + pm)
        check_apply(lib, M, A, nvec=5, seed=7 + pm)
    lengths = np.array([32_768, 32_769, 17, 0, 1])
    nc = 70_000
    col = np.concatenate([np.arange(L) * 2 for L in lengths]).astype(np.int32)
    W = gen.CSR(lengths.size, nc, np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64), col,
                np.full(lengths.sum(), m - 1, dtype=np.uint32), m)
    MW = make(lib, W, "PANEL", use_pm1=0, transpose_mode=lib.TRANSPOSE.NONE)
    y = to_host(MW.apply(to_dev(np.full(nc, m - 1, dtype=np.uint32))))
    assert list(y) == [int(L) * (m - 1) * (m - 1) % m for L in lengths]


@pytest.mark.parametrize("m,q", [(2**31 - 1, 1), (2**31 - 1, 2), (4294967291, 2), (65537, 4), (2**20, 2)])
def test_panel_wide_sums_at_worst_values(lib, m, q):
    """m > 2^16: every value and every x at m - 1, long rows split over the
    column groups of a cluster (the CTAs' partial sums, pairs of u32 sums,
    meet in the cluster epilogue); the results equal the closed form
    L (m-1)^2 mod m.  Odd m < 2^31 takes Montgomery terms, 2^20 (even) and
    4294967291 (above 2^31) the 64-bit Barrett reduction."""
    lengths = np.array([32_768, 20_000, 4097, 17, 1, 0, 3000])
    nc = 120_000
    rng = np.random.default_rng(q)
    col = np.concatenate([np.sort(rng.choice(nc, L, replace=False)) for L in lengths]).astype(np.int32)
    A = gen.CSR(lengths.size, nc, np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64), col,
                np.full(lengths.sum(), m - 1, dtype=np.uint32), m)
    M = make(lib, A, "PANEL", panel_cluster=q, use_pm1=0, transpose_mode=lib.TRANSPOSE.NONE)
    assert "panels:" in M.describe()
    y = to_host(M.apply(to_dev(np.full(nc, m - 1, dtype=np.uint32))))
    assert list(y) == [int(L) * (m - 1) * (m - 1) % m for L in lengths]
    check_apply(lib, M, A, alpha=m - 2, beta=m - 3, seed=q)


@pytest.mark.parametrize("m,q,nvec", [(4294967291, 1, 1), (4294967291, 2, 2), (2**31 - 1, 2, 1), (2**31 - 1, 1, 2)])
def test_panel_split_row_sums_at_their_limit(lib, m, q, nvec):
    """m > 2^16 keeps each row sum as two u32 sums, of the terms' low 16
    bits and of the rest.  Rows of 32 768 entries (the most a row in the
    panels has) with the largest terms the reduction gives: at 4294967291
    every value m - 1 against x = 1, each term m - 1 = 2^32 - 6, so both
    halves of the sum approach 2^31; at 2^31 - 1 (Montgomery terms below 2m)
    values and x uniform.  Results against the closed form and the oracle,
    for one- and two-vector passes."""
    lengths = np.array([32_768, 32_768, 30_000, 1, 0, 32_767])
    nc = 140_000
    rng = np.random.default_rng(m % 1000 + q)
    col = np.concatenate([np.sort(rng.choice(nc, L, replace=False)) for L in lengths]).astype(np.int32)
    nnz = int(lengths.sum())
    vals = (np.full(nnz, m - 1, dtype=np.uint32) if m > 2**31
            else rng.integers(1, m, nnz, dtype=np.uint64).astype(np.uint32))
    A = gen.CSR(lengths.size, nc, np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64), col, vals, m)
    hooks = 4 if nvec > 1 else 0   # test hook 4: keep the 2-vector layout
    M = make(lib, A, "PANEL", panel_cluster=q, use_pm1=0, transpose_mode=lib.TRANSPOSE.NONE, test_hooks=hooks)
    assert "panels:" in M.describe()
    if m > 2**31:
        X = np.ones((nc, nvec), dtype=np.uint32)
        Y = to_host(M.apply(to_dev(X if nvec > 1 else X[:, 0]))).reshape(lengths.size, nvec)
        for k in range(nvec):
            assert list(Y[:, k]) == [int(L) * (m - 1) % m for L in lengths]
    check_apply(lib, M, A, nvec=nvec, alpha=m - 2, beta=m - 3, seed=q + nvec)


def test_panel_wide_passes_kept_only_when_faster(lib):
    """Without the test hook a block on the 1M power-law matrix (few entries
    per column of a CTA) keeps one-vector passes if the timed 2-vector pass
    is not faster; either way the products are exact."""
    A = gen.powerlaw_matrix(seed=1002, m=65521)
    M = make(lib, A, "PANEL", transpose_mode=lib.TRANSPOSE.NONE)
    n = M.launches(False, 2)
    assert n in (1, 2)
    x = rand_block(5, A.ncols, 2, A.modulus)
    got = to_host(M.apply(to_dev(x)))
    rows = np.random.default_rng(5).integers(0, A.nrows, 2000)
    for r in rows:
        a, b = A.row_ptr[r], A.row_ptr[r + 1]
        want = (A.val[a:b].astype(object) @ x[A.col[a:b]].astype(object)) % A.modulus
        assert list(got[r]) == [int(w) for w in want], r


def test_panel_staging_launch_when_groups_exceed_resident(lib):
    """Row groups beyond the resident clusters: x is staged by a launch of
    its own before the panel kernel (two launches per pass), for one vector
    (32-bit residues, clusters of 4) and for passes of 4 vectors (16-bit
    residues, whose row sums take 4x the shared memory per row)."""
    n = 1_200_000
    for m, q, nvec in ((2**31 - 1, 4, 1), (65521, 2, 4)):
        A = gen.uniform_matrix(9, n, 200_000, np.full(n, 3), m, pm_fraction=0.2)
        M = make(lib, A, "PANEL", panel_cluster=q, transpose_mode=lib.TRANSPOSE.NONE, test_hooks=4)
        assert M.launches(False, nvec) == 2, M.describe()
        check_apply(lib, M, A, nvec=nvec, alpha=3, beta=7, seed=q)


@pytest.mark.parametrize("use_pm1", [0, 1])
def test_panel_longest_rows_worst_values(lib, use_pm1):
    # m <= 2^16: general terms are reduced only below 2m, and a -1 entry's
    # term is m - x <= m, so a row sum of 32 768 terms is the most a 32-bit
    # shared-memory sum holds; longer rows leave the panels.  Every value is
    # m - 1: with +-1 sections off these are the largest general terms (x =
    # m - 1), with them on the largest -1 terms (x = 0).
    m = 65521
    lengths = np.array([32_768, 32_769, 40_000, 5, 0, 1])
    n, nc = lengths.size, 100_000
    col = np.concatenate([np.arange(L) * 2 for L in lengths]).astype(np.int32)
    A = gen.CSR(n, nc, np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64), col,
                np.full(lengths.sum(), m - 1, dtype=np.uint32), m)
    M = make(lib, A, "PANEL", transpose_mode=lib.TRANSPOSE.NONE, use_pm1=use_pm1, test_hooks=4)
    assert "panels:" in M.describe()
    xv = 0 if use_pm1 else m - 1
    x = np.full(nc, xv, dtype=np.uint32)
    y = to_host(M.apply(to_dev(x)))
    assert list(y) == [int(L) * (m - 1) * xv % m for L in lengths]
    check_apply(lib, M, A, alpha=2, beta=3, seed=6)
    # passes of 2 and 4 vectors keep two u32 sums side by side in a u64:
    # the same limit, with no carry from one into the other
    for nvec in (2, 4):
        X = np.full((nc, nvec), xv, dtype=np.uint32)
        Y = to_host(M.apply(to_dev(X)))
        assert all(list(Y[:, k]) == [int(L) * (m - 1) * xv % m for L in lengths] for k in range(nvec))
        check_apply(lib, M, A, nvec=nvec, alpha=2, beta=3, seed=7)


def test_rectangular_and_empty_rows(lib):
    A = gen.random_small(3, 517, 1283, 0.01, 65521, pm_fraction=0.4, dup=True)
    for fmt in FORMATS:
        M = make(lib, A, fmt)
        check_apply(lib, M, A, seed=1)
        check_apply(lib, M, A, transpose=True, seed=2)
        check_apply(lib, M, A, nvec=5, alpha=9, beta=4, seed=3)


def test_long_rows_wide_accumulator(lib):
    # rows of (m-1) entries against x = m-1 overflow 64 bits for m ~ 2^32
    m = 4294967291
    lengths = np.array([0, 1, 5, 4000, 10_000, 3, 0, 77])
    n = lengths.size
    col = np.concatenate([np.arange(L) for L in lengths]).astype(np.int32)
    A = gen.CSR(n, 10_000, np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64), col,
                np.full(lengths.sum(), m - 1, dtype=np.uint32), m)
    for fmt in FORMATS:
        M = make(lib, A, fmt, guard_bytes=1 << 30)
        x = np.full(10_000, m - 1, dtype=np.uint32)
        y = to_host(M.apply(to_dev(x)))
        assert list(y) == [int(L) % m for L in lengths]
        check_apply(lib, M, A, seed=4)
        check_apply(lib, M, A, transpose=True, seed=5)


def test_empty_matrix(lib):
    m = 65521
    Z = gen.CSR(6, 4, np.zeros(7, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint32), m)
    for fmt in FORMATS:
        M = make(lib, Z, fmt)
        check_apply(lib, M, Z, alpha=2, beta=3, seed=1)
        check_apply(lib, M, Z, transpose=True, alpha=2, beta=5, seed=2)


def test_atomic_transpose(lib):
    A = gen.powerlaw_matrix(seed=9, n=20_000, lmax=2000, m=2**31 - 1)
    M = lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.ATOMIC)
    for nvec in (1, 4, 17):
        check_apply(lib, M, A, nvec=nvec, transpose=True, alpha=3, beta=7, seed=nvec)
        check_apply(lib, M, A, nvec=nvec, transpose=True, seed=nvec + 50)


def test_value_check_and_errors(lib):
    import torch
    A = gen.tiny_matrix(n=100, per_row=4)
    M = lib.Matrix.from_csr(A, value_check=1)
    x = np.full(100, 70000, dtype=np.uint32)            # >= m
    with pytest.raises(lib.FFSPMVError) as e:
        M.apply(to_dev(x))
    assert e.value.status == 2
    check_apply(lib, M, A, seed=3)                      # handle still usable
    with pytest.raises(lib.FFSPMVError):
        lib.Matrix(2, 2, [0, 1, 2], [0, 5], [1, 1], 7)  # column out of range
    with pytest.raises(lib.FFSPMVError):
        lib.Matrix(2, 2, [0, 1, 2], [0, 1], [1, 1], 1)  # modulus < 2
    N = lib.Matrix.from_csr(A, transpose_mode=lib.TRANSPOSE.NONE)
    with pytest.raises(lib.FFSPMVError) as e:
        N.apply_transpose(to_dev(np.zeros(100, np.uint32)))
    assert e.value.status == 5
    y = torch.empty(100, dtype=torch.int32, device="cuda")
    with pytest.raises(lib.FFSPMVError):
        lib.spmv_apply(M.handle, to_dev(np.zeros(100, np.uint32)), 0, y, 1, 1)   # ldx < nvec


def test_device_input_csr(lib):
    import torch
    A = gen.tiny_matrix(n=500, per_row=7)
    M = lib.Matrix(A.nrows, A.ncols, torch.from_numpy(A.row_ptr).cuda(),
                   torch.from_numpy(A.col).cuda(), to_dev(A.val), A.modulus)
    check_apply(lib, M, A, seed=8)


def test_describe_and_info(lib):
    A = gen.powerlaw_matrix(seed=2, n=20_000, lmax=500)
    M = make(lib, A, "HYBRID")
    d = M.describe()
    assert "HYBRID" in d and "ELL_R" in d
    info = M.info()
    assert info["nnz"] == A.nnz and info["modulus"] == A.modulus


@pytest.mark.parametrize("m", [65521, 2**31 - 1, 3])
def test_full_size_powerlaw(lib, m):
    # 1M x 1M Zipf (mean 16, max 10k): the benchmark's matrix, checked whole
    A = gen.powerlaw_matrix(seed=1002, m=m)
    for fmt in ("HYBRID", "BINNED", "CSR", "PANEL"):
        M = make(lib, A, fmt)
        check_apply(lib, M, A, seed=21)
        check_apply(lib, M, A, transpose=True, seed=22)
        del M
