"""The row-partitioned block sequence (paper_1004_3719_gb300.dist_sequence):
rows of A, X and Y split over the ranks, an all-reduce of the partial
projections and an all-gather of V per step.  On CPU (gloo, 2 and 3 ranks)
the local arithmetic is the CPU oracle's; on a GPU (one rank, NCCL) it is the
library's kernels.  Both must give the single-process oracle's sequence."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rows(A, r0, r1):
    import gen
    a, b = int(A.row_ptr[r0]), int(A.row_ptr[r1])
    return gen.CSR(r1 - r0, A.ncols, (A.row_ptr[r0:r1 + 1] - a).astype(np.int64), A.col[a:b], A.val[a:b],
                   A.modulus)


def test_row_range_covers_all_rows_evenly():
    from paper_1004_3719_gb300.dist_sequence import row_range
    for n, world in ((10, 3), (7, 7), (5, 8), (100_000, 6), (0, 2)):
        rs = [row_range(n, world, r) for r in range(world)]
        assert rs[0][0] == 0 and rs[-1][1] == n
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
        sizes = [b - a for a, b in rs]
        assert max(sizes) - min(sizes) <= 1


def _oracle_compute(A_rows, X_rows, p):
    import torch

    import oracle
    from paper_1004_3719_gb300.dist_sequence import RowCompute

    def project(V_rows, Sacc):
        Sacc += torch.from_numpy(X_rows.astype(np.int64).T @ V_rows.numpy().view(np.uint32).astype(np.int64))

    def finish(Sacc):
        S = (Sacc % p).clone()
        Sacc.zero_()
        return S

    def apply(V_full):
        return torch.from_numpy(oracle.csr_spmv(A_rows, V_full.numpy().view(np.uint32)).view(np.int32))

    return RowCompute(project, finish, apply)


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import gen
    from paper_1004_3719_gb300.dist_sequence import block_sequence, row_range
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, s, L = 65521, 4, 9
    A = gen.wiedemann_matrix(seed=31, n=601, p=p, n_random=3)
    X = gen.uniform_block(32, A.nrows, s, p)
    Y = gen.uniform_block(33, A.nrows, s, p)
    r0, r1 = row_range(A.nrows, world, rank)
    comp = _oracle_compute(_rows(A, r0, r1), X[r0:r1], p)
    S = block_sequence(A.nrows, s, L, torch.from_numpy(np.ascontiguousarray(Y[r0:r1]).view(np.int32)), comp)
    q.put((rank, [t.numpy().astype(np.int64) for t in S]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_give_the_single_process_sequence(world):
    import torch.multiprocessing as mp

    import gen
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + world * 7 + (os.getpid() % 500)
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = dict(q.get(timeout=180) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, s, L = 65521, 4, 9
    A = gen.wiedemann_matrix(seed=31, n=601, p=p, n_random=3)
    X = gen.uniform_block(32, A.nrows, s, p)
    Y = gen.uniform_block(33, A.nrows, s, p)
    want = oracle.csr_block_sequence(A, X, Y, L)
    for r in range(world):
        assert np.array_equal(np.array(got[r]), np.asarray(want, dtype=np.int64).reshape(L, s, s)), r


@pytest.mark.gpu
def test_one_rank_on_the_library_kernels():
    """World size 1 over NCCL: the all-reduce and all-gather are identities,
    the projection, its reduction and the SpMM are the library's."""
    import torch
    import torch.distributed as dist

    import gen
    import oracle
    import paper_1004_3719_gb300 as ff
    from paper_1004_3719_gb300.dist_sequence import block_sequence, library_compute
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(29900 + os.getpid() % 90))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        for p, s in ((65521, 16), (2**31 - 1, 5)):
            A = gen.wiedemann_matrix(seed=34, n=20_011, p=p)
            X = gen.uniform_block(35, A.nrows, s, p)
            Y = gen.uniform_block(36, A.nrows, s, p)
            M = ff.Matrix.from_csr(A, transpose_mode=ff.TRANSPOSE.NONE)
            Xd = torch.from_numpy(X.view(np.int32)).cuda()
            comp = library_compute(M, Xd, p, s)
            S = block_sequence(A.nrows, s, 7, torch.from_numpy(Y.view(np.int32)).cuda(), comp)
            got = np.stack([t.cpu().numpy().view(np.uint32) for t in S])
            want = np.asarray(oracle.csr_block_sequence(A, X, Y, 7)).reshape(7, s, s)
            assert np.array_equal(got, want), p
    finally:
        dist.destroy_process_group()
