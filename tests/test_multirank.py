"""The N-rank path on CPU (gloo, world size 2): independent units are split
round robin with no data-path collective, and the job time is the maximum
over ranks.  Each rank computes its share of a small batch with the CPU
oracle; the union must equal the single-process result."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import gen
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = gen.batch_problems(seed=5, count=9, rows_lo=30, rows_hi=300)
    mine = bench.shard(len(probs), rank, world)
    out = {}
    for j in mine:
        A, s = probs[j]
        x = gen.uniform_block(100 + j, A.ncols, s, A.modulus)
        out[j] = oracle.csr_spmv(A, x)
    gathered = [None] * world
    dist.all_gather_object(gathered, out)
    t = bench.max_over_ranks(dist, 1.5 + rank)
    if rank == 0:
        q.put((gathered, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_units_and_max_time():
    import torch.multiprocessing as mp
    import gen
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 2.5
    merged = {}
    for d in gathered:
        assert not set(d) & set(merged)          # no unit done twice
        merged.update(d)
    probs = gen.batch_problems(seed=5, count=9, rows_lo=30, rows_hi=300)
    assert sorted(merged) == list(range(len(probs)))
    for j, (A, s) in enumerate(probs):
        x = gen.uniform_block(100 + j, A.ncols, s, A.modulus)
        assert np.array_equal(merged[j], oracle.csr_spmv(A, x))
