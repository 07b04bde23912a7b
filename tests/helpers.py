"""Shared helpers for the tests: seeded inputs and GPU<->host copies."""
import numpy as np

import gen


def rand_block(seed, rows, nvec, m):
    rng = np.random.default_rng(seed)
    v = (rng.random((rows, nvec)) * m).astype(np.uint64)
    v = np.minimum(v, m - 1).astype(np.uint32)
    return v[:, 0].copy() if nvec == 1 else v


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def to_host(t):
    return t.detach().cpu().numpy().view(np.uint32)


def with_modulus(A, m, pm_fraction=0.2, seed=0):
    """A copy of A's structure with fresh nonzero residues mod m."""
    rng = gen.rng_for(seed, 99, m)
    vals = gen.residues(rng, A.nnz, m, pm_fraction)
    return gen.CSR(A.nrows, A.ncols, A.row_ptr, A.col, vals, m, A.name)
