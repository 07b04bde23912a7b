"""The block Wiedemann matrix sequence (Sec. 3, step 1) with the rows of A
split over the processes of a torch.distributed group, one GPU each.

Rank r owns the contiguous rows row_range(n, world, r) of A (a handle of that
row slice over all n columns), of X and of Y.  Per step i:

* S_i = sum over the ranks of X[rows]^T V_i[rows]: each rank adds its rows'
  products into a u64 accumulator (spmv_block_project), an all-reduce sums
  the accumulators, and spmv_block_project_finish reduces them mod p;
* V_{i+1}[rows] = A[rows, :] V_i: an all-gather of the row slices of V_i
  first, then the rank's SpMM (spmv_apply, s vectors).

The two exchanges are the only collectives; everything else is the library's
kernels.  The compute steps are passed in as callables (RowCompute) so that
the exchange logic can be run and tested with any local arithmetic.
"""
from __future__ import annotations


def row_range(n, world, rank):
    """Rows [r0, r1) of rank `rank` when n rows are split as evenly as
    possible over `world` ranks (the first n % world ranks get one more)."""
    base, extra = divmod(int(n), int(world))
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


class RowCompute:
    """The local arithmetic of one rank.

    project(V_rows, Sacc): add X[rows]^T V_rows into the int64 tensor Sacc (s x s);
    finish(Sacc) -> S: S = Sacc mod p (s x s), and zero Sacc;
    apply(V_full) -> V_rows: A[rows, :] V_full mod p (V_full: n x s).
    """

    def __init__(self, project, finish, apply):
        self.project, self.finish, self.apply = project, finish, apply


def library_compute(M_rows, X_rows, p, s, stream=None):
    """RowCompute on the library's kernels: M_rows a Matrix (or handle owner)
    of the rank's row slice of A (all n columns), X_rows its rows of X (an
    int32 CUDA tensor, rows x s)."""
    import torch

    from ._api import spmv_apply, spmv_block_project, spmv_block_project_finish

    nrows = X_rows.shape[0]
    S = torch.empty((s, s), dtype=torch.int32, device=X_rows.device)

    def project(V_rows, Sacc):
        spmv_block_project(p, nrows, s, X_rows, V_rows, Sacc, stream)

    def finish(Sacc):
        spmv_block_project_finish(p, s, Sacc, S, stream)
        return S.clone()

    def apply(V_full):
        out = torch.empty((nrows, s), dtype=torch.int32, device=V_full.device)
        spmv_apply(M_rows.handle, V_full, s, out, s, s, 1, 0, stream)
        return out

    return RowCompute(project, finish, apply)


def block_sequence(n, s, L, Y_rows, compute, group=None):
    """S_0 .. S_{L-1} (a list of s x s tensors, the same on every rank) for
    the rank's rows Y_rows of Y (rows x s) and its RowCompute."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    sizes = [row_range(n, world, r) for r in range(world)]
    rmax = max(r1 - r0 for r0, r1 in sizes)
    V = Y_rows.contiguous()
    Sacc = torch.zeros((s, s), dtype=torch.int64, device=V.device)
    # the all-gather moves equal-sized pieces: each rank's rows padded to rmax
    pad = torch.zeros((rmax, s), dtype=V.dtype, device=V.device)
    parts = [torch.empty((rmax, s), dtype=V.dtype, device=V.device) for _ in range(world)]
    out = []
    for i in range(L):
        compute.project(V, Sacc)
        dist.all_reduce(Sacc, group=group)      # exact: u64 sums far below 2^63
        out.append(compute.finish(Sacc))
        if i + 1 < L:
            pad[:V.shape[0]].copy_(V)
            dist.all_gather(parts, pad, group=group)
            V = compute.apply(torch.cat([q[:r1 - r0] for q, (r0, r1) in zip(parts, sizes)], 0).contiguous())
    return out


__all__ = ["row_range", "RowCompute", "library_compute", "block_sequence"]
