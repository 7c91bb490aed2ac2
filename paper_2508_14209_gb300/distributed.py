"""Block-row multisketch across ranks (the distribution of Section 7).

Every rank holds a contiguous block of rows of the tall [A b]
(`row_partition`).  The CountSketch is a sum over rows, hashed with the
*global* row index, and the Gaussian stage is linear, so

    Z = G S [A b] = sum over ranks of G S_r [A_r b_r],

where S_r is the CountSketch of rank r's rows with their global indices.
Each rank therefore computes its block's Z with `ms_sketch_rows` (G comes
from the seed on every rank: nothing is broadcast), and one sum all-reduce of
the p x (n+1) FP64 Z completes the sketch.  The communication is the same as
a distributed Gaussian sketch's, as Section 7 notes; the QR of Z then runs on
any rank.
"""
from __future__ import annotations

import torch


def row_partition(d: int, world: int, rank: int):
    """(row0, rows) of rank `rank`'s block in a balanced contiguous split of d
    rows over `world` ranks (the first d % world ranks take one more row)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(int(d), int(world))
    row0 = rank * base + min(rank, extra)
    return row0, base + (1 if rank < extra else 0)


def ms_sketch_distributed(A_local, row0, k, p, seed, b_local=None, gemm_prec=None, group=None,
                          local_sketch=None, **kwargs):
    """Z = G S [A b] of the row-distributed matrix, on every rank.

    A_local (and b_local) hold rows row0 .. row0 + d_local - 1.  The local
    block's sketch is `local_sketch(A_local, b_local, row0)` if given (any
    function returning the block's p x ncol FP64 Z), else the library's
    `ms_sketch_rows`.  Returns the all-reduced Z (the same tensor)."""
    import torch.distributed as dist

    if local_sketch is None:
        from . import GEMM_F64, ms_sketch_rows

        gp = GEMM_F64 if gemm_prec is None else gemm_prec
        Z = ms_sketch_rows(A_local, int(row0), k, p, seed, b=b_local, gemm_prec=gp, **kwargs)
    else:
        Z = local_sketch(A_local, b_local, int(row0))
    if not isinstance(Z, torch.Tensor):
        Z = torch.as_tensor(Z)
    Z = Z.contiguous()
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(Z, op=dist.ReduceOp.SUM, group=group)
    return Z
