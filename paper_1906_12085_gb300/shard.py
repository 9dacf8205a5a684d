"""Row-block partition of A for rsvd_sharded and its host reduction over torch.distributed.

A = [A_1; ...; A_N]: rank r of N owns rows [row_block(m, N, r)), contiguous and balanced
(block sizes differ by at most one row).  The library sums what the method reduces over
rows through a host callback; dist_allreduce() supplies one that runs a SUM all-reduce of
a CPU tensor over a torch.distributed process group (gloo here: there is one GPU per run,
so no NCCL or device collective is involved).
"""
from __future__ import annotations


def row_block(m: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [r0, r1) of rank `rank` among `world` ranks: the first m % world ranks take one
    row more than the others."""
    if world < 1 or not 0 <= rank < world or m < 0:
        raise ValueError(f"row_block({m}, {world}, {rank})")
    base, extra = divmod(m, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def dist_allreduce(group=None):
    """reduce_inplace(buf) for rsvd_sharded: buf (float64 numpy) <- its sum over the ranks of
    `group` (every rank receives the same bits: gloo sums in a fixed order)."""
    import torch
    import torch.distributed as dist

    def reduce_inplace(buf):
        t = torch.from_numpy(buf)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)

    return reduce_inplace
