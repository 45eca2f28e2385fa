"""Sharding a volume's bricks over the ranks of a torch.distributed group.

Bricks are independent (Sec. 3: every brick is encoded and decoded on its own), so decoding needs
no exchange between ranks: each rank owns a contiguous range of brick ids.  Encoding has one
exchange, the frequency prepass (Sec. 3.4): the two tables must be the same on every rank, so the
32 nibble counts of each rank's sampled bricks are summed (all-reduce) before they are normalised.
"""
import numpy as np


def brick_range(n_bricks, rank, world):
    """Contiguous brick ids [lo, hi) owned by `rank` (sizes differ by at most one)."""
    base, extra = divmod(int(n_bricks), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shared_tables(local_counts, group=None):
    """Sum each rank's 32 prepass counts over the group and normalise them (same tables on every rank)."""
    import torch
    import torch.distributed as dist
    import paper_2308_16619_b300 as csgv
    c = torch.tensor(np.asarray(local_counts, np.int64), dtype=torch.int64)
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "nccl":
            c = c.cuda()
        dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    return csgv.csgv_freq_table_from_counts(c.cpu().numpy().astype(np.uint64))
