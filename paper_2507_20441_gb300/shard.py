"""Sharding samples across ranks (one process per GPU).

Every sample draws from its own counter-based stream keyed by (seed, sample
id), so a k-sample estimate splits into disjoint id ranges whose integer sums
add exactly: rank r of N runs tm_sample(k_r, seed, first_r) on a replica of
the graph and weights, and one all-reduce of hits2 and the counters gives the
single-process result bit for bit.  hits2 is up to 128 bits wide; it travels
as 16-bit limbs in 64-bit lanes so that sums over up to 2^47 ranks cannot
overflow.
"""
from __future__ import annotations


def sample_range(rank: int, world: int, k: int):
    """(first sample id, count) of rank's share of k samples."""
    base, extra = divmod(k, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


class combine:
    LIMB_BITS = 16
    LIMBS = 8          # 128-bit hits2

    @staticmethod
    def to_limbs(hits2: int, valid: int, rej_vertex: int, rej_delta: int, rej_order: int):
        mask = (1 << combine.LIMB_BITS) - 1
        h = [(hits2 >> (combine.LIMB_BITS * i)) & mask for i in range(combine.LIMBS)]
        return h + [valid, rej_vertex, rej_delta, rej_order]

    @staticmethod
    def from_limbs(limbs):
        h = sum(int(x) << (combine.LIMB_BITS * i) for i, x in enumerate(limbs[:combine.LIMBS]))
        return (h,) + tuple(int(x) for x in limbs[combine.LIMBS:])


def all_reduce_counts(hits2: int, valid: int, rej_vertex: int, rej_delta: int, rej_order: int, device=None):
    """One integer all-reduce (torch.distributed, the default group) of a
    rank's hits2 and counters; returns the sums over all ranks as
    (hits2, valid, rej_vertex, rej_delta, rej_order)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(combine.to_limbs(hits2, valid, rej_vertex, rej_delta, rej_order), dtype=torch.int64,
                     device=device)
    dist.all_reduce(t)
    return combine.from_limbs(t.tolist())
