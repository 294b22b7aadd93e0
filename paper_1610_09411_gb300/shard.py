"""One census split over the ranks of a torch.distributed process group.

Every rank holds the whole graph.  escape_census5_part counts the work items a
rank owns (vertex ranks r of the degree order with r mod world = rank); the one
exchange step adds every rank's raw 128-bit sums and per-element arrays (K4 and
C4 per edge, C4 per vertex); escape_census5_finish applies the closed forms to
the totals.  NCCL has no 128-bit integers, so the sums travel as four 32-bit
limbs in int64 (a limb total stays below 2^63 for fewer than 2^31 ranks) and
the carries are resolved after the reduction, which keeps the result exact
modulo 2^128 -- and every true census count is below 2^127.
"""
from __future__ import annotations

LIMB_BITS = 32
LIMBS = 4
_MASK = (1 << LIMB_BITS) - 1


def to_limbs(values) -> list:
    """128-bit unsigned values (taken modulo 2^128) as 4 x 32-bit limbs each,
    least significant first."""
    out = []
    for v in values:
        v %= 1 << 128
        out.extend((v >> (LIMB_BITS * k)) & _MASK for k in range(LIMBS))
    return out


def from_limbs(limbs) -> list:
    """Inverse of to_limbs after a sum: limb totals may exceed 32 bits; the
    carries move up and the value is reduced modulo 2^128."""
    vals = []
    for i in range(0, len(limbs), LIMBS):
        v = sum(int(limbs[i + k]) << (LIMB_BITS * k) for k in range(LIMBS))
        vals.append(v % (1 << 128))
    return vals


def allreduce_u128(values, group=None, device="cpu") -> list:
    """Sum of every rank's 128-bit values, exactly modulo 2^128."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(to_limbs(values), dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return from_limbs(t.cpu().tolist())


def sharded_census(h, n: int, nnz: int, group=None, stream=None) -> dict:
    """The full census of the loaded graph `h` (n vertices, nnz entries),
    counted by every rank of `group` together; every rank returns it."""
    import torch
    import torch.distributed as dist
    from . import escape as esc
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    sums = esc.escape_census5_part(h, rank, world, stream)
    total = allreduce_u128(sums, group, device="cuda")
    k4e = torch.empty(max(nnz, 1), dtype=torch.int64, device="cuda")
    c4e = torch.empty(max(nnz, 1), dtype=torch.int64, device="cuda")
    c4v = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    esc.escape_part_counts(h, k4e, c4e, c4v, put=False, stream=stream)
    for t in (k4e, c4e, c4v):                  # int64 addition wraps like uint64: exact
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    esc.escape_part_counts(h, k4e, c4e, c4v, put=True, stream=stream)
    return esc.escape_census5_finish(h, total, stream)
