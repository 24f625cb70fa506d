"""Row sharding across ranks (one process per GPU) and the rank reductions of
the benchmark.

Rows are independent (each has its own rule, points and band, so the
assembly needs no data exchange between rows): a shard is a row range, given
to the assembly calls as row_begin / row_end.  Ranges are cut at x3-plane
boundaries so that each rank's partial contractions cover whole planes and
its band output is one contiguous block.  The coefficient gradient of the
adjoint is the one quantity a sharded run would have to sum across ranks
(neighbouring slabs share three coefficient layers); sum_over_ranks is that
reduction.
"""
from __future__ import annotations


def plane_row_ranges(n, world):
    """Contiguous row ranges, one per rank, cut at x3-plane boundaries (the
    last direction of n = (n1, n2[, n3]) basis-function counts), as even as
    the plane count allows.  Ranks beyond the plane count get empty ranges."""
    n = list(n)
    per_plane = 1
    for v in n[:-1]:
        per_plane *= v
    planes = n[-1]
    out = []
    for r in range(world):
        p0 = planes * r // world
        p1 = planes * (r + 1) // world
        out.append((p0 * per_plane, p1 * per_plane))
    return out


def shard_rows(n, rank, world):
    """This rank's row range of plane_row_ranges(n, world)."""
    return plane_row_ranges(n, world)[rank]


def _reduce(values, op, dist, device):
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return t.tolist()


def max_over_ranks(values, dist, device="cpu"):
    """Element-wise maximum of a list of numbers over all ranks (timing)."""
    return _reduce(values, dist.ReduceOp.MAX, dist, device)


def sum_over_ranks(values, dist, device="cpu"):
    """Element-wise sum of a list of numbers over all ranks."""
    return _reduce(values, dist.ReduceOp.SUM, dist, device)
