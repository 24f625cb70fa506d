"""Row sharding across ranks (one process per GPU) and the rank reductions of
the benchmark.

Rows are independent (each has its own rule, points and band, so the
assembly needs no data exchange between rows): a shard is a row range, given
to the assembly calls as row_begin / row_end.  Ranges are cut at x3-plane
boundaries so that each rank's partial contractions cover whole planes and
its band output is one contiguous block.  The coefficient gradient of the
adjoint is the one quantity a sharded run has to sum across ranks: a slab of
rows touches the coefficient layers of its planes plus a halo (p layers below,
three above, through the cubic coefficient spline), so neighbouring slabs'
partial gradients overlap there.  halo_reduce_gradient sums exactly those
overlaps into the layers each rank owns, with point-to-point messages between
the ranks concerned (all_reduce of the whole gradient is the simple
alternative).
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


def coef_layers_touched(n_last, nel_last, p, row_planes):
    """Coefficient layers [lo, hi) of the last direction that rows in planes
    [row_planes[0], row_planes[1]) touch: row r spans elements
    max(0, r - p) .. min(nel_last - 1, r), and each element the four layers
    e .. e + 3 of the cubic coefficient spline.  Empty planes give (0, 0)."""
    a, b = row_planes
    if b <= a:
        return (0, 0)
    return (max(0, a - p), min(nel_last - 1, b - 1) + 4)


def owned_coef_layers(nel_last, p, world):
    """The coefficient layers each rank owns (a partition of the nel_last + 3
    layers): those of its plane range, the last rank also the ones past the
    last row plane."""
    n_last = nel_last + p
    nc = nel_last + 3
    out = []
    for r in range(world):
        a = n_last * r // world
        b = n_last * (r + 1) // world if r < world - 1 else max(n_last, nc)
        out.append((min(a, nc), min(b, nc)))
    return out


def halo_reduce_gradient(grad, nel, p, rank, world, dist):
    """Sums the ranks' partial gradients over the layers this rank owns.

    grad: this rank's partial gradient, a torch tensor of prod(nel_a + 3)
    values (x fastest, so a coefficient layer of the last direction is one
    contiguous block), non-zero only on the layers its rows touch.  Every
    rank sends the part of its touched layers that another rank owns to that
    rank, and adds what it receives, in rank order, to its own layers.
    Returns this rank's owned layer range; grad is updated in place there
    (the other layers are left as they were)."""
    nel = [int(v) for v in nel]
    layer = 1
    for v in nel[:-1]:
        layer *= v + 3
    n_last = nel[-1] + p
    planes = [(n_last * r // world, n_last * (r + 1) // world) for r in range(world)]
    touched = [coef_layers_touched(n_last, nel[-1], p, planes[r]) for r in range(world)]
    owned = owned_coef_layers(nel[-1], p, world)

    def overlap(u, v):
        lo, hi = max(u[0], v[0]), min(u[1], v[1])
        return (lo, hi) if hi > lo else None

    sends, recvs = [], []
    for s in range(world):
        if s == rank:
            continue
        ov = overlap(touched[rank], owned[s])
        if ov is not None:
            sends.append(dist.isend(grad[ov[0] * layer:ov[1] * layer].contiguous(), dst=s))
        ov = overlap(touched[s], owned[rank])
        if ov is not None:
            buf = grad.new_empty((ov[1] - ov[0]) * layer)
            recvs.append((s, ov, buf, dist.irecv(buf, src=s)))
    for s, ov, buf, req in recvs:  # rank order: the sum does not depend on timing
        req.wait()
        grad[ov[0] * layer:ov[1] * layer] += buf
    for req in sends:
        req.wait()
    return owned[rank]
