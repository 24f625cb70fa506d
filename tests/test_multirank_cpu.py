"""The N > 1 host path on CPU: two gloo ranks shard the rows of a mesh at
x3-plane boundaries, count their shards' non-zeros and flops with the host
library, and reduce them; the shards must cover every row exactly once and
the reduced counts must equal the whole mesh's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1710_01048_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, dim, p, nel, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1710_01048_gb300 import binding as wq

        R = wq.Rules(dim, p, nel, device=False)
        n = [v + p for v in nel]
        rb, re = shard.shard_rows(n, rank, world)
        nnz = wq.wq_band_nnz_rows(R.handle, rb, re)
        flops = R.flops(row_begin=rb, row_end=re)[0] if re > rb else 0.0
        tot_nnz, tot_flops, nrows = shard.sum_over_ranks([nnz, flops, re - rb], dist)
        mx = shard.max_over_ranks([float(rank), -float(rank)], dist)
        ranges = [None] * world
        dist.all_gather_object(ranges, (rb, re))
        if rank == 0:
            q.put(dict(tot_nnz=tot_nnz, tot_flops=tot_flops, nrows=nrows, mx=mx, ranges=ranges,
                       nnz_all=wq.wq_band_nnz_rows(R.handle, 0, R.rows), flops_all=R.flops()[0], rows=R.rows))
        R.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dim,p,nel", [(3, 3, (6, 5, 7)), (3, 2, (4, 3, 1)), (2, 3, (9, 4))])
def test_two_rank_row_shards(dim, p, nel):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, dim, p, nel, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    # the shards tile the rows in order, cut at plane boundaries
    n = [v + p for v in nel]
    per_plane = 1
    for v in n[:-1]:
        per_plane *= v
    ranges = res["ranges"]
    assert ranges[0][0] == 0 and ranges[-1][1] == res["rows"]
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    for a0, a1 in ranges:
        assert a0 % per_plane == 0 and a1 % per_plane == 0
    assert res["nrows"] == res["rows"]
    assert res["tot_nnz"] == res["nnz_all"]
    assert abs(res["tot_flops"] - res["flops_all"]) <= 1e-9 * res["flops_all"]
    assert res["mx"] == [1.0, 0.0]


def test_plane_ranges_more_ranks_than_planes():
    ranges = shard.plane_row_ranges((4, 4, 3), 5)
    assert sum(b - a for a, b in ranges) == 48
    assert all(a % 16 == 0 and b % 16 == 0 for a, b in ranges)
    assert sum(1 for a, b in ranges if a == b) == 2


def _adjoint_rank_main(rank, world, port, p, nel, q):
    # each rank: the oracle's gradient of its own rows' weights (the partial
    # gradient a sharded adjoint computes), then the halo reduction
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np

        import oracle
        from paper_1710_01048_gb300 import inputs

        g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=41)
        rows = int(np.prod([v + p for v in nel]))
        band = (2 * p + 1) ** 3
        rng = np.random.default_rng(42)
        G = rng.standard_normal((rows, band))
        H = rng.standard_normal((rows, band))
        rb, re = shard.shard_rows([v + p for v in nel], rank, world)
        mask = np.zeros((rows, 1))
        mask[rb:re] = 1.0
        part = torch.from_numpy(oracle.gradient(3, p, nel, g, G * mask, H * mask))
        lo, hi = shard.halo_reduce_gradient(part, nel, p, rank, world, dist)
        layer = (nel[0] + 3) * (nel[1] + 3)
        owned = part[lo * layer:hi * layer].numpy().copy()
        pieces = [None] * world
        dist.all_gather_object(pieces, (lo, hi, owned))
        if rank == 0:
            full = oracle.gradient(3, p, nel, g, G, H)
            q.put(dict(pieces=pieces, full=full, layer=layer, ncl=nel[2] + 3))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,p,nel", [(2, 3, (4, 3, 6)), (3, 2, (3, 4, 5)), (3, 3, (3, 2, 2))])
def test_sharded_adjoint_halo_reduction(world, p, nel):
    # the owned coefficient layers of the halo-reduced partial gradients tile
    # the layers and equal the gradient of the whole mesh
    import numpy as np

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_adjoint_rank_main, args=(r, world, port, p, nel, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=300)
        assert pr.exitcode == 0
    layer, full = res["layer"], res["full"]
    covered = []
    for lo, hi, owned in res["pieces"]:
        covered.extend(range(lo, hi))
        ref = full[lo * layer:hi * layer]
        assert np.max(np.abs(owned - ref)) <= 1e-12 * np.max(np.abs(full))
    assert sorted(covered) == list(range(res["ncl"]))


def _assembly_rank_main(rank, world, port, dim, p, nel, q):
    # each rank assembles its own row slab (the oracle stands in for the
    # device call on a CPU-only host); rank 0 gathers the slabs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1710_01048_gb300 import inputs

        g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=43)
        n = [v + p for v in nel]
        rb, re = shard.shard_rows(n, rank, world)
        M, K, _ = oracle.assemble(dim, p, nel, g, c, rb, re)
        pieces = [None] * world
        dist.all_gather_object(pieces, (rb, re, M, K))
        if rank == 0:
            Mf, Kf, _ = oracle.assemble(dim, p, nel, g, c)
            q.put(dict(pieces=pieces, Mf=Mf, Kf=Kf))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,dim,p,nel", [(2, 3, 3, (5, 4, 6)), (3, 3, 2, (4, 3, 5)), (2, 2, 3, (7, 6))])
def test_rank_slabs_reassemble_the_mesh(world, dim, p, nel):
    # the ranks' slabs, each assembled over its own row range, tile the rows
    # and equal the whole mesh's bands row for row (every row has its own
    # rule and points, so a slab needs nothing from another rank)
    import numpy as np

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_assembly_rank_main, args=(r, world, port, dim, p, nel, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=300)
        assert pr.exitcode == 0
    rows = res["Mf"].shape[0]
    nxt = 0
    for rb, re, M, K in res["pieces"]:
        assert rb == nxt
        nxt = re
        assert np.array_equal(M, res["Mf"][rb:re]) and np.array_equal(K, res["Kf"][rb:re])
    assert nxt == rows
