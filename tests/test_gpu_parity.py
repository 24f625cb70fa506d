"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

FP64 mode and the double-float mode (df64, FP64 output): max-entry and
Frobenius relative errors <= 1e-12 per matrix (the target the method's FP64
path is held to).  Mixed mode: <= 1e-6.  Sizes span
several row chunks per line, both line classes (interior / boundary) and
ragged chunk tails; tiny meshes make every row a boundary row.  At the
benchmark size the comparison runs on sampled row ranges, plus invariants
over every row."""
import numpy as np
import pytest

import oracle
from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-6


def rel_errs(A, O):
    d = A.astype(np.float64) - O
    return np.max(np.abs(d)) / np.max(np.abs(O)), np.linalg.norm(d) / np.linalg.norm(O)


def gpu_assemble(dim, p, nel, g, c, prec="fp64", rb=0, re=None, mass=True, stiffness=True):
    R = wq.Rules(dim, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda() if c is not None else None
    M, K = wq.assemble(R, gd, cd, prec, mass, stiffness, rb, re)
    out = (M.cpu().numpy() if M is not None else None, K.cpu().numpy() if K is not None else None)
    R.close()
    return out


def check(A, O, tol, what):
    em, ef = rel_errs(A, O)
    assert em <= tol and ef <= tol, f"{what}: rel_max {em:.3e} rel_fro {ef:.3e}"
    return em, ef


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("coef", ["sincos", "one"])
def test_2d_cubic_32x32(coef, prec):
    p, nel = 3, (32, 32)
    g, c = inputs.make(2, p, nel, 0.0, coef)
    M, K = gpu_assemble(2, p, nel, g, c, prec)
    Mo, Ko, _ = oracle.assemble(2, p, nel, g, c)
    check(M, Mo, FP64_TOL, "M")
    check(K, Ko, FP64_TOL, "K")


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("nel", [(20, 7, 6), (9, 11, 8), (37, 5, 5)])
def test_3d_full_parity(p, nel, prec):
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=3)
    M, K = gpu_assemble(3, p, nel, g, c, prec)
    Mo, Ko, off = oracle.assemble(3, p, nel, g, c)
    assert off < 1e-13
    check(M, Mo, FP64_TOL, "M")
    check(K, Ko, FP64_TOL, "K")


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("nel", [(1, 1, 1), (2, 1, 3), (3, 3, 3), (1, 4, 2), (4, 4, 1)])
def test_tiny_meshes_all_boundary(p, nel, prec):
    g, c = inputs.make(3, p, nel, 0.03, "exp", 0.2, seed=1)
    M, K = gpu_assemble(3, p, nel, g, c, prec)
    Mo, Ko, _ = oracle.assemble(3, p, nel, g, c)
    check(M, Mo, FP64_TOL, "M")
    check(K, Ko, FP64_TOL, "K")


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("p", [2, 3])
def test_2d_meshes(p, prec):
    for nel in [(1, 1), (5, 2), (40, 13)]:
        g, c = inputs.make(2, p, nel, 0.04, "exp", 0.1, seed=2)
        M, K = gpu_assemble(2, p, nel, g, c, prec)
        Mo, Ko, _ = oracle.assemble(2, p, nel, g, c)
        check(M, Mo, FP64_TOL, f"M {nel}")
        check(K, Ko, FP64_TOL, f"K {nel}")


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_row_ranges_and_single_matrices(prec):
    p, nel = 3, (23, 9, 7)
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=4)
    Mf, Kf = gpu_assemble(3, p, nel, g, c, prec)
    rows = Mf.shape[0]
    rng = np.random.default_rng(0)
    for _ in range(6):
        rb = int(rng.integers(0, rows))
        re = int(rng.integers(rb, rows + 1))
        M, K = gpu_assemble(3, p, nel, g, c, prec, rb=rb, re=re)
        assert np.array_equal(M, Mf[rb:re]) and np.array_equal(K, Kf[rb:re])
    M, _ = gpu_assemble(3, p, nel, g, c, prec, stiffness=False)
    _, K = gpu_assemble(3, p, nel, g, c, prec, mass=False)
    assert np.array_equal(M, Mf) and np.array_equal(K, Kf)
    # empty range
    M, K = gpu_assemble(3, p, nel, g, c, prec, rb=10, re=10)
    assert M.shape[0] == 0 and K.shape[0] == 0


def test_constant_coefficient_null_pointer():
    p, nel = 2, (7, 6, 5)
    g = inputs.geometry(p, nel, 0.05)
    M, K = gpu_assemble(3, p, nel, g, None)
    Mo, Ko, _ = oracle.assemble(3, p, nel, g, None)
    check(M, Mo, FP64_TOL, "M")
    check(K, Ko, FP64_TOL, "K")


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("name", ["3d_p3_64", "3d_p2_64"])
def test_benchmark_size_sampled(name, prec):
    w, g, c = inputs.workload(name)
    p, nel = w["p"], w["nel"]
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    M, K = wq.assemble(R, gd, cd, prec)
    rows = R.rows
    n1 = nel[0] + p
    n12 = n1 * (nel[1] + p)
    # row ranges: first rows (corner), a line through the middle, a plane edge, last rows
    ranges = [(0, 60), (n12 * 33 + n1 * 20, n12 * 33 + n1 * 21), (n12 * 40 + n1 * (nel[1] + p - 1), n12 * 40 + n12),
              (rows - 60, rows)]
    for rb, re in ranges:
        Mo, Ko, _ = oracle.assemble(3, p, nel, g, c, rb, re)
        check(M[rb:re].cpu().numpy(), Mo, FP64_TOL, f"M rows {rb}:{re}")
        check(K[rb:re].cpu().numpy(), Ko, FP64_TOL, f"K rows {rb}:{re}")
    # zero row sums of K over every row (any c, any separable map)
    ks = K.sum(dim=1).abs().max().item()
    kabs = K.abs().sum(dim=1).max().item()
    assert ks < 1e-12 * kabs
    # out-of-range band entries are exactly zero
    mask = torch.from_numpy(inputs.band_mask(nel, p)).cuda()
    assert (M * (1 - mask)).abs().max().item() == 0.0
    assert (K * (1 - mask)).abs().max().item() == 0.0
    R.close()


@pytest.mark.parametrize("p", [2, 3])
def test_mixed_precision(p):
    nel = (20, 9, 11)
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=5)
    M, K = gpu_assemble(3, p, nel, g, c, prec="mixed")
    assert M.dtype == np.float32
    Mo, Ko, _ = oracle.assemble(3, p, nel, g, c)
    em, ef = check(M, Mo, MIXED_TOL, "M mixed")
    ek, efk = check(K, Ko, MIXED_TOL, "K mixed")
    print(f"mixed p={p}: M {em:.2e}/{ef:.2e} K {ek:.2e}/{efk:.2e}")


def test_status_geometry_and_nonfinite():
    p, nel = 2, (5, 4, 3)
    g, c = inputs.make(3, p, nel, 0.0, "one")
    R = wq.Rules(3, p, nel)
    # a folded map: direction 2 reversed gives J_22 < 0 everywhere
    gbad = [g[0], g[1][::-1].copy(), g[2]]
    gd = [torch.from_numpy(x).cuda() for x in gbad]
    cd = torch.from_numpy(c).cuda()
    with pytest.raises(wq.WqError) as ei:
        wq.assemble(R, gd, cd, "fp64")
    assert ei.value.status == wq.WQ_ERR_GEOMETRY
    # the result is still written with |J| (Eq. Mass): equals the reflected map's
    M, K = wq.assemble(R, gd, cd, "fp64", check=False)
    assert wq.wq_status_check(R.handle, wq._stream_handle(None)) == wq.WQ_ERR_GEOMETRY
    gd_ok = [torch.from_numpy(x).cuda() for x in g]
    Mr, Kr = wq.assemble(R, gd_ok, cd, "fp64")
    assert torch.allclose(M, Mr, rtol=1e-13, atol=0) and torch.allclose(K, Kr, rtol=1e-13, atol=1e-300)
    # a NaN coefficient
    cn = c.copy()
    cn[3] = np.nan
    with pytest.raises(wq.WqError) as ei:
        wq.assemble(R, gd_ok, torch.from_numpy(cn).cuda(), "fp64")
    assert ei.value.status == wq.WQ_ERR_NONFINITE
    # the status is cleared by the check
    wq.assemble(R, gd_ok, cd, "fp64")
    R.close()


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_128_cubed_sampled(prec):
    # the 128^3 cubic workload (2.25M rows x 343): sampled rows against the
    # oracle, and invariants over every row
    w, g, c = inputs.workload("3d_p3_128")
    p, nel = w["p"], w["nel"]
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    M, K = wq.assemble(R, gd, cd, prec)
    n1 = nel[0] + p
    n12 = n1 * (nel[1] + p)
    tol = MIXED_TOL if prec == "mixed" else FP64_TOL
    # first rows, one interior line, a line of the boundary plane r2 = 1,
    # rows at the x1 end of an interior line, the last rows, and a seeded
    # sample of single rows anywhere in the mesh
    rng = np.random.default_rng(128)
    ranges = [(0, 40), (n12 * 70 + n1 * 60, n12 * 70 + n1 * 61), (n12 * 33 + n1 * 1, n12 * 33 + n1 * 2),
              (n12 * 99 + n1 * 77 + n1 - 9, n12 * 99 + n1 * 78 + 4), (R.rows - 40, R.rows)]
    ranges += [(int(r), int(r) + 1) for r in rng.integers(0, R.rows, size=24)]
    for rb, re in ranges:
        Mo, Ko, _ = oracle.assemble(3, p, nel, g, c, rb, re)
        check(M[rb:re].double().cpu().numpy(), Mo, tol, f"M rows {rb}:{re}")
        check(K[rb:re].double().cpu().numpy(), Ko, tol, f"K rows {rb}:{re}")
    kabs = K.abs().sum(dim=1, dtype=torch.float64)
    ks = K.sum(dim=1, dtype=torch.float64).abs()
    assert (ks <= (1e-5 if prec == "mixed" else 1e-12) * kabs).all()
    del M, K
    R.close()


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_assemble_to_host_overlapped(prec):
    # wq_assemble_mass_stiffness_host: host inputs, bands assembled range by
    # range with their host copies overlapped, equal the one-call device
    # result bit for bit (and c = 1 through a NULL coefficient)
    p, nel = 3, (21, 10, 9)
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=8)
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    gh = [torch.from_numpy(x).pin_memory() for x in g]
    ch = torch.from_numpy(c).pin_memory()
    for coef_dev, coef_host in ((cd, ch), (None, None)):
        M, K = wq.assemble(R, gd, coef_dev, prec)
        dt = M.dtype
        Mh = torch.empty((R.rows, R.band), dtype=dt).pin_memory()
        Kh = torch.empty((R.rows, R.band), dtype=dt).pin_memory()
        Md, Kd = torch.empty_like(M), torch.empty_like(K)
        gdd = [torch.empty_like(x) for x in gd]
        cdd = torch.empty_like(cd)
        for nch in (1, 5, 8):
            Mh.zero_()
            Kh.zero_()
            wq.assemble_to_host(R, gh, coef_host, prec, Mh, Kh, gdd, cdd, Md, Kd, nchunks=nch)
            torch.cuda.synchronize()
            assert torch.equal(Mh, M.cpu()) and torch.equal(Kh, K.cpu())
    assert wq.wq_status_check(R.handle, wq._stream_handle(None)) == wq.WQ_OK
    R.close()


def test_assemble_to_host_arguments():
    # argument errors are reported before anything is enqueued
    import ctypes

    p, nel = 2, (4, 3, 5)
    g, c = inputs.make(3, p, nel, 0.0, "one")
    R = wq.Rules(3, p, nel)
    gh = [torch.from_numpy(x) for x in g]
    gd = [x.cuda() for x in gh]
    M = torch.empty((R.rows, R.band), dtype=torch.float64, device="cuda")
    Mh = torch.empty((R.rows, R.band), dtype=torch.float64)
    s = torch.cuda.current_stream()
    hp, dp = [x.data_ptr() for x in gh], [x.data_ptr() for x in gd]
    mp, mhp = ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(Mh.data_ptr())
    ss = ctypes.c_void_p(s.cuda_stream)
    other = ctypes.c_void_p(torch.cuda.Stream().cuda_stream)
    call = wq.wq_assemble_mass_stiffness_host
    assert call(R.handle, hp, None, wq.WQ_FP64, mhp, mhp, dp, None, mp, mp, 0, R.rows, 0, ss, other) == wq.WQ_ERR_ARG
    assert call(R.handle, hp, None, wq.WQ_FP64, mhp, mhp, dp, None, mp, mp, 0, R.rows, 2, ss, ss) == wq.WQ_ERR_ARG
    assert call(R.handle, hp, None, wq.WQ_FP64, mhp, mhp, dp, None, mp, mp, 0, R.rows + 1, 2, ss, other) == \
        wq.WQ_ERR_ARG
    assert call(R.handle, hp, None, wq.WQ_FP64, None, None, dp, None, None, None, 3, 3, 2, ss, other) == wq.WQ_OK
    R.close()


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_plane_shards_equal_whole_mesh(prec):
    # the row slabs that ranks take (cut at x3 planes) assembled one by one
    # reproduce the whole mesh's bands bit for bit
    from paper_1710_01048_gb300 import shard

    p, nel = 3, (9, 7, 8)
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=31)
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    M, K = wq.assemble(R, gd, cd, prec)
    n = [v + p for v in nel]
    for world in (2, 3, 5):
        for rank in range(world):
            rb, re = shard.shard_rows(n, rank, world)
            Ms, Ks = wq.assemble(R, gd, cd, prec, row_begin=rb, row_end=re)
            assert torch.equal(Ms, M[rb:re]) and torch.equal(Ks, K[rb:re]), (world, rank)
    R.close()
