"""Matrix-free apply (wq_apply_mass_stiffness) and the load vector
(wq_assemble_load, Eq. Load) through the C-ABI.

Parity: y = M x and y = K x against the band matvec of the oracle's bands
(tests/bandops.py, pinned in test_oracle_apply.py), per row relative to
sum |B| |x| over the row: <= 1e-12 for fp64 and df64, <= 1e-5 for mixed.
Sizes span several apply chunks per line (24 rows in 3D, the assembly's
chunks in 2D) with ragged tails, interior and boundary lines, and tiny
all-boundary meshes, in 3D (split kernels) and 2D (fused kernel).  The load vector
for f = 1 on the identity map is pinned to its closed form directly.  At the
benchmark size (64^3 cubic) the apply is compared with the band of the
assembly on the GPU (itself parity-tested against the oracle) and K 1 = 0 is
checked over every row."""
import numpy as np
import pytest

import oracle
from bandops import band_abs_matvec, band_columns, band_matvec
from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df64": 1e-12, "mixed": 1e-5}
MESHES = [(3, (23, 9, 7)), (2, (40, 6, 5)), (3, (1, 1, 1)), (2, (2, 3, 4)), (3, (5, 17, 3))]


def gpu_inputs(p, nel, seed, prec):
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=seed)
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(v).cuda() for v in g]
    cd = torch.from_numpy(c).cuda()
    dt = torch.float32 if prec == "mixed" else torch.float64
    x = np.random.default_rng(seed + 100).standard_normal(R.rows)
    if prec == "mixed":
        x = x.astype(np.float32).astype(np.float64)  # the values the FP32 path sees
    return R, g, c, gd, cd, x, torch.from_numpy(x).to(dt).cuda()


def row_errors(y, yo, scale):
    return np.abs(y.astype(np.float64) - yo) / np.maximum(scale, 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
@pytest.mark.parametrize("p,nel", MESHES)
def test_apply_matches_oracle_band_matvec(p, nel, prec):
    R, g, c, gd, cd, x, xd = gpu_inputs(p, nel, 11, prec)
    yM, yK = wq.apply(R, gd, xd, cd, prec)
    M, K, _ = oracle.assemble(3, p, nel, g, c)
    cols = band_columns(3, p, nel)
    for y, B in ((yM, M), (yK, K)):
        e = row_errors(y.cpu().numpy(), band_matvec(B, cols, x), band_abs_matvec(B, cols, x))
        assert e.max() <= TOL[prec], f"{nel} {prec}: {e.max():.3e}"
    R.close()


MESHES_2D = [(3, (32, 32)), (2, (40, 9)), (3, (1, 1)), (2, (3, 50)), (3, (57, 2))]


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
@pytest.mark.parametrize("p,nel", MESHES_2D)
def test_apply_2d_matches_oracle_band_matvec(p, nel, prec):
    g, c = inputs.make(2, p, nel, 0.05, "exp", 0.1, seed=13)
    R = wq.Rules(2, p, nel)
    gd = [torch.from_numpy(v).cuda() for v in g]
    cd = torch.from_numpy(c).cuda()
    dt = torch.float32 if prec == "mixed" else torch.float64
    x = np.random.default_rng(14).standard_normal(R.rows)
    if prec == "mixed":
        x = x.astype(np.float32).astype(np.float64)
    yM, yK = wq.apply(R, gd, torch.from_numpy(x).to(dt).cuda(), cd, prec)
    M, K, _ = oracle.assemble(2, p, nel, g, c)
    cols = band_columns(2, p, nel)
    for y, B in ((yM, M), (yK, K)):
        e = row_errors(y.cpu().numpy(), band_matvec(B, cols, x), band_abs_matvec(B, cols, x))
        assert e.max() <= TOL[prec], f"{nel} {prec}: {e.max():.3e}"
    # row ranges and the load vector (f = 1 on the identity map: the basis integrals)
    rb, re = 7, R.rows - 5
    a, b = wq.apply(R, gd, torch.from_numpy(x).to(dt).cuda(), cd, prec, row_begin=rb, row_end=re)
    assert torch.equal(a, yM[rb:re]) and torch.equal(b, yK[rb:re])
    gi = [torch.from_numpy(v).cuda() for v in inputs.geometry(p, nel)]
    bl = wq.assemble_load(R, gi, None, prec).cpu().numpy().astype(np.float64)
    ints = []
    for ne in nel:
        t = np.concatenate([np.zeros(p), np.linspace(0.0, 1.0, ne + 1), np.ones(p)])
        ints.append(np.array([(t[r + p + 1] - t[r]) / (p + 1) for r in range(ne + p)]))
    expect = np.multiply.outer(ints[1], ints[0]).reshape(-1)
    tol = {"fp64": 1e-14, "df64": 1e-13, "mixed": 1e-6}[prec]
    assert np.max(np.abs(bl - expect)) <= tol * np.max(expect)
    R.close()


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_row_ranges_single_outputs_and_load(prec):
    p, nel = 3, (23, 9, 7)
    R, g, c, gd, cd, x, xd = gpu_inputs(p, nel, 12, prec)
    yM, yK = wq.apply(R, gd, xd, cd, prec)
    rng = np.random.default_rng(1)
    for _ in range(5):
        rb = int(rng.integers(0, R.rows))
        re = int(rng.integers(rb, R.rows + 1))
        a, b = wq.apply(R, gd, xd, cd, prec, row_begin=rb, row_end=re)
        assert torch.equal(a, yM[rb:re]) and torch.equal(b, yK[rb:re])
    a, _ = wq.apply(R, gd, xd, cd, prec, stiffness=False)
    _, b = wq.apply(R, gd, xd, cd, prec, mass=False)
    assert torch.equal(a, yM) and torch.equal(b, yK)
    # load vector = M(f) 1, bit for bit the apply with x = 1
    ones = torch.ones_like(xd)
    a, _ = wq.apply(R, gd, ones, cd, prec, stiffness=False)
    bl = wq.assemble_load(R, gd, cd, prec)
    assert torch.equal(a, bl)
    # empty range
    a, b = wq.apply(R, gd, xd, cd, prec, row_begin=7, row_end=7)
    assert a.numel() == 0 and b.numel() == 0
    R.close()


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
@pytest.mark.parametrize("p,nel", [(3, (20, 17, 6)), (2, (9, 33, 4)), (3, (1, 2, 1))])
def test_load_vector_unit_source_closed_form(p, nel, prec):
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(v).cuda() for v in inputs.geometry(p, nel)]
    b = wq.assemble_load(R, gd, None, prec).cpu().numpy().astype(np.float64)
    ints = []
    for e in nel:
        t = np.concatenate([np.zeros(p), np.linspace(0.0, 1.0, e + 1), np.ones(p)])
        ints.append(np.array([(t[r + p + 1] - t[r]) / (p + 1) for r in range(e + p)]))
    expect = np.multiply.outer(ints[2], np.multiply.outer(ints[1], ints[0])).reshape(-1)
    # FP64: a few ulps; double-float carries 48 bits (unit roundoff 2^-48,
    # 3.6e-15) through a few hundred operations per row; FP32: 2^-24 likewise
    tol = {"fp64": 1e-14, "df64": 1e-13, "mixed": 1e-6}[prec]
    assert np.max(np.abs(b - expect)) <= tol * np.max(expect)
    assert abs(b.sum() - 1.0) <= (1e-5 if prec == "mixed" else 1e-13)
    R.close()


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_load_vector_matches_oracle(prec):
    p, nel = 3, (13, 6, 9)
    g, f = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=21)
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(v).cuda() for v in g]
    b = wq.assemble_load(R, gd, torch.from_numpy(f).cuda(), prec).cpu().numpy()
    M, _, _ = oracle.assemble(3, p, nel, g, f)
    cols = band_columns(3, p, nel)
    one = np.ones(M.shape[0])
    e = row_errors(b, band_matvec(M, cols, one), band_abs_matvec(M, cols, one))
    assert e.max() <= TOL[prec]
    R.close()


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_benchmark_size_against_assembled_band(prec):
    # 64^3 cubic, the benchmark workload: apply vs the assembled band's matvec
    # on the GPU in FP64, every row; K 1 = 0 over every row
    w, g, c = inputs.workload("3d_p3_64")
    p, nel = w["p"], w["nel"]
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(v).cuda() for v in g]
    cd = torch.from_numpy(c).cuda()
    dt = torch.float32 if prec == "mixed" else torch.float64
    gen = torch.Generator(device="cuda").manual_seed(3)
    xd = torch.randn(R.rows, dtype=torch.float64, device="cuda", generator=gen).to(dt)
    yM, yK = wq.apply(R, gd, xd, cd, prec)
    M, K = wq.assemble(R, gd, cd, prec)
    cols = torch.from_numpy(band_columns(3, p, nel)).cuda()
    ok = cols >= 0
    xs = torch.where(ok, xd.double()[cols.clamp(min=0)], torch.zeros((), dtype=torch.float64, device="cuda"))
    for y, B in ((yM, M), (yK, K)):
        ref = (B.double() * xs).sum(1)
        scale = (B.double().abs() * xs.abs()).sum(1)
        e = ((y.double() - ref).abs() / scale).max().item()
        assert e <= TOL[prec], f"{prec}: {e:.3e}"
    del xs
    one = torch.ones(R.rows, dtype=dt, device="cuda")
    _, k1 = wq.apply(R, gd, one, cd, prec, mass=False)
    e = (k1.double().abs() / K.double().abs().sum(1)).max().item()
    assert e <= (1e-5 if prec == "mixed" else 1e-13)
    R.close()


def test_apply_arguments():
    p, nel = 2, (4, 5, 3)
    R, g, c, gd, cd, x, xd = gpu_inputs(p, nel, 3, "fp64")
    y = torch.empty(R.rows, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    gp = [v.data_ptr() for v in gd]
    import ctypes
    st = wq.wq_apply_mass_stiffness(R.handle, gp, None, wq.WQ_FP64, None, ctypes.c_void_p(y.data_ptr()), None, 0,
                                    R.rows, ctypes.c_void_p(s))
    assert st == wq.WQ_ERR_ARG  # x missing
    st = wq.wq_apply_mass_stiffness(R.handle, gp, None, wq.WQ_FP64, ctypes.c_void_p(xd.data_ptr()), None, None, 0,
                                    R.rows, ctypes.c_void_p(s))
    assert st == wq.WQ_ERR_ARG  # no output
    st = wq.wq_assemble_load(R.handle, gp, None, wq.WQ_FP64, None, 0, R.rows, ctypes.c_void_p(s))
    assert st == wq.WQ_ERR_ARG  # no output
    R.close()
    # the comparison rules: not supported by the apply kernels
    Rg = wq.Rules(3, 2, (3, 3, 3), rule="gl")
    g3 = [torch.from_numpy(v).cuda() for v in inputs.geometry(2, (3, 3, 3))]
    with pytest.raises(wq.WqError) as ei:
        wq.assemble_load(Rg, g3)
    assert ei.value.status == wq.WQ_ERR_UNSUPPORTED
    Rg.close()
