"""The adjoint of the assembly (wq_assemble_adjoint) and its autograd wrapper.

J(C) = sum G * K(C) + sum H * M(C) is linear in the coefficient spline's C,
so its gradient is checked three independent ways:
* against the oracle's gradient (nested loops over rows, points and columns,
  no sum factorisation) on small meshes: <= 1e-12 relative in FP64 and df64,
  <= 1e-5 in the mixed mode (FP32 weights and contractions);
* Euler's identity <dJ/dC, C> = J(C) with J from the forward GPU assembly;
* central finite differences of J along random directions (h = 1e-6) on the
  96^3 cubic workload: <= 1e-6 relative.
"""
import numpy as np
import pytest

import oracle
from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5


def rel_max(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def gpu_grad(dim, p, nel, g, G, H, prec="fp64", rb=0, re=None):
    R = wq.Rules(dim, p, nel)
    dt = torch.float32 if prec == "mixed" else torch.float64
    gd = [torch.from_numpy(x).cuda() for x in g]
    re = R.rows if re is None else re
    Gd = torch.from_numpy(G[rb:re]).to(dt).cuda().contiguous() if G is not None else None
    Hd = torch.from_numpy(H[rb:re]).to(dt).cuda().contiguous() if H is not None else None
    out = wq.assemble_adjoint(R, gd, Gd, Hd, prec, rb, re).cpu().numpy()
    R.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("nel", [(12, 12, 12), (20, 7, 6), (3, 9, 2)])
def test_gradient_vs_oracle_3d(p, nel, prec):
    g, _ = inputs.make(3, p, nel, 0.05, "one")
    G = inputs.band_random(nel, p, 11)
    H = inputs.band_random(nel, p, 12)
    go = oracle.gradient(3, p, nel, g, G, H)
    gg = gpu_grad(3, p, nel, g, G, H, prec)
    err = rel_max(gg, go)
    assert err <= (MIXED_TOL if prec == "mixed" else FP64_TOL), f"rel_max {err:.3e}"


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("p", [2, 3])
def test_gradient_vs_oracle_2d(p, prec):
    for nel in [(1, 1), (32, 32), (41, 5)]:
        g, _ = inputs.make(2, p, nel, 0.04, "one")
        G = inputs.band_random(nel, p, 13)
        H = inputs.band_random(nel, p, 14)
        go = oracle.gradient(2, p, nel, g, G, H)
        gg = gpu_grad(2, p, nel, g, G, H, prec)
        assert rel_max(gg, go) <= FP64_TOL, f"{nel}"


@pytest.mark.parametrize("p", [2, 3])
def test_gradient_tiny_meshes(p):
    for nel in [(1, 1, 1), (2, 1, 3), (4, 4, 1)]:
        g, _ = inputs.make(3, p, nel, 0.03, "one")
        G = inputs.band_random(nel, p, 15)
        H = inputs.band_random(nel, p, 16)
        go = oracle.gradient(3, p, nel, g, G, H)
        assert rel_max(gpu_grad(3, p, nel, g, G, H), go) <= FP64_TOL, f"{nel}"


def test_gradient_single_weights_and_row_ranges():
    p, nel = 3, (23, 9, 7)
    g, _ = inputs.make(3, p, nel, 0.05, "one")
    G = inputs.band_random(nel, p, 17)
    H = inputs.band_random(nel, p, 18)
    rows = G.shape[0]
    # G only, H only: the oracle with the other weight zero
    assert rel_max(gpu_grad(3, p, nel, g, G, None), oracle.gradient(3, p, nel, g, G, None)) <= FP64_TOL
    assert rel_max(gpu_grad(3, p, nel, g, None, H), oracle.gradient(3, p, nel, g, None, H)) <= FP64_TOL
    # a row range: the oracle with the weights zero outside it
    rng = np.random.default_rng(1)
    for _ in range(4):
        rb = int(rng.integers(0, rows - 1))
        re = int(rng.integers(rb + 1, rows + 1))
        Gz, Hz = np.zeros_like(G), np.zeros_like(H)
        Gz[rb:re], Hz[rb:re] = G[rb:re], H[rb:re]
        go = oracle.gradient(3, p, nel, g, Gz, Hz)
        assert rel_max(gpu_grad(3, p, nel, g, G, H, rb=rb, re=re), go) <= FP64_TOL, f"{rb}:{re}"
    # no weight, or an empty range: zero
    assert not np.any(gpu_grad(3, p, nel, g, None, None))
    assert not np.any(gpu_grad(3, p, nel, g, G, H, rb=5, re=5))


def test_out_of_range_band_entries_are_ignored():
    # the forward map never writes band entries whose column lies outside
    # the mesh, so weights placed there must not reach the gradient
    p, nel = 2, (9, 8, 7)
    g, _ = inputs.make(3, p, nel, 0.05, "one")
    rng = np.random.default_rng(3)
    rows, band = int(np.prod([v + p for v in nel])), (2 * p + 1) ** 3
    G = rng.standard_normal((rows, band))
    H = rng.standard_normal((rows, band))
    mask = inputs.band_mask(nel, p)
    full = gpu_grad(3, p, nel, g, G, H)
    masked = gpu_grad(3, p, nel, g, G * mask, H * mask)
    assert rel_max(full, masked) <= 1e-14


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_euler_identity(prec):
    # J is linear in C: <dJ/dC, C> = J(C), J from the forward assembly
    p, nel = 3, (30, 17, 12)
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=2)
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    M, K = wq.assemble(R, gd, cd, prec)
    gen = torch.Generator(device="cuda").manual_seed(5)
    G = torch.randn(M.shape, dtype=torch.float64, device="cuda", generator=gen)
    H = torch.randn(M.shape, dtype=torch.float64, device="cuda", generator=gen)
    J = (G * K).sum() + (H * M).sum()
    grad = wq.assemble_adjoint(R, gd, G, H, prec)
    scale = (G * K).abs().sum() + (H * M).abs().sum()
    assert abs(torch.dot(grad, cd).item() - J.item()) <= 1e-13 * scale.item()
    R.close()


def test_autograd_function():
    p, nel = 2, (11, 10, 9)
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=4)
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda().requires_grad_(True)
    M, K = wq.assemble_differentiable(R, gd, cd, "fp64")
    gen = torch.Generator(device="cuda").manual_seed(6)
    G = torch.randn(M.shape, dtype=torch.float64, device="cuda", generator=gen)
    H = torch.randn(M.shape, dtype=torch.float64, device="cuda", generator=gen)
    ((G * K).sum() + (H * M).sum()).backward()
    ref = wq.assemble_adjoint(R, gd, G, H, "fp64")
    assert torch.allclose(cd.grad, ref, rtol=1e-13, atol=1e-13 * ref.abs().max().item())
    # only one matrix used: the other's incoming gradient is zero
    cd.grad = None
    M, K = wq.assemble_differentiable(R, gd, cd, "fp64")
    (G * K).sum().backward()
    ref = wq.assemble_adjoint(R, gd, G, None, "fp64")
    assert torch.allclose(cd.grad, ref, rtol=1e-13, atol=1e-13 * ref.abs().max().item())
    R.close()


def test_autograd_gradcheck_tiny():
    p, nel = 2, (2, 2, 1)
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=7)
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: wq.assemble_differentiable(R, gd, x, "fp64"), (cd,),
                                    eps=1e-6, atol=1e-9, rtol=1e-7)
    R.close()


def test_finite_differences_96():
    # central differences of J along 64 random directions, h = 1e-6, on the
    # 96^3 cubic workload (99^3 coefficients)
    w, g, c = inputs.workload("3d_p3_96")
    p, nel = w["p"], w["nel"]
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    gen = torch.Generator(device="cuda").manual_seed(96)
    shape = (R.rows, R.band)
    G = torch.randn(shape, dtype=torch.float64, device="cuda", generator=gen)
    H = torch.randn(shape, dtype=torch.float64, device="cuda", generator=gen)
    grad = wq.assemble_adjoint(R, gd, G, H, "fp64")
    M = torch.empty(shape, dtype=torch.float64, device="cuda")
    K = torch.empty_like(M)

    def J(x):
        wq.assemble(R, gd, x, "fp64", out=(M, K))
        return (G * K).sum().item() + (H * M).sum().item()

    h = 1e-6
    worst = 0.0
    for _ in range(64):
        d = torch.randn(R.ncoef, dtype=torch.float64, device="cuda", generator=gen)
        fd = (J(cd + h * d) - J(cd - h * d)) / (2 * h)
        ad = torch.dot(grad, d).item()
        worst = max(worst, abs(fd - ad) / abs(ad))
    assert worst <= 1e-6, f"worst relative FD mismatch {worst:.3e}"
    # the df64 gradient agrees with the FP64 one
    g64 = wq.assemble_adjoint(R, gd, G, H, "df64")
    assert (g64 - grad).abs().max().item() <= FP64_TOL * grad.abs().max().item()
    R.close()


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_gradient_is_bitwise_repeatable(prec):
    # the chunk blocks are summed in a fixed order: calls on the same inputs
    # give the same bits, over the whole mesh and over a row range whose
    # first and last lines are cut
    p, nel = 3, (23, 9, 8)
    g, _ = inputs.make(3, p, nel, 0.05, "one")
    R = wq.Rules(3, p, nel)
    dt = torch.float32 if prec == "mixed" else torch.float64
    gd = [torch.from_numpy(x).cuda() for x in g]
    gen = torch.Generator(device="cuda").manual_seed(3)
    G = torch.randn((R.rows, R.band), dtype=dt, device="cuda", generator=gen)
    H = torch.randn((R.rows, R.band), dtype=dt, device="cuda", generator=gen)
    for rb, re in ((0, R.rows), (37, R.rows - 101)):
        first = wq.assemble_adjoint(R, gd, G[rb:re].contiguous(), H[rb:re].contiguous(), prec, rb, re)
        for _ in range(3):
            again = wq.assemble_adjoint(R, gd, G[rb:re].contiguous(), H[rb:re].contiguous(), prec, rb, re)
            assert torch.equal(first, again)
    # the row-range gradients add up to the whole mesh's (up to rounding)
    full = wq.assemble_adjoint(R, gd, G, H, prec)
    cut = R.rows // 3
    a = wq.assemble_adjoint(R, gd, G[:cut].contiguous(), H[:cut].contiguous(), prec, 0, cut)
    b = wq.assemble_adjoint(R, gd, G[cut:].contiguous(), H[cut:].contiguous(), prec, cut, R.rows)
    tol = MIXED_TOL if prec == "mixed" else FP64_TOL
    assert rel_max((a + b).cpu().numpy(), full.cpu().numpy()) <= tol
    R.close()
