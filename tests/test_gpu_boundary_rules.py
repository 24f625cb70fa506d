"""Assembly with weighted Gaussian rules on the boundary rows too
(WQ_RULES_BOUNDARY_WEIGHTED) against the oracle's 'wqb' mode, through the
C-ABI: FP64 and double-float <= 1e-12, FP32 <= 1e-6 per matrix (max-entry and
Frobenius).  Meshes mix directions with at least 2p+1 elements (boundary rows
on their own rules) and fewer (Gauss-Legendre kept), ragged chunk tails and
row ranges; the entry points that do not take these rules refuse them."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df64": 1e-12, "mixed": 1e-6}


def check(A, O, tol, what):
    d = A.double().cpu().numpy() - O
    em = np.max(np.abs(d)) / np.max(np.abs(O))
    ef = np.linalg.norm(d) / np.linalg.norm(O)
    assert em <= tol and ef <= tol, f"{what}: rel_max {em:.3e} rel_fro {ef:.3e}"


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
@pytest.mark.parametrize("dim,p,nel", [(3, 3, (41, 9, 7)), (3, 2, (11, 5, 6)), (3, 3, (7, 3, 8)), (2, 3, (33, 12)),
                                       (2, 2, (9, 4)), (3, 3, (2, 3, 1))])
def test_boundary_weighted_parity(dim, p, nel, prec):
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=51)
    R = wq.Rules(dim, p, nel, rule="wqb")
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    M, K = wq.assemble(R, gd, cd, prec)
    Mo, Ko = oracle.assemble_rule("wqb", dim, p, nel, g, c)
    check(M, Mo, TOL[prec], f"M {prec}")
    check(K, Ko, TOL[prec], f"K {prec}")
    R.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_boundary_weighted_row_ranges_and_single_matrices(prec):
    p, nel = 3, (23, 8, 9)
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=52)
    R = wq.Rules(3, p, nel, rule="wqb")
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    M, K = wq.assemble(R, gd, cd, prec)
    rng = np.random.default_rng(5)
    for _ in range(4):
        rb = int(rng.integers(0, R.rows))
        re = int(rng.integers(rb + 1, R.rows + 1))
        Mr, _ = wq.assemble(R, gd, cd, prec, True, False, rb, re)
        _, Kr = wq.assemble(R, gd, cd, prec, False, True, rb, re)
        assert torch.equal(Mr, M[rb:re]) and torch.equal(Kr, K[rb:re])
    R.close()


def test_boundary_weighted_exact_on_affine_maps():
    # c = 1, identity map: every rule is exact, the bands are the exact
    # integrals -- and equal those of the default rules
    p, nel = 3, (9, 10, 8)
    g, _ = inputs.make(3, p, nel, 0.0, "one")
    gd = [torch.from_numpy(x).cuda() for x in g]
    Rb = wq.Rules(3, p, nel, rule="wqb")
    R = wq.Rules(3, p, nel)
    Mb, Kb = wq.assemble(Rb, gd, None, "fp64")
    M, K = wq.assemble(R, gd, None, "fp64")
    for A, B in ((Mb, M), (Kb, K)):
        assert (A - B).abs().max().item() <= 1e-13 * B.abs().max().item()
    Rb.close()
    R.close()


def test_entry_points_that_refuse_boundary_weighted_rules():
    p, nel = 3, (8, 7, 7)
    g, c = inputs.make(3, p, nel, 0.05, "exp", 0.1, seed=53)
    R = wq.Rules(3, p, nel, rule="wqb")
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    s = wq._stream_handle(None)
    x = torch.ones(R.rows, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    G = torch.zeros((R.rows, R.band), dtype=torch.float64, device="cuda")
    grad = torch.empty(R.ncoef, dtype=torch.float64, device="cuda")
    gp = [t.data_ptr() for t in gd]
    assert wq.wq_apply_mass_stiffness(R.handle, gp, ctypes.c_void_p(cd.data_ptr()), wq.WQ_FP64,
                                      ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), None, 0, R.rows,
                                      s) == wq.WQ_ERR_UNSUPPORTED
    assert wq.wq_assemble_adjoint(R.handle, gp, wq.WQ_FP64, ctypes.c_void_p(G.data_ptr()), None,
                                  ctypes.c_void_p(grad.data_ptr()), 0, R.rows, s) == wq.WQ_ERR_UNSUPPORTED
    M = torch.empty((R.rows, R.band), dtype=torch.float64, device="cuda")
    Rh = wq.Rules(3, p, nel, device=False, rule="wqb")
    assert wq.wq_assemble_noalloc(Rh.handle, gp, ctypes.c_void_p(cd.data_ptr()), wq.WQ_FP64,
                                  ctypes.c_void_p(M.data_ptr()), None, 0, R.rows, s, 1) == wq.WQ_ERR_UNSUPPORTED
    with pytest.raises(wq.WqError) as ei:
        wq.Batch([(R, gd, cd, M, torch.empty_like(M))], "fp64")
    assert ei.value.status == wq.WQ_ERR_UNSUPPORTED
    Rh.close()
    R.close()
