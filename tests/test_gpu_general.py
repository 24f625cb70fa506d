"""Assembly for maps given by a full control net (wq_assemble_general)
against the oracle's wqo_assemble_general, through the C-ABI: FP64 within
1e-12 per matrix (max-entry and Frobenius, relative to the oracle's), on
warped non-separable maps in 2D and 3D, p = 2 and 3, meshes with ragged
chunk tails and with no interior row; exactness on sheared affine maps
against the element-wise Gauss-Legendre integrals; a separable net against
the separable assembly; row ranges, single matrices and the slab loop
bitwise; the status word and the refused arguments."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
TOL32 = 1e-6


def check(A, O, tol, what):
    d = A.double().cpu().numpy() - O
    em = np.max(np.abs(d)) / np.max(np.abs(O))
    ef = np.linalg.norm(d) / np.linalg.norm(O)
    assert em <= tol and ef <= tol, f"{what}: rel_max {em:.3e} rel_fro {ef:.3e}"


def dev(x):
    return torch.from_numpy(x).cuda()


@pytest.mark.parametrize("dim,p,nel", [(3, 3, (19, 9, 7)), (3, 2, (11, 5, 6)), (3, 3, (2, 3, 1)), (3, 2, (1, 1, 1)),
                                       (3, 3, (140, 4, 3)), (2, 3, (33, 12)), (2, 2, (9, 4)), (2, 3, (1, 2)),
                                       (2, 2, (131, 5))])
def test_general_parity_warped(dim, p, nel):
    net, c = inputs.make_net(dim, p, nel, "warp", 0.05, "exp", 0.1, seed=61)
    R = wq.Rules(dim, p, nel)
    M, K = wq.assemble_general(R, dev(net), dev(c))
    Mo, Ko = oracle.assemble_general(dim, p, nel, net, c)
    check(M, Mo, TOL, "M")
    check(K, Ko, TOL, "K")
    R.close()


@pytest.mark.parametrize("dim,p,nel", [(3, 3, (19, 9, 7)), (3, 2, (11, 5, 6)), (3, 3, (2, 3, 1)), (3, 2, (1, 1, 1)),
                                       (3, 3, (140, 4, 3)), (2, 3, (33, 12)), (2, 2, (9, 4)), (2, 3, (1, 2)),
                                       (2, 2, (131, 5))])
def test_general_parity_warped_fp32(dim, p, nel):
    net, c = inputs.make_net(dim, p, nel, "warp", 0.05, "exp", 0.1, seed=61)
    R = wq.Rules(dim, p, nel)
    M, K = wq.assemble_general(R, dev(net), dev(c), prec="mixed")
    assert M.dtype == torch.float32 and K.dtype == torch.float32
    Mo, Ko = oracle.assemble_general(dim, p, nel, net, c)
    check(M, Mo, TOL32, "M")
    check(K, Ko, TOL32, "K")
    # the slab loop and row ranges give the same bits in FP32 too
    Mr, Kr = wq.assemble_general(R, dev(net), dev(c), prec="mixed", row_begin=R.rows // 3, row_end=R.rows - 1)
    assert torch.equal(Mr, M[R.rows // 3:R.rows - 1]) and torch.equal(Kr, K[R.rows // 3:R.rows - 1])
    R.close()


def test_general_fp32_accuracy_at_64_cubed_sampled():
    dim, p, nel = 3, 3, (64, 64, 64)
    net, c = inputs.make_net(dim, p, nel, "warp", 0.05, "exp", 0.1, seed=0)
    R = wq.Rules(dim, p, nel)
    M, K = wq.assemble_general(R, dev(net), dev(c), prec="mixed")
    rng = np.random.default_rng(8)
    rows = sorted(set(rng.integers(0, R.rows, size=24).tolist()) | {0, R.rows - 1, R.rows // 2})
    Mh, Kh = M.double().cpu().numpy(), K.double().cpu().numpy()
    for r in rows:
        Mo, Ko = oracle.assemble_general(dim, p, nel, net, c, row_begin=r, row_end=r + 1)
        for A, O in ((Mh[r], Mo[0]), (Kh[r], Ko[0])):
            assert np.max(np.abs(A - O)) <= TOL32 * np.max(np.abs(O)), r
    R.close()


@pytest.mark.parametrize("dim,p,nel", [(3, 3, (9, 8, 10)), (3, 2, (6, 7, 5)), (2, 3, (12, 9)), (2, 2, (1, 3))])
def test_general_exact_on_sheared_affine_maps(dim, p, nel):
    net = inputs.full_net(p, nel, "affine")
    R = wq.Rules(dim, p, nel)
    M, K = wq.assemble_general(R, dev(net))
    Me, Ke = oracle.assemble_gl_net(dim, p, nel, net)
    check(M, Me, TOL, "M")
    check(K, Ke, TOL, "K")
    R.close()


@pytest.mark.parametrize("dim,p,nel", [(3, 3, (10, 7, 6)), (2, 2, (8, 11))])
def test_separable_net_matches_separable_assembly(dim, p, nel):
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=62)
    net = inputs.net_from_separable(p, nel, g)
    R = wq.Rules(dim, p, nel)
    M, K = wq.assemble_general(R, dev(net), dev(c))
    Ms, Ks = wq.assemble(R, [dev(x) for x in g], dev(c), "fp64")
    for A, B in ((M, Ms), (K, Ks)):
        assert (A - B).abs().max().item() <= 1e-13 * B.abs().max().item()
    R.close()


def test_row_ranges_single_matrices_and_slabs(monkeypatch):
    dim, p, nel = 3, 3, (13, 7, 9)
    net, c = inputs.make_net(dim, p, nel, "warp", 0.05, "exp", 0.1, seed=63)
    R = wq.Rules(dim, p, nel)
    nd, cd = dev(net), dev(c)
    M, K = wq.assemble_general(R, nd, cd)
    rng = np.random.default_rng(3)
    for _ in range(4):
        rb = int(rng.integers(0, R.rows))
        re = int(rng.integers(rb + 1, R.rows + 1))
        Mr, _ = wq.assemble_general(R, nd, cd, stiffness=False, row_begin=rb, row_end=re)
        _, Kr = wq.assemble_general(R, nd, cd, mass=False, row_begin=rb, row_end=re)
        assert torch.equal(Mr, M[rb:re]) and torch.equal(Kr, K[rb:re])
    # one x3 plane per slab: the same bits
    monkeypatch.setenv("WQ_GENERAL_SLAB_BYTES", "1")
    R2 = wq.Rules(dim, p, nel)
    M2, K2 = wq.assemble_general(R2, nd, cd)
    assert torch.equal(M2, M) and torch.equal(K2, K)
    M3, K3 = wq.assemble_general(R2, nd, cd, row_begin=100, row_end=R.rows - 77)
    assert torch.equal(M3, M[100:R.rows - 77]) and torch.equal(K3, K[100:R.rows - 77])
    R2.close()
    R.close()


def test_sampled_rows_at_64_cubed():
    dim, p, nel = 3, 3, (64, 64, 64)
    net, c = inputs.make_net(dim, p, nel, "warp", 0.05, "exp", 0.1, seed=0)
    R = wq.Rules(dim, p, nel)
    M, K = wq.assemble_general(R, dev(net), dev(c))
    rng = np.random.default_rng(7)
    rows = sorted(set(rng.integers(0, R.rows, size=24).tolist()) | {0, R.rows - 1, R.rows // 2})
    Mh, Kh = M.cpu().numpy(), K.cpu().numpy()
    for r in rows:
        Mo, Ko = oracle.assemble_general(dim, p, nel, net, c, row_begin=r, row_end=r + 1)
        for A, O in ((Mh[r], Mo[0]), (Kh[r], Ko[0])):
            assert np.max(np.abs(A - O)) <= TOL * np.max(np.abs(O)), r
    R.close()


def test_status_and_refusals():
    dim, p, nel = 3, 2, (5, 4, 6)
    net = inputs.full_net(p, nel, "affine")
    R = wq.Rules(dim, p, nel)
    # a mirrored map: det J < 0 everywhere -> WQ_ERR_GEOMETRY, bands with |det J|
    flipped = net.copy()
    n = int(np.prod([nel[a] + p for a in range(dim)]))
    flipped[:n] = -flipped[:n]
    with pytest.raises(wq.WqError) as ei:
        wq.assemble_general(R, dev(flipped))
    assert ei.value.status == wq.WQ_ERR_GEOMETRY
    with pytest.raises(wq.WqError) as ei:
        wq.assemble_general(R, dev(flipped), prec="mixed")
    assert ei.value.status == wq.WQ_ERR_GEOMETRY
    M, K = wq.assemble_general(R, dev(flipped), check=False)
    assert wq.wq_status_check(R.handle, wq._stream_handle(None)) == wq.WQ_ERR_GEOMETRY
    Mo, Ko = wq.assemble_general(R, dev(net))
    assert (M - Mo).abs().max().item() <= 1e-13 * Mo.abs().max().item()
    bad = net.copy()
    bad[7] = np.nan
    with pytest.raises(wq.WqError) as ei:
        wq.assemble_general(R, dev(bad))
    assert ei.value.status == wq.WQ_ERR_NONFINITE
    s = wq._stream_handle(None)
    out = torch.empty((R.rows, R.band), dtype=torch.float64, device="cuda")
    lib = wq.library()
    nd = dev(net)
    for prec in (wq.WQ_DF64,):
        assert lib.wq_assemble_general(R.handle, ctypes.c_void_p(nd.data_ptr()), None, prec,
                                       ctypes.c_void_p(out.data_ptr()), None, 0, R.rows, s) == wq.WQ_ERR_UNSUPPORTED
    assert lib.wq_assemble_general(R.handle, None, None, wq.WQ_FP64, ctypes.c_void_p(out.data_ptr()), None, 0,
                                   R.rows, s) == wq.WQ_ERR_ARG
    assert lib.wq_assemble_general(R.handle, ctypes.c_void_p(nd.data_ptr()), None, wq.WQ_FP64, None, None, 0,
                                   R.rows, s) == wq.WQ_ERR_ARG
    assert lib.wq_assemble_general(R.handle, ctypes.c_void_p(nd.data_ptr()), None, wq.WQ_FP64,
                                   ctypes.c_void_p(out.data_ptr()), None, 0, R.rows + 1, s) == wq.WQ_ERR_ARG
    assert lib.wq_assemble_general(R.handle, ctypes.c_void_p(nd.data_ptr()), None, wq.WQ_FP64, None, None, 5, 5,
                                   s) == wq.WQ_OK
    for rule in ("gl", "nc", "wqb"):
        Rx = wq.Rules(dim, p, nel, rule=rule)
        assert lib.wq_assemble_general(Rx.handle, ctypes.c_void_p(nd.data_ptr()), None, wq.WQ_FP64,
                                       ctypes.c_void_p(out.data_ptr()), None, 0, R.rows, s) == wq.WQ_ERR_UNSUPPORTED
        Rx.close()
    R.close()
