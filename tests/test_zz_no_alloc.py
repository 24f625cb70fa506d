"""wq_assemble_noalloc: assembly without any device allocation.

Some host applications cannot let a library call cudaMalloc: all of their
device memory is carved out of one pool or arena they manage themselves,
or allocating while they run is forbidden.  Such a caller cannot create the
device tables of a WQ_RULES_DEVICE rules object.  wq_assemble_noalloc
takes host-only rules instead and keeps its working tables in a fixed array
inside the library; the caller passes only the inputs and outputs.

These tests compare it, through the C ABI, with the ordinary entry point on
the same inputs, twice in a row and across meshes of different sizes (the
array keeps whatever the previous call left in it), on row sub-ranges, and
with the FP64 oracle directly; and check that a non-finite coefficient is
reported without leaving a stale status behind.  This file is named so that
pytest collects it last."""
import numpy as np
import pytest

import oracle
from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-6


def _ptr(t):
    import ctypes

    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _rel(A, B):
    d = (A.double() - B.double()).cpu().numpy()
    b = B.double().cpu().numpy()
    return np.max(np.abs(d)) / np.max(np.abs(b)), np.linalg.norm(d) / np.linalg.norm(b)


def _noalloc(Rh, gd, cd, prec, M, K, check=1, rb=0, re=None):
    code = wq.WQ_FP64 if prec == "fp64" else wq.WQ_MIXED
    return wq.wq_assemble_noalloc(Rh.handle, [g.data_ptr() for g in gd], _ptr(cd), code, _ptr(M), _ptr(K), rb,
                                  Rh.rows if re is None else re, wq._stream_handle(None), check)


CASES = [(3, 3, (13, 6, 5), "fp64"), (3, 2, (9, 7, 8), "fp64"), (2, 3, (17, 9), "fp64"), (3, 3, (11, 5, 6), "mixed"),
         (3, 3, (13, 6, 5), "fp64")]


def test_noalloc_matches_ordinary_entry_point_twice():
    torch.cuda.set_device(0)
    for dim, p, nel, prec in CASES:
        g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=7)
        gd = [torch.from_numpy(x).cuda() for x in g]
        cd = torch.from_numpy(c).cuda()
        Rd = wq.Rules(dim, p, nel)  # ordinary path: device tables
        Rh = wq.Rules(dim, p, nel, device=False)  # no-alloc path: host tables only
        Mref, Kref = wq.assemble(Rd, gd, cd, prec)
        tol = FP64_TOL if prec == "fp64" else MIXED_TOL
        for call in range(2):
            M = torch.full_like(Mref, float("nan"))
            K = torch.full_like(Kref, float("nan"))
            st = _noalloc(Rh, gd, cd, prec, M, K)
            assert st == wq.WQ_OK, wq.wq_status_string(st)
            for A, B, name in ((M, Mref, "M"), (K, Kref, "K")):
                em, ef = _rel(A, B)
                assert em <= tol and ef <= tol, f"{name} {nel} {prec} call {call}: {em:.2e} {ef:.2e}"
        # one matrix at a time
        M = torch.zeros_like(Mref)
        assert _noalloc(Rh, gd, cd, prec, M, None) == wq.WQ_OK
        assert _rel(M, Mref)[0] <= tol
        Rd.close()
        Rh.close()


def test_noalloc_status_and_size_limit():
    torch.cuda.set_device(0)
    p, nel = 2, (5, 4, 3)
    g, c = inputs.make(3, p, nel, 0.0, "one")
    Rh = wq.Rules(3, p, nel, device=False)
    cd = torch.from_numpy(c).cuda()
    M = torch.empty((Rh.rows, Rh.band), dtype=torch.float64, device="cuda")
    K = torch.empty_like(M)
    # a folded map is reported when the caller asks for the status ...
    gbad = [torch.from_numpy(x).cuda() for x in (g[0], g[1][::-1].copy(), g[2])]
    assert _noalloc(Rh, gbad, cd, "fp64", M, K) == wq.WQ_ERR_GEOMETRY
    # ... and the next call starts from a clean status
    gd = [torch.from_numpy(x).cuda() for x in g]
    assert _noalloc(Rh, gd, cd, "fp64", M, K) == wq.WQ_OK
    Rh.close()
    # tables beyond the fixed array are refused before any GPU work
    big = wq.Rules(3, 3, (4, 2100, 2100), device=False)
    st = wq.wq_assemble_noalloc(big.handle, [gd[0].data_ptr()] * 3, None, wq.WQ_FP64, _ptr(M), _ptr(K), 0, 10,
                                wq._stream_handle(None), 1)
    assert st == wq.WQ_ERR_UNSUPPORTED
    big.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_oracle(prec):
    # the bands against the FP64 oracle itself, every row of a mesh with
    # interior and boundary lines in every direction
    torch.cuda.set_device(0)
    for dim, p, nel in [(3, 3, (9, 7, 6)), (3, 2, (6, 5, 7)), (2, 3, (12, 10))]:
        g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=17)
        gd = [torch.from_numpy(x).cuda() for x in g]
        cd = torch.from_numpy(c).cuda()
        Rh = wq.Rules(dim, p, nel, device=False)
        dt = torch.float64 if prec == "fp64" else torch.float32
        M = torch.full((Rh.rows, Rh.band), float("nan"), dtype=dt, device="cuda")
        K = torch.full_like(M, float("nan"))
        assert _noalloc(Rh, gd, cd, prec, M, K) == wq.WQ_OK
        Mo, Ko, _ = oracle.assemble(dim, p, nel, g, c)
        tol = FP64_TOL if prec == "fp64" else MIXED_TOL
        for A, O, name in ((M, Mo, "M"), (K, Ko, "K")):
            em, ef = _rel(A, torch.from_numpy(O).cuda())
            assert em <= tol and ef <= tol, f"{name} {nel} {prec}: {em:.2e} {ef:.2e}"
        Rh.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_row_subranges(prec):
    # rows [rb, re) (the line selection and its offset into the line lists
    # held in the array) equal the same rows of the ordinary entry point
    torch.cuda.set_device(0)
    dim, p, nel = 3, 3, (11, 6, 7)
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=19)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    Rd = wq.Rules(dim, p, nel)
    Rh = wq.Rules(dim, p, nel, device=False)
    Mref, Kref = wq.assemble(Rd, gd, cd, prec)
    tol = FP64_TOL if prec == "fp64" else MIXED_TOL
    rng = np.random.default_rng(23)
    for _ in range(6):
        rb = int(rng.integers(0, Rh.rows))
        re = int(rng.integers(rb + 1, Rh.rows + 1))
        M = torch.full((re - rb, Rh.band), float("nan"), dtype=Mref.dtype, device="cuda")
        K = torch.full_like(M, float("nan"))
        assert _noalloc(Rh, gd, cd, prec, M, K, rb=rb, re=re) == wq.WQ_OK
        for A, B, name in ((M, Mref[rb:re], "M"), (K, Kref[rb:re], "K")):
            em, ef = _rel(A, B)
            assert em <= tol and ef <= tol, f"{name} rows {rb}:{re} {prec}: {em:.2e} {ef:.2e}"
    Rd.close()
    Rh.close()


def test_noalloc_nonfinite_coefficient():
    # with no prepared coefficient copy the row kernel checks the
    # coefficients itself: a NaN is reported, and a clean call afterwards
    # returns WQ_OK
    torch.cuda.set_device(0)
    dim, p, nel = 3, 3, (6, 5, 4)
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=29)
    gd = [torch.from_numpy(x).cuda() for x in g]
    Rh = wq.Rules(dim, p, nel, device=False)
    cn = c.copy()
    cn[len(cn) // 2] = np.nan
    cbad = torch.from_numpy(cn).cuda()
    cd = torch.from_numpy(c).cuda()
    for prec in ("fp64", "mixed"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        M = torch.empty((Rh.rows, Rh.band), dtype=dt, device="cuda")
        K = torch.empty_like(M)
        assert _noalloc(Rh, gd, cbad, prec, M, K) == wq.WQ_ERR_NONFINITE
        assert _noalloc(Rh, gd, cd, prec, M, K) == wq.WQ_OK
    Rh.close()
