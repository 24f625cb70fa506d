"""Guard bands around the outputs (a stand-in for a device memory checker).

Every assembly writes exactly the band rows of its range: the output buffers
are embedded in larger ones filled with a sentinel, at offsets that also
break 16-byte alignment (the FP32 path's bulk copies then start and end
mid-granule), and after the call the sentinel must be intact on both sides
while the rows equal those of a whole-mesh assembly bit for bit."""
import ctypes

import numpy as np
import pytest

from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 1000  # entries of sentinel on each side (plus the offset below)
SENTINEL = -7.25e29


def _embedded(nrows, band, dt, shift):
    """A sentinel-filled buffer and the view at GUARD + shift entries."""
    buf = torch.full((2 * GUARD + 8 + nrows * band,), SENTINEL, dtype=dt, device="cuda")
    view = buf[GUARD + shift:GUARD + shift + nrows * band]
    return buf, view


def _guards_intact(buf, shift, n):
    pre = buf[:GUARD + shift]
    post = buf[GUARD + shift + n:]
    return bool((pre == SENTINEL).all()) and bool((post == SENTINEL).all())


MESHES = [(3, (6, 5, 7)), (3, (70, 4, 3)), (2, (37, 3, 5)), (3, (1, 2, 1)), (2, (3, 4, 5))]


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
@pytest.mark.parametrize("p,nel", MESHES)
def test_row_ranges_write_only_their_rows(p, nel, prec):
    g, c = inputs.make(3, p, nel, 0.04, "exp", 0.1, seed=11)
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    Mf, Kf = wq.assemble(R, gd, cd, prec)
    dt = Mf.dtype
    rng = np.random.default_rng(p * 1000 + nel[0])
    ranges = [(0, R.rows), (0, 1), (R.rows - 1, R.rows)]
    for _ in range(6):
        a = int(rng.integers(0, R.rows))
        b = int(rng.integers(a + 1, R.rows + 1))
        ranges.append((a, b))
    s = wq._stream_handle(None)
    for k, (rb, re) in enumerate(ranges):
        n = (re - rb) * R.band
        sm, sk = k % 4, (k + 1) % 4  # offsets in entries: M and K differently misaligned
        bm, vm = _embedded(re - rb, R.band, dt, sm)
        bk, vk = _embedded(re - rb, R.band, dt, sk)
        st = wq.wq_assemble_mass_stiffness(R.handle, [x.data_ptr() for x in gd], ctypes.c_void_p(cd.data_ptr()),
                                           wq.PRECISIONS[prec], ctypes.c_void_p(vm.data_ptr()),
                                           ctypes.c_void_p(vk.data_ptr()), rb, re, s)
        assert st == wq.WQ_OK
        assert wq.wq_status_check(R.handle, s) == wq.WQ_OK
        assert _guards_intact(bm, sm, n) and _guards_intact(bk, sk, n), (rb, re)
        assert torch.equal(vm.view(re - rb, R.band), Mf[rb:re]) and torch.equal(vk.view(re - rb, R.band), Kf[rb:re])
        # single-matrix calls write only their matrix's rows too
        bm.fill_(SENTINEL)
        st = wq.wq_assemble_mass(R.handle, [x.data_ptr() for x in gd], ctypes.c_void_p(cd.data_ptr()),
                                 wq.PRECISIONS[prec], ctypes.c_void_p(vm.data_ptr()), rb, re, s)
        assert st == wq.WQ_OK
        torch.cuda.synchronize()
        assert _guards_intact(bm, sm, n) and torch.equal(vm.view(re - rb, R.band), Mf[rb:re])
        bk.fill_(SENTINEL)
        st = wq.wq_assemble_stiffness(R.handle, [x.data_ptr() for x in gd], ctypes.c_void_p(cd.data_ptr()),
                                      wq.PRECISIONS[prec], ctypes.c_void_p(vk.data_ptr()), rb, re, s)
        assert st == wq.WQ_OK
        torch.cuda.synchronize()
        assert _guards_intact(bk, sk, n) and torch.equal(vk.view(re - rb, R.band), Kf[rb:re])
    R.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_apply_and_adjoint_write_only_their_outputs(prec):
    p, nel = 3, (9, 6, 5)
    g, c = inputs.make(3, p, nel, 0.04, "exp", 0.1, seed=12)
    R = wq.Rules(3, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    dt = torch.float32 if prec == "mixed" else torch.float64
    gen = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(R.rows, dtype=torch.float64, device="cuda", generator=gen).to(dt)
    yM, yK = wq.apply(R, gd, x, cd, prec)
    rb, re = 17, R.rows - 23
    b1, v1 = _embedded(re - rb, 1, dt, 1)
    b2, v2 = _embedded(re - rb, 1, dt, 3)
    s = wq._stream_handle(None)
    st = wq.wq_apply_mass_stiffness(R.handle, [t.data_ptr() for t in gd], ctypes.c_void_p(cd.data_ptr()),
                                    wq.PRECISIONS[prec], ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(v1.data_ptr()),
                                    ctypes.c_void_p(v2.data_ptr()), rb, re, s)
    assert st == wq.WQ_OK
    torch.cuda.synchronize()
    assert _guards_intact(b1, 1, re - rb) and _guards_intact(b2, 3, re - rb)
    assert torch.equal(v1, yM[rb:re]) and torch.equal(v2, yK[rb:re])
    # the adjoint overwrites exactly the coefficient gradient
    G = torch.randn((R.rows, R.band), dtype=dt, device="cuda", generator=gen)
    bg = torch.full((2 * GUARD + R.ncoef,), SENTINEL, dtype=torch.float64, device="cuda")
    grad = bg[GUARD:GUARD + R.ncoef]
    wq.assemble_adjoint(R, gd, G, None, prec, out=grad)
    assert bool((bg[:GUARD] == SENTINEL).all()) and bool((bg[GUARD + R.ncoef:] == SENTINEL).all())
    assert bool(torch.isfinite(grad).all())
    R.close()
