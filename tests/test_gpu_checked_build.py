"""The checked build (-DWQ_CHECKED=1): compute-sanitizer is not available to
this project's tests, so the library can be built with range checks on its
guarded global accesses (band and partial-contraction writes and reads, the
adjoint's chunk blocks, the non-separable path's factors and bands); a failed
check sets a status bit that wq_status_check reports as WQ_ERR_CHECK and the
access is skipped, never trapping.

The checked library is built into a temporary directory and loaded by a child
process (WQ_LIBRARY), which runs the assembly (3D and 2D, every precision, a
row range), the matrix-free apply, the adjoint, a batch, the no-alloc entry
point and the non-separable assembly; every call must report WQ_OK (no check
fired) and give the same bits as the default build in this process."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import build as wqbuild
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
from paper_1710_01048_gb300 import binding as wq, inputs
out = {}

def run(tag, fn):
    r = fn()
    s = wq.wq_status_check(keep[-1].handle, wq._stream_handle(None))
    out["status_" + tag] = np.array([s])
    for i, t in enumerate(r):
        if t is not None:
            out[tag + "_" + str(i)] = t.double().cpu().numpy()

keep = []
for dim, p, nel in ((3, 3, (13, 7, 9)), (2, 2, (9, 7))):
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=5)
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    R = wq.Rules(dim, p, nel)
    keep.append(R)
    for prec in ("fp64", "df64", "mixed"):
        run(f"asm{dim}_{prec}", lambda: wq.assemble(R, gd, cd, prec, check=False))
    run(f"rng{dim}", lambda: wq.assemble(R, gd, cd, "fp64", row_begin=R.rows // 3, row_end=R.rows - 5, check=False))
    x = torch.linspace(-1.0, 1.0, R.rows, dtype=torch.float64, device="cuda")
    run(f"apply{dim}", lambda: wq.apply(R, gd, x, cd, "fp64", check=False))
    Gw = torch.linspace(-1.0, 1.0, R.rows * R.band, dtype=torch.float64, device="cuda").reshape(R.rows, R.band)
    run(f"adj{dim}", lambda: (wq.assemble_adjoint(R, gd, Gw, Gw.flip(0).contiguous(), "fp64", check=False),))
    if dim == 3:
        net, cn = inputs.make_net(3, p, nel, "warp", 0.05, "exp", 0.1, seed=5)
        nd, cnd = torch.from_numpy(net).cuda(), torch.from_numpy(cn).cuda()
        for prec in ("fp64", "mixed"):
            run(f"gen_{prec}", lambda: wq.assemble_general(R, nd, cnd, prec, check=False))
        Mb = torch.empty((R.rows, R.band), dtype=torch.float64, device="cuda")
        Kb = torch.empty_like(Mb)
        B = wq.Batch([(R, gd, cd, Mb, Kb)], "fp64")
        B.launch()
        out["status_batch"] = np.array([B.status()])
        out["batch_0"] = Mb.cpu().numpy()
        out["batch_1"] = Kb.cpu().numpy()
        B.close()
        Rh = wq.Rules(dim, p, nel, device=False)
        Mn = torch.empty_like(Mb)
        Kn = torch.empty_like(Mb)
        st = wq.wq_assemble_noalloc(Rh.handle, [t.data_ptr() for t in gd], ctypes.c_void_p(cd.data_ptr()), wq.WQ_FP64,
                                    ctypes.c_void_p(Mn.data_ptr()), ctypes.c_void_p(Kn.data_ptr()), 0, Rh.rows,
                                    wq._stream_handle(None), 1)
        out["status_noalloc"] = np.array([st])
        out["noalloc_0"] = Mn.cpu().numpy()
        out["noalloc_1"] = Kn.cpu().numpy()
        Rh.close()
np.savez(OUT, **out)
'''


def test_checked_build_reports_no_violation_and_changes_no_bits(tmp_path):
    lib = wqbuild.build(out_dir=str(tmp_path / "checked"), extra_nvcc=["-DWQ_CHECKED=1"])
    script = tmp_path / "child.py"
    outf = tmp_path / "out.npz"
    script.write_text(f"ROOT = {ROOT!r}\nOUT = {str(outf)!r}\n" + CHILD)
    env = dict(os.environ, WQ_LIBRARY=lib)
    r = subprocess.run([sys.executable, str(script)], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout + r.stderr
    got = np.load(outf)
    statuses = {k: int(got[k][0]) for k in got.files if k.startswith("status_")}
    assert all(v == wq.WQ_OK for v in statuses.values()), statuses
    # the same calls through the default build in this process
    assert os.path.abspath(wq.LIB_PATH) != os.path.abspath(lib)
    for dim, p, nel in ((3, 3, (13, 7, 9)), (2, 2, (9, 7))):
        g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=5)
        gd = [torch.from_numpy(x).cuda() for x in g]
        cd = torch.from_numpy(c).cuda()
        R = wq.Rules(dim, p, nel)
        ref = {}
        for prec in ("fp64", "df64", "mixed"):
            ref[f"asm{dim}_{prec}"] = wq.assemble(R, gd, cd, prec)
        ref[f"rng{dim}"] = wq.assemble(R, gd, cd, "fp64", row_begin=R.rows // 3, row_end=R.rows - 5)
        x = torch.linspace(-1.0, 1.0, R.rows, dtype=torch.float64, device="cuda")
        ref[f"apply{dim}"] = wq.apply(R, gd, x, cd, "fp64")
        Gw = torch.linspace(-1.0, 1.0, R.rows * R.band, dtype=torch.float64, device="cuda").reshape(R.rows, R.band)
        ref[f"adj{dim}"] = (wq.assemble_adjoint(R, gd, Gw, Gw.flip(0).contiguous(), "fp64"),)
        if dim == 3:
            net, cn = inputs.make_net(3, p, nel, "warp", 0.05, "exp", 0.1, seed=5)
            nd, cnd = torch.from_numpy(net).cuda(), torch.from_numpy(cn).cuda()
            for prec in ("fp64", "mixed"):
                ref[f"gen_{prec}"] = wq.assemble_general(R, nd, cnd, prec)
            Mb = torch.empty((R.rows, R.band), dtype=torch.float64, device="cuda")
            Kb = torch.empty_like(Mb)
            B = wq.Batch([(R, gd, cd, Mb, Kb)], "fp64")
            B.launch()
            B.check()
            B.close()
            ref["batch"] = (Mb, Kb)
            Rh = wq.Rules(dim, p, nel, device=False)
            Mn = torch.empty_like(Mb)
            Kn = torch.empty_like(Mb)
            st = wq.wq_assemble_noalloc(Rh.handle, [t.data_ptr() for t in gd], ctypes.c_void_p(cd.data_ptr()),
                                        wq.WQ_FP64, ctypes.c_void_p(Mn.data_ptr()), ctypes.c_void_p(Kn.data_ptr()), 0,
                                        Rh.rows, wq._stream_handle(None), 1)
            assert st == wq.WQ_OK
            Rh.close()
            ref["noalloc"] = (Mn, Kn)
        for tag, ts in ref.items():
            for i, t in enumerate(ts):
                if t is None:
                    continue
                a = got[f"{tag}_{i}"]
                assert np.array_equal(a, t.double().cpu().numpy()), tag
        R.close()
