"""ctypes binding of libwq (``include/wq.h``).

The ``wq_*`` functions have the C names and signatures; they marshal
arguments and return the C status.  ``Rules`` and ``assemble`` are thin
conveniences over them that allocate outputs with torch (device memory and
the current stream only).  Every numerical step runs in libwq; there is no
fallback: if the library is not built, the first call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the in-tree build; WQ_LIBRARY may name another build of the same sources
# (e.g. the checked build, compiled with -DWQ_CHECKED=1)
LIB_PATH = os.environ.get("WQ_LIBRARY") or os.path.join(_HERE, "_build", "libwq.so")

WQ_OK, WQ_ERR_ARG, WQ_ERR_UNSUPPORTED, WQ_ERR_NO_CONVERGENCE = 0, 1, 2, 3
WQ_ERR_GEOMETRY, WQ_ERR_NONFINITE, WQ_ERR_CUDA, WQ_ERR_OOM, WQ_ERR_TIMEOUT, WQ_ERR_CHECK = 4, 5, 6, 7, 8, 9
WQ_FP64, WQ_MIXED, WQ_DF64 = 0, 1, 2
PRECISIONS = {"fp64": WQ_FP64, "mixed": WQ_MIXED, "df64": WQ_DF64}
WQ_KIND_MASS, WQ_KIND_STIFFNESS, WQ_KIND_MIXED_DW, WQ_KIND_MIXED_WD = 0, 1, 2, 3
WQ_RULES_HOST_ONLY, WQ_RULES_DEVICE, WQ_RULES_GAUSS_LEGENDRE, WQ_RULES_NEWTON_COTES = 0, 1, 2, 4
WQ_RULES_BOUNDARY_WEIGHTED = 8
RULE_FLAGS = {"wq": 0, "gl": WQ_RULES_GAUSS_LEGENDRE, "nc": WQ_RULES_NEWTON_COTES, "wqb": WQ_RULES_BOUNDARY_WEIGHTED}

# every function declared in include/wq.h
EXPORTS = ["wq_status_string", "wq_version", "wq_rule_1d", "wq_rule_1d_from", "wq_rules_build", "wq_rules_free",
           "wq_rules_row", "wq_rows", "wq_band_width", "wq_band_nnz", "wq_coef_count", "wq_flop_count",
           "wq_assemble_mass", "wq_assemble_stiffness", "wq_assemble_mass_stiffness", "wq_status_check",
           "wq_assemble_noalloc", "wq_assemble_adjoint", "wq_batch_create", "wq_batch_launch", "wq_batch_status",
           "wq_batch_get_config", "wq_batch_set_config", "wq_batch_tune", "wq_batch_free", "wq_assemble_batch", "wq_band_nnz_rows", "wq_band_to_csr",
           "wq_apply_mass_stiffness", "wq_assemble_load", "wq_assemble_mass_stiffness_host", "wq_rule_1d_mixed",
           "wq_assemble_general"]


class WqError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = _lib().wq_status_string(status).decode() if _loaded is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else f"{msg} (status {status})")


class wq_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("nel", ctypes.c_int * 3)]


class wq_patch(ctypes.Structure):
    _fields_ = [("rules", ctypes.c_void_p), ("geom", ctypes.c_void_p * 3), ("coef", ctypes.c_void_p),
                ("M", ctypes.c_void_p), ("K", ctypes.c_void_p)]


_loaded = None


def _lib():
    global _loaded
    if _loaded is not None:
        return _loaded
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libwq.so is not built ({LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    try:  # load torch's CUDA runtime first when torch is present, so both share it
        import torch  # noqa: F401
    except ImportError:
        pass
    lib = ctypes.CDLL(LIB_PATH)
    c_int, c_double, c_void_p, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64
    PD, PI = ctypes.POINTER(c_double), ctypes.POINTER(c_int)
    PP = ctypes.POINTER(c_void_p)
    lib.wq_status_string.argtypes = [c_int]
    lib.wq_status_string.restype = ctypes.c_char_p
    lib.wq_version.restype = c_int
    lib.wq_rule_1d.argtypes = [c_int, c_int, PD, PD]
    lib.wq_rule_1d_from.argtypes = [c_int, c_int, PD, PD, PD]
    lib.wq_rules_build.argtypes = [ctypes.POINTER(wq_mesh), c_int, ctypes.POINTER(c_void_p)]
    lib.wq_rules_free.argtypes = [c_void_p]
    lib.wq_rules_free.restype = None
    lib.wq_rules_row.argtypes = [c_void_p, c_int, c_int, c_int, PI, PD, PD, PI]
    for f in ("wq_rows", "wq_band_width", "wq_band_nnz", "wq_coef_count"):
        getattr(lib, f).argtypes = [c_void_p]
        getattr(lib, f).restype = i64
    lib.wq_flop_count.argtypes = [c_void_p, c_int, c_int, i64, i64, PD]
    lib.wq_flop_count.restype = c_double
    lib.wq_assemble_mass.argtypes = [c_void_p, PP, c_void_p, c_int, c_void_p, i64, i64, c_void_p]
    lib.wq_assemble_stiffness.argtypes = [c_void_p, PP, c_void_p, c_int, c_void_p, i64, i64, c_void_p]
    lib.wq_assemble_mass_stiffness.argtypes = [c_void_p, PP, c_void_p, c_int, c_void_p, c_void_p, i64, i64,
                                               c_void_p]
    lib.wq_apply_mass_stiffness.argtypes = [c_void_p, PP, c_void_p, c_int, c_void_p, c_void_p, c_void_p, i64, i64,
                                            c_void_p]
    lib.wq_assemble_load.argtypes = [c_void_p, PP, c_void_p, c_int, c_void_p, i64, i64, c_void_p]
    lib.wq_assemble_mass_stiffness_host.argtypes = [c_void_p, PP, c_void_p, c_int, c_void_p, c_void_p, PP, c_void_p,
                                                    c_void_p, c_void_p, i64, i64, c_int, c_void_p, c_void_p]
    lib.wq_status_check.argtypes = [c_void_p, c_void_p]
    lib.wq_rule_1d_mixed.argtypes = [c_int, PD, PD, PD]
    lib.wq_assemble_general.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, i64, i64, c_void_p]
    lib.wq_assemble_noalloc.argtypes = [c_void_p, PP, c_void_p, c_int, c_void_p, c_void_p, i64, i64, c_void_p, c_int]
    lib.wq_assemble_adjoint.argtypes = [c_void_p, PP, c_int, c_void_p, c_void_p, c_void_p, i64, i64, c_void_p]
    PPatch = ctypes.POINTER(wq_patch)
    lib.wq_batch_create.argtypes = [PPatch, c_int, c_int, ctypes.POINTER(c_void_p)]
    lib.wq_batch_launch.argtypes = [c_void_p, c_void_p]
    lib.wq_batch_status.argtypes = [c_void_p, c_void_p]
    lib.wq_batch_get_config.argtypes = [c_void_p, PI]
    lib.wq_batch_set_config.argtypes = [c_void_p, PI]
    lib.wq_batch_tune.argtypes = [c_void_p, c_void_p, c_int, PD]
    lib.wq_batch_free.argtypes = [c_void_p]
    lib.wq_batch_free.restype = None
    lib.wq_assemble_batch.argtypes = [PPatch, c_int, c_int, c_void_p]
    lib.wq_band_nnz_rows.argtypes = [c_void_p, i64, i64]
    lib.wq_band_nnz_rows.restype = i64
    lib.wq_band_to_csr.argtypes = [c_void_p, c_int, c_void_p, i64, i64, c_void_p, c_void_p, c_void_p, c_void_p]
    for f in EXPORTS:
        if f not in ("wq_status_string", "wq_version", "wq_rules_free", "wq_rows", "wq_band_width", "wq_band_nnz",
                     "wq_coef_count", "wq_flop_count", "wq_batch_free", "wq_band_nnz_rows"):
            getattr(lib, f).restype = c_int
    _loaded = lib
    return lib


def library():
    """The loaded ctypes library (loads it on first use)."""
    return _lib()


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st, what):
    if st != WQ_OK:
        raise WqError(st, what)


# ------------------------------------------------------------------ C names
def wq_status_string(status):
    return _lib().wq_status_string(status).decode()


def wq_version():
    return _lib().wq_version()


def wq_rule_1d(degree, kind):
    """(tau, omega) of the cardinal rule (numpy arrays)."""
    tau = np.zeros(degree + 1)
    om = np.zeros(degree + 1)
    _check(_lib().wq_rule_1d(degree, kind, _pd(tau), _pd(om)), "wq_rule_1d")
    return tau, om


def wq_rule_1d_mixed(degree):
    """(y, w, v) of the mixed-derivative rules (numpy arrays)."""
    y = np.zeros(degree + 1)
    w = np.zeros(degree + 1)
    v = np.zeros(degree + 1)
    _check(_lib().wq_rule_1d_mixed(degree, _pd(y), _pd(w), _pd(v)), "wq_rule_1d_mixed")
    return y, w, v


def wq_rule_1d_from(degree, kind, start):
    """(status, tau, omega) of a Newton solve from `start`."""
    s = np.ascontiguousarray(start, dtype=np.float64)
    tau = np.zeros(degree + 1)
    om = np.zeros(degree + 1)
    st = _lib().wq_rule_1d_from(degree, kind, _pd(s), _pd(tau), _pd(om))
    return st, tau, om


def wq_rules_build(dim, degree, nel, flags=WQ_RULES_DEVICE):
    """Raw handle (int) of a new wq_rules; release with wq_rules_free."""
    m = wq_mesh(dim, degree, (ctypes.c_int * 3)(*(list(nel) + [1] * (3 - len(nel)))))
    h = ctypes.c_void_p()
    _check(_lib().wq_rules_build(ctypes.byref(m), flags, ctypes.byref(h)), "wq_rules_build")
    return h.value


def wq_rules_free(handle):
    _lib().wq_rules_free(handle)


def wq_rules_row(handle, dir, kind, row):
    """(x, W, elem) of one row's 1D rule."""
    n = ctypes.c_int(0)
    x = np.zeros(16)
    w = np.zeros(16)
    e = np.zeros(16, dtype=np.int32)
    _check(_lib().wq_rules_row(handle, dir, kind, row, ctypes.byref(n), _pd(x), _pd(w),
                               e.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "wq_rules_row")
    k = n.value
    return x[:k].copy(), w[:k].copy(), e[:k].copy()


def wq_rows(handle):
    return _lib().wq_rows(handle)


def wq_band_width(handle):
    return _lib().wq_band_width(handle)


def wq_band_nnz(handle):
    return _lib().wq_band_nnz(handle)


def wq_coef_count(handle):
    return _lib().wq_coef_count(handle)


def wq_flop_count(handle, want_m, want_k, row_begin, row_end):
    """(contraction flops, coefficient-evaluation flops)."""
    cf = ctypes.c_double(0.0)
    f = _lib().wq_flop_count(handle, int(want_m), int(want_k), int(row_begin), int(row_end), ctypes.byref(cf))
    return f, cf.value


def _geom_array(geom_ptrs):
    arr = (ctypes.c_void_p * 3)(*(list(geom_ptrs) + [None] * (3 - len(geom_ptrs))))
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def wq_assemble_mass(handle, geom_ptrs, coef_ptr, prec, M_ptr, row_begin, row_end, stream):
    g, keep = _geom_array(geom_ptrs)
    return _lib().wq_assemble_mass(handle, g, coef_ptr, prec, M_ptr, row_begin, row_end, stream)


def wq_assemble_stiffness(handle, geom_ptrs, coef_ptr, prec, K_ptr, row_begin, row_end, stream):
    g, keep = _geom_array(geom_ptrs)
    return _lib().wq_assemble_stiffness(handle, g, coef_ptr, prec, K_ptr, row_begin, row_end, stream)


def wq_assemble_mass_stiffness(handle, geom_ptrs, coef_ptr, prec, M_ptr, K_ptr, row_begin, row_end, stream):
    g, keep = _geom_array(geom_ptrs)
    return _lib().wq_assemble_mass_stiffness(handle, g, coef_ptr, prec, M_ptr, K_ptr, row_begin, row_end, stream)


def wq_apply_mass_stiffness(handle, geom_ptrs, coef_ptr, prec, x_ptr, yM_ptr, yK_ptr, row_begin, row_end, stream):
    g, keep = _geom_array(geom_ptrs)
    return _lib().wq_apply_mass_stiffness(handle, g, coef_ptr, prec, x_ptr, yM_ptr, yK_ptr, row_begin, row_end,
                                          stream)


def wq_assemble_load(handle, geom_ptrs, f_ptr, prec, b_ptr, row_begin, row_end, stream):
    g, keep = _geom_array(geom_ptrs)
    return _lib().wq_assemble_load(handle, g, f_ptr, prec, b_ptr, row_begin, row_end, stream)


def wq_status_check(handle, stream):
    return _lib().wq_status_check(handle, stream)


def wq_assemble_noalloc(handle, geom_ptrs, coef_ptr, prec, M_ptr, K_ptr, row_begin, row_end, stream, check_status):
    """The assembly entry point that allocates no device memory (see wq.h)."""
    g, keep = _geom_array(geom_ptrs)
    return _lib().wq_assemble_noalloc(handle, g, coef_ptr, prec, M_ptr, K_ptr, row_begin, row_end, stream,
                                      int(check_status))


def wq_assemble_adjoint(handle, geom_ptrs, prec, G_ptr, H_ptr, grad_ptr, row_begin, row_end, stream):
    g, keep = _geom_array(geom_ptrs)
    return _lib().wq_assemble_adjoint(handle, g, prec, G_ptr, H_ptr, grad_ptr, row_begin, row_end, stream)


# ------------------------------------------------------------------ conveniences
class Rules:
    """Owns a wq_rules handle (host tables, and device tables when device=True)."""

    def __init__(self, dim, degree, nel, device=True, rule="wq"):
        """rule: 'wq' (the weighted Gaussian rules, Gauss-Legendre on the
        boundary rows), 'wqb' (weighted Gaussian rules for the boundary rows
        too, where defined), or the comparison rules 'gl' (Gauss-Legendre on
        every element of each row's support) and 'nc' (Newton-Cotes-type
        weighted rules on the interior rows)."""
        self.dim, self.degree, self.nel = int(dim), int(degree), tuple(int(v) for v in nel)
        self.rule = rule
        flags = (WQ_RULES_DEVICE if device else WQ_RULES_HOST_ONLY) | RULE_FLAGS[rule]
        self.handle = wq_rules_build(self.dim, self.degree, self.nel, flags)

    def close(self):
        if getattr(self, "handle", None):
            wq_rules_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def rows(self):
        return wq_rows(self.handle)

    @property
    def band(self):
        return wq_band_width(self.handle)

    @property
    def nnz(self):
        return wq_band_nnz(self.handle)

    @property
    def ncoef(self):
        return wq_coef_count(self.handle)

    def row(self, dir, kind, r):
        return wq_rules_row(self.handle, dir, kind, r)

    def flops(self, mass=True, stiffness=True, row_begin=0, row_end=None):
        return wq_flop_count(self.handle, mass, stiffness, row_begin, self.rows if row_end is None else row_end)


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def assemble(rules, geom, coef=None, prec="fp64", mass=True, stiffness=True, row_begin=0, row_end=None, out=None,
             stream=None, check=True):
    """Assembles rows [row_begin, row_end) of M and/or K (band layout) on the
    current CUDA device.  geom: list of dim float64 CUDA tensors (control
    values); coef: float64 CUDA tensor of rules.ncoef values or None (c = 1).
    prec: 'fp64', 'df64' (double-float on the FP32 pipe, FP64 output) or
    'mixed' (FP32).  Returns (M, K) torch tensors of shape (rows, band),
    float64 for 'fp64' and 'df64', float32 for 'mixed'.  With check=True the stream is synchronised and a
    device-detected problem raises WqError."""
    import torch

    if row_end is None:
        row_end = rules.rows
    p = PRECISIONS[prec]
    dt = torch.float32 if p == WQ_MIXED else torch.float64
    nrows = row_end - row_begin
    for g in geom:
        assert g.is_cuda and g.dtype == torch.float64 and g.is_contiguous()
    if coef is not None:
        assert coef.is_cuda and coef.dtype == torch.float64 and coef.is_contiguous() and coef.numel() == rules.ncoef
    dev = geom[0].device
    if out is None:
        M = torch.empty((nrows, rules.band), dtype=dt, device=dev) if mass else None
        K = torch.empty((nrows, rules.band), dtype=dt, device=dev) if stiffness else None
    else:
        M, K = out
    s = _stream_handle(stream)
    gp = [g.data_ptr() for g in geom]
    cp = ctypes.c_void_p(coef.data_ptr()) if coef is not None else None
    if mass and stiffness:
        st = wq_assemble_mass_stiffness(rules.handle, gp, cp, p, ctypes.c_void_p(M.data_ptr()),
                                        ctypes.c_void_p(K.data_ptr()), row_begin, row_end, s)
    elif mass:
        st = wq_assemble_mass(rules.handle, gp, cp, p, ctypes.c_void_p(M.data_ptr()), row_begin, row_end, s)
    else:
        st = wq_assemble_stiffness(rules.handle, gp, cp, p, ctypes.c_void_p(K.data_ptr()), row_begin, row_end, s)
    _check(st, "wq_assemble")
    if check:
        _check(wq_status_check(rules.handle, s), "wq_status_check")
    return M, K


def assemble_general(rules, net, coef=None, prec="fp64", mass=True, stiffness=True, row_begin=0, row_end=None,
                     out=None, stream=None, check=True):
    """Rows [row_begin, row_end) of M and/or K for the map given by its full
    control net (wq_assemble_general).  net: float64 CUDA tensor of
    dim * prod(nel + p) values (component-major, x fastest); coef as for
    assemble(); prec 'fp64' (float64 bands) or 'mixed' (FP32, float32
    bands).  Returns (M, K), None for a matrix not asked for."""
    import torch

    if row_end is None:
        row_end = rules.rows
    p = PRECISIONS[prec]
    assert net.is_cuda and net.dtype == torch.float64 and net.is_contiguous()
    if coef is not None:
        assert coef.is_cuda and coef.dtype == torch.float64 and coef.is_contiguous() and coef.numel() == rules.ncoef
    nrows = row_end - row_begin
    dt = torch.float32 if p == WQ_MIXED else torch.float64
    if out is None:
        M = torch.empty((nrows, rules.band), dtype=dt, device=net.device) if mass else None
        K = torch.empty((nrows, rules.band), dtype=dt, device=net.device) if stiffness else None
    else:
        M, K = out
    s = _stream_handle(stream)
    st = _lib().wq_assemble_general(rules.handle, ctypes.c_void_p(net.data_ptr()),
                                    ctypes.c_void_p(coef.data_ptr()) if coef is not None else None, p,
                                    ctypes.c_void_p(M.data_ptr()) if M is not None else None,
                                    ctypes.c_void_p(K.data_ptr()) if K is not None else None, row_begin, row_end, s)
    _check(st, "wq_assemble_general")
    if check:
        _check(wq_status_check(rules.handle, s), "wq_status_check")
    return M, K


def apply(rules, geom, x, coef=None, prec="fp64", mass=True, stiffness=True, row_begin=0, row_end=None, out=None,
          stream=None, check=True):
    """Matrix-free y_M = M x and y_K = K x for rows [row_begin, row_end)
    (the band is never stored).  x: CUDA tensor of rules.rows values, float64
    for 'fp64'/'df64', float32 for 'mixed'.  Returns (yM, yK), None for a
    matrix not asked for; `out` = (yM, yK) tensors to write instead."""
    import torch

    if row_end is None:
        row_end = rules.rows
    p = PRECISIONS[prec]
    dt = torch.float32 if p == WQ_MIXED else torch.float64
    assert x.is_cuda and x.dtype == dt and x.is_contiguous() and x.numel() == rules.rows
    if coef is not None:
        assert coef.is_cuda and coef.dtype == torch.float64 and coef.is_contiguous() and coef.numel() == rules.ncoef
    n = row_end - row_begin
    if out is None:
        yM = torch.empty(n, dtype=dt, device=x.device) if mass else None
        yK = torch.empty(n, dtype=dt, device=x.device) if stiffness else None
    else:
        yM, yK = out
    s = _stream_handle(stream)
    gp = [g.data_ptr() for g in geom]
    cp = ctypes.c_void_p(coef.data_ptr()) if coef is not None else None
    st = wq_apply_mass_stiffness(rules.handle, gp, cp, p, ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(yM.data_ptr()) if yM is not None else None,
                                 ctypes.c_void_p(yK.data_ptr()) if yK is not None else None, row_begin, row_end, s)
    _check(st, "wq_apply_mass_stiffness")
    if check:
        _check(wq_status_check(rules.handle, s), "wq_status_check")
    return yM, yK


def assemble_load(rules, geom, f=None, prec="fp64", row_begin=0, row_end=None, out=None, stream=None, check=True):
    """Load vector b_r = integral of f B_r |det J| (Eq. Load) for rows
    [row_begin, row_end) with the weighted Gaussian mass rules; f: CUDA
    float64 tensor of rules.ncoef spline coefficients, or None for f = 1."""
    import torch

    if row_end is None:
        row_end = rules.rows
    p = PRECISIONS[prec]
    dt = torch.float32 if p == WQ_MIXED else torch.float64
    if f is not None:
        assert f.is_cuda and f.dtype == torch.float64 and f.is_contiguous() and f.numel() == rules.ncoef
    b = torch.empty(row_end - row_begin, dtype=dt, device=geom[0].device) if out is None else out
    s = _stream_handle(stream)
    gp = [g.data_ptr() for g in geom]
    fp = ctypes.c_void_p(f.data_ptr()) if f is not None else None
    _check(wq_assemble_load(rules.handle, gp, fp, p, ctypes.c_void_p(b.data_ptr()), row_begin, row_end, s),
           "wq_assemble_load")
    if check:
        _check(wq_status_check(rules.handle, s), "wq_status_check")
    return b


def assemble_adjoint(rules, geom, G=None, H=None, prec="fp64", row_begin=0, row_end=None, out=None, stream=None,
                     check=True):
    """Gradient of J(C) = sum G * K(C) + H * M(C) over rows [row_begin,
    row_end) with respect to the coefficient spline's C (the backward pass of
    assemble).  G, H: CUDA tensors of shape (rows in range, band), float64
    for 'fp64'/'df64', float32 for 'mixed', or None.  Returns a float64 CUDA
    tensor of rules.ncoef values (written into `out` if given)."""
    import torch

    if row_end is None:
        row_end = rules.rows
    p = PRECISIONS[prec]
    dt = torch.float32 if p == WQ_MIXED else torch.float64
    nrows = row_end - row_begin
    for g in geom:
        assert g.is_cuda and g.dtype == torch.float64 and g.is_contiguous()
    for X in (G, H):
        if X is not None:
            assert X.is_cuda and X.dtype == dt and X.is_contiguous() and tuple(X.shape) == (nrows, rules.band)
    grad = out if out is not None else torch.empty(rules.ncoef, dtype=torch.float64, device=geom[0].device)
    s = _stream_handle(stream)
    st = wq_assemble_adjoint(rules.handle, [g.data_ptr() for g in geom], p,
                             ctypes.c_void_p(G.data_ptr()) if G is not None else None,
                             ctypes.c_void_p(H.data_ptr()) if H is not None else None,
                             ctypes.c_void_p(grad.data_ptr()), row_begin, row_end, s)
    _check(st, "wq_assemble_adjoint")
    if check:
        _check(wq_status_check(rules.handle, s), "wq_status_check")
    return grad


def _autograd_function():
    import torch

    class _Assemble(torch.autograd.Function):
        @staticmethod
        def forward(ctx, coef, rules, geom, prec):
            M, K = assemble(rules, geom, coef, prec)
            ctx.rules, ctx.geom, ctx.prec = rules, geom, prec
            return M, K

        @staticmethod
        def backward(ctx, dM, dK):
            dt = torch.float32 if ctx.prec == "mixed" else torch.float64
            H = dM.to(dt).contiguous() if dM is not None else None
            G = dK.to(dt).contiguous() if dK is not None else None
            grad = assemble_adjoint(ctx.rules, ctx.geom, G, H, ctx.prec)
            return grad, None, None, None

    return _Assemble


_ASSEMBLE_FN = None


def assemble_differentiable(rules, geom, coef, prec="fp64"):
    """(M, K) = assemble(rules, geom, coef, prec) as a torch autograd
    operation of coef: backward calls wq_assemble_adjoint."""
    global _ASSEMBLE_FN
    if _ASSEMBLE_FN is None:
        _ASSEMBLE_FN = _autograd_function()
    return _ASSEMBLE_FN.apply(coef, rules, list(geom), prec)


# ------------------------------------------------------------------ batches
def _patch_array(patches):
    """patches: sequence of (rules, geom list of 3 CUDA tensors, coef tensor or None, M, K)."""
    arr = (wq_patch * len(patches))()
    for i, (rules, geom, coef, M, K) in enumerate(patches):
        arr[i].rules = rules.handle
        for a in range(3):
            arr[i].geom[a] = geom[a].data_ptr()
        arr[i].coef = coef.data_ptr() if coef is not None else None
        arr[i].M = M.data_ptr()
        arr[i].K = K.data_ptr()
    return arr


class Batch:
    """A batched-assembly plan (wq_batch): patches are tuples (rules, geom,
    coef, M, K) of Rules objects and CUDA tensors that must stay alive while
    the plan is used; launch() replays the plan's CUDA graph."""

    def __init__(self, patches, prec="fp64"):
        self._keep = list(patches)
        arr = _patch_array(self._keep)
        h = ctypes.c_void_p()
        _check(_lib().wq_batch_create(arr, len(self._keep), PRECISIONS[prec], ctypes.byref(h)), "wq_batch_create")
        self.handle = h
        self.prec = prec

    def launch(self, stream=None):
        _check(_lib().wq_batch_launch(self.handle, _stream_handle(stream)), "wq_batch_launch")

    def status(self, stream=None):
        return _lib().wq_batch_status(self.handle, _stream_handle(stream))

    def check(self, stream=None):
        _check(self.status(stream), "wq_batch_status")

    @property
    def config(self):
        c = (ctypes.c_int * 6)()
        _check(_lib().wq_batch_get_config(self.handle, c), "wq_batch_get_config")
        return dict(chunk=c[0], u_ctas_per_sm=c[1], ctas_per_sm=c[2], schedule=c[3], max_u_ctas_per_sm=c[4],
                    max_ctas_per_sm=c[5])

    def set_config(self, chunk, u_ctas_per_sm, ctas_per_sm, schedule):
        """schedule 0: the degree-2 kernels on a second stream beside the
        degree-3 ones; 1: degree 3 then degree 2 on the launch stream."""
        c = (ctypes.c_int * 4)(chunk, u_ctas_per_sm, ctas_per_sm, schedule)
        _check(_lib().wq_batch_set_config(self.handle, c), "wq_batch_set_config")

    def tune(self, reps=2, stream=None):
        ms = ctypes.c_double()
        _check(_lib().wq_batch_tune(self.handle, _stream_handle(stream), int(reps), ctypes.byref(ms)), "wq_batch_tune")
        return ms.value

    def close(self):
        if getattr(self, "handle", None):
            _lib().wq_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def assemble_batch(patches, prec="fp64", stream=None):
    """One-shot batched assembly (wq_assemble_batch) of (rules, geom, coef, M, K) tuples."""
    arr = _patch_array(patches)
    _check(_lib().wq_assemble_batch(arr, len(patches), PRECISIONS[prec], _stream_handle(stream)), "wq_assemble_batch")


# ------------------------------------------------------------------ CSR
def wq_band_nnz_rows(handle, row_begin, row_end):
    return _lib().wq_band_nnz_rows(handle, row_begin, row_end)


def band_to_csr(rules, band, prec="fp64", row_begin=0, row_end=None, stream=None):
    """CSR (rowptr int64, col int32, val) CUDA tensors of band rows
    [row_begin, row_end) (wq_band_to_csr)."""
    import torch

    if row_end is None:
        row_end = rules.rows
    nnz = wq_band_nnz_rows(rules.handle, row_begin, row_end)
    if nnz < 0:
        raise WqError(WQ_ERR_ARG, "wq_band_nnz_rows")
    dev = band.device
    assert band.is_cuda and band.is_contiguous() and tuple(band.shape) == (row_end - row_begin, rules.band)
    rowptr = torch.empty(row_end - row_begin + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    val = torch.empty(max(nnz, 1), dtype=band.dtype, device=dev)
    _check(_lib().wq_band_to_csr(rules.handle, PRECISIONS[prec], ctypes.c_void_p(band.data_ptr()), row_begin, row_end,
                                 ctypes.c_void_p(rowptr.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                 ctypes.c_void_p(val.data_ptr()), _stream_handle(stream)), "wq_band_to_csr")
    return rowptr, col[:nnz], val[:nnz]


def wq_assemble_mass_stiffness_host(handle, geom_host_ptrs, coef_host_ptr, prec, M_host_ptr, K_host_ptr,
                                    geom_dev_ptrs, coef_dev_ptr, M_dev_ptr, K_dev_ptr, row_begin, row_end, nchunks,
                                    stream, copy_stream):
    gh, keep_h = _geom_array(geom_host_ptrs)
    gd, keep_d = _geom_array(geom_dev_ptrs)
    return _lib().wq_assemble_mass_stiffness_host(handle, gh, coef_host_ptr, prec, M_host_ptr, K_host_ptr, gd,
                                                  coef_dev_ptr, M_dev_ptr, K_dev_ptr, row_begin, row_end,
                                                  int(nchunks), stream, copy_stream)


def assemble_to_host(rules, geom_host, coef_host, prec, M_host, K_host, geom_dev, coef_dev, M_dev, K_dev, nchunks=8,
                     stream=None, row_begin=0, row_end=None):
    """wq_assemble_mass_stiffness_host: inputs from host tensors (geom_host,
    coef_host; pinned for overlap) to the device buffers geom_dev, coef_dev,
    the rows assembled in nchunks ranges into M_dev, K_dev, each range copied
    into the host tensors M_host, K_host on a second stream while the next is
    assembled.  Rows [row_begin, row_end) (default all); the band tensors
    hold those rows.  Returns after enqueueing; `stream` waits for the copies."""
    import torch

    if row_end is None:
        row_end = rules.rows
    if stream is None:
        stream = torch.cuda.current_stream()
    copy = _copy_stream(stream.device)
    for X in list(geom_host) + list(geom_dev) + [M_host, K_host, M_dev, K_dev]:
        assert X.is_contiguous()
    if coef_host is not None:
        assert coef_host.is_contiguous() and coef_dev is not None and coef_dev.is_contiguous()
    st = wq_assemble_mass_stiffness_host(
        rules.handle, [g.data_ptr() for g in geom_host],
        ctypes.c_void_p(coef_host.data_ptr()) if coef_host is not None else None, PRECISIONS[prec],
        ctypes.c_void_p(M_host.data_ptr()), ctypes.c_void_p(K_host.data_ptr()), [g.data_ptr() for g in geom_dev],
        ctypes.c_void_p(coef_dev.data_ptr()) if coef_host is not None else None, ctypes.c_void_p(M_dev.data_ptr()),
        ctypes.c_void_p(K_dev.data_ptr()), row_begin, row_end, nchunks, ctypes.c_void_p(stream.cuda_stream),
        ctypes.c_void_p(copy.cuda_stream))
    _check(st, "wq_assemble_mass_stiffness_host")


_COPY_STREAMS = {}


def _copy_stream(device):
    import torch

    key = str(device)
    if key not in _COPY_STREAMS:
        _COPY_STREAMS[key] = torch.cuda.Stream(device=device)
    return _COPY_STREAMS[key]
