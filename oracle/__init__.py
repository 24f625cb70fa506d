"""Plain FP64 CPU oracle for weighted-Gaussian-quadrature assembly.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
(``paper_1710_01048_gb300``) never imports this package, and this package
never imports the product library; the two share only the seeded input
generators, which hold none of the method's arithmetic.

The arithmetic lives in ``wq_oracle.c`` (plain C, FP64, OpenMP over rows):
Cox-de Boor B-splines, Newton solves of the exactness systems of Sec. 3
(Eq. GaussQuadSys, Eq. GaussQuadSysStiff), Gauss-Legendre on boundary rows
(Remark closing Sec. 3), and row-by-row assembly of M (Eq. Mass) and K
(Eq. Stiffness) by nested loops over rows x rule points x band columns.

Parity status of each function is stated in its docstring; the pins live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libwq_oracle.so")
_lib = None

MASS, STIFFNESS = 0, 1


def build(force: bool = False) -> str:
    """Compiles wq_oracle.c into a shared library with gcc (no fast-math,
    no FMA contraction, OpenMP over rows)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    D, I, LL = ctypes.c_double, ctypes.c_int, ctypes.c_longlong
    PD, PI = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.wqo_gauss_legendre.argtypes = [I, PD, PD]
    lib.wqo_moment.argtypes = [I, I, I]
    lib.wqo_moment.restype = D
    lib.wqo_bspline.argtypes = [I, I, I, I, D]
    lib.wqo_bspline.restype = D
    lib.wqo_cardinal.argtypes = [I, I, D]
    lib.wqo_cardinal.restype = D
    lib.wqo_rule_check.argtypes = [I, I, PD, PD, D, PD]
    lib.wqo_rule.argtypes = [I, I, PD, PD, PD]
    lib.wqo_rule_newton.argtypes = [I, I, PD, I, PI, PD, PD, PD]
    lib.wqo_assemble.argtypes = [I, I, PI, PD, PD, PD, PD, LL, LL, PD, PD, PD, I]
    lib.wqo_assemble_gl.argtypes = [I, I, PI, PD, PD, PD, PD, I, LL, LL, PD, PD, I]
    lib.wqo_gradient.argtypes = [I, I, PI, PD, PD, PD, PD, PD, PD]
    lib.wqo_row_points.argtypes = [I, I, I, I, PD, PD]
    lib.wqo_rule_nc.argtypes = [I, I, PD, PD, PD]
    lib.wqo_assemble_rule.argtypes = [I, I, I, PI, PD, PD, PD, PD, LL, LL, PD, PD, I]
    lib.wqo_boundary_rule.argtypes = [I, I, I, PD, PD, PI, PD]
    lib.wqo_row_points_mode.argtypes = [I, I, I, I, I, PD, PD]
    lib.wqo_cross_rule.argtypes = [I, PD, PD, PD, PD]
    lib.wqo_row_points_cross.argtypes = [I, I, I, I, PD, PD]
    lib.wqo_assemble_general.argtypes = [I, I, PI, PD, PD, LL, LL, PD, PD, I]
    lib.wqo_assemble_gl_net.argtypes = [I, I, PI, PD, PD, I, LL, LL, PD, PD, I]
    _lib = lib
    return lib


def _pd(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes/weights on [-1, 1] (Newton on P_n)."""
    x = np.zeros(n)
    w = np.zeros(n)
    if _load().wqo_gauss_legendre(n, _pd(x), _pd(w)):
        raise ValueError("bad n")
    return x, w


def moment(p: int, kind: int, d: int) -> float:
    """int_0^{p+1} N_p^(nu)(y) N_p^(nu)(y-d) dy: the right-hand sides of
    Eq. GaussQuadSys (kind=0) and Eq. GaussQuadSysStiff (kind=1)."""
    return _load().wqo_moment(p, kind, d)


def bspline(p: int, nel: int, i: int, x: float, deriv: int = 0) -> float:
    """B_i (or B_i') of degree p on the open uniform knot vector of Eq. 3."""
    return _load().wqo_bspline(p, nel, i, deriv, float(x))


def cardinal(p: int, y: float, deriv: int = 0) -> float:
    """Cardinal B-spline N_p on knots 0..p+1 (or its derivative)."""
    return _load().wqo_cardinal(p, deriv, float(y))


def rule(p: int, kind: int):
    """The symmetric weighted Gaussian rule (tau, omega) on [0, p+1] for the
    mass (kind=0, Sec. 3.1) or stiffness (kind=1, Sec. 3.2) terms, solved by
    Newton and checked against all 2p+1 exactness conditions.  Returns
    (tau, omega, max_residual); raises RuntimeError if the solve fails."""
    tau = np.zeros(p + 1)
    om = np.zeros(p + 1)
    res = ctypes.c_double(0.0)
    st = _load().wqo_rule(p, kind, _pd(tau), _pd(om), ctypes.byref(res))
    if st:
        raise RuntimeError(f"oracle rule p={p} kind={kind} failed (status {st})")
    return tau, om, res.value


def rule_check(p: int, kind: int, tau, omega, tol: float = 1e-14):
    """(passes, max_residual) of a rule against the exactness conditions
    d = -p..p, one node per element and (mass) positive weights."""
    tau = _f64(tau)
    om = _f64(omega)
    res = ctypes.c_double(0.0)
    st = _load().wqo_rule_check(p, kind, _pd(tau), _pd(om), tol, ctypes.byref(res))
    return st == 0, res.value


def rule_newton(p: int, kind: int, u0, shifts):
    """Newton from a caller-supplied start (for the initial-guess study of
    Sec. 3.1.2).  Returns (status, tau, omega, max_residual); status 0 means
    a root that passes the exactness check."""
    u = _f64(np.array(u0, dtype=np.float64).copy())
    ds = np.ascontiguousarray(shifts, dtype=np.int32)
    tau = np.zeros(p + 1)
    om = np.zeros(p + 1)
    res = ctypes.c_double(0.0)
    st = _load().wqo_rule_newton(p, kind, _pd(u), len(u), ds.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 _pd(tau), _pd(om), ctypes.byref(res))
    return st, tau, om, res.value


def rule_nc(p: int, kind: int):
    """The Newton-Cotes-type weighted rule on the cardinal support: nodes y
    (knots and element midpoints, 2p+1) and weights v with the weight
    function's value folded in; the stiffness rule's centre weight is 0.
    Returns (y, v, max residual of the 2p+1 exactness conditions)."""
    y = np.zeros(2 * p + 1)
    v = np.zeros(2 * p + 1)
    res = ctypes.c_double(0.0)
    st = _load().wqo_rule_nc(p, kind, _pd(y), _pd(v), ctypes.byref(res))
    if st:
        raise RuntimeError(f"oracle NC rule failed (status {st})")
    return y, v, res.value


def boundary_rule(p: int, kind: int, r: int):
    """The weighted Gaussian rule of low-side boundary row r < p (the Remark
    closing Sec. 3, read as in wq_oracle.c): nodes t and weights Wl in units
    of h (x = t h, W = Wl h^(1 - kind)), and the largest relative
    residual of its conditions; None where no such rule is defined."""
    t = np.zeros(p + 1)
    W = np.zeros(p + 1)
    n = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    st = _load().wqo_boundary_rule(p, kind, r, _pd(t), _pd(W), ctypes.byref(n), ctypes.byref(res))
    if st == 2:
        return None
    if st:
        raise RuntimeError(f"oracle boundary rule p={p} kind={kind} row={r} not found")
    return t[:n.value].copy(), W[:n.value].copy(), res.value


def assemble_rule(mode, dim, p, nel, geom, coef=None, row_begin=0, row_end=None, mass=True, stiffness=True,
                  threads=0):
    """assemble() with another rule set: mode 'gl' = (p+1)-point
    Gauss-Legendre on every element of supp B_r for every row, 'nc' = the
    Newton-Cotes-type weighted rules on interior rows (the comparison
    rules), 'wqb' = the weighted Gaussian rules with the boundary rows on
    their own weighted rules (boundary_rule).  Returns (M, K)."""
    code = {"gl": 1, "nc": 2, "wqb": 3}[mode]
    nel = [int(v) for v in nel]
    n = [nel[a] + p for a in range(dim)]
    nrows = int(np.prod(n))
    if row_end is None:
        row_end = nrows
    band = (2 * p + 1) ** dim
    M = np.zeros((row_end - row_begin, band)) if mass else None
    K = np.zeros((row_end - row_begin, band)) if stiffness else None
    g = _geom_args(dim, geom)
    nel_c = (ctypes.c_int * 3)(*(nel + [1] * (3 - dim)))
    st = _load().wqo_assemble_rule(code, dim, p, nel_c, _pd(g[0]), _pd(g[1]), _pd(g[2]), _pd(_f64(coef)), row_begin,
                                   row_end, _pd(M), _pd(K), int(threads))
    if st:
        raise RuntimeError(f"oracle assemble_rule failed (status {st})")
    return M, K


def row_points(p: int, nel: int, kind: int, r: int, mode: str = "wq"):
    """Rule points and combined weights W = h*omega*B_r^(nu)(x) of row r of
    one direction (mode 'wq': GL on boundary rows; 'wqb': boundary rows on
    their weighted rules where defined)."""
    x = np.zeros(16)
    W = np.zeros(16)
    if mode == "wq":
        L = _load().wqo_row_points(p, nel, kind, r, _pd(x), _pd(W))
    else:
        L = _load().wqo_row_points_mode({"wq": 0, "gl": 1, "nc": 2, "wqb": 3}[mode], p, nel, kind, r, _pd(x), _pd(W))
    if L < 0:
        raise ValueError("bad row")
    return x[:L].copy(), W[:L].copy()


def _geom_args(dim, geom):
    g = [_f64(geom[a]) if a < dim else None for a in range(3)]
    return g


def assemble(dim, p, nel, geom, coef=None, row_begin=0, row_end=None, mass=True, stiffness=True, threads=0):
    """Rows [row_begin, row_end) of M and K in band layout, FP64.

    geom: list of dim 1D control arrays (n_a = nel_a + p each) of the
    separable map; coef: degree-3 coefficient spline on the same mesh
    (prod(nel_a+3) values, x fastest) or None for c = 1.
    Returns (M, K, offdiag) with M/K of shape (rows, (2p+1)**dim) or None,
    offdiag the largest off-diagonal metric entry relative to the diagonal."""
    nel = [int(v) for v in nel]
    n = [nel[a] + p for a in range(dim)]
    nrows = int(np.prod(n))
    if row_end is None:
        row_end = nrows
    band = (2 * p + 1) ** dim
    rows = row_end - row_begin
    M = np.zeros((rows, band)) if mass else None
    K = np.zeros((rows, band)) if stiffness else None
    g = _geom_args(dim, geom)
    c = _f64(coef)
    off = ctypes.c_double(0.0)
    nel_c = (ctypes.c_int * 3)(*(nel + [1] * (3 - dim)))
    st = _load().wqo_assemble(dim, p, nel_c, _pd(g[0]), _pd(g[1]), _pd(g[2]), _pd(c), row_begin, row_end,
                              _pd(M), _pd(K), ctypes.byref(off), int(threads))
    if st:
        raise RuntimeError(f"oracle assemble failed (status {st})")
    return M, K, off.value


def assemble_gl(dim, p, nel, geom, coef=None, ng=None, row_begin=0, row_end=None, threads=0):
    """Element-wise Gauss-Legendre assembly (ng points per direction and
    element) of the exact integrals of Eq. Mass and Eq. Stiffness with the
    full metric, in the same band layout."""
    nel = [int(v) for v in nel]
    if ng is None:
        ng = p + 3
    n = [nel[a] + p for a in range(dim)]
    nrows = int(np.prod(n))
    if row_end is None:
        row_end = nrows
    band = (2 * p + 1) ** dim
    rows = row_end - row_begin
    M = np.zeros((rows, band))
    K = np.zeros((rows, band))
    g = _geom_args(dim, geom)
    c = _f64(coef)
    nel_c = (ctypes.c_int * 3)(*(nel + [1] * (3 - dim)))
    st = _load().wqo_assemble_gl(dim, p, nel_c, _pd(g[0]), _pd(g[1]), _pd(g[2]), _pd(c), ng, row_begin, row_end,
                                 _pd(M), _pd(K), int(threads))
    if st:
        raise RuntimeError(f"oracle GL assemble failed (status {st})")
    return M, K


def gradient(dim, p, nel, geom, G=None, H=None):
    """dJ/dc for J(c) = sum(G * K(c)) + sum(H * M(c)) over the degree-3
    coefficient spline (prod(nel_a + 3) values, x fastest)."""
    nel = [int(v) for v in nel]
    ncoef = int(np.prod([nel[a] + 3 for a in range(dim)]))
    grad = np.zeros(ncoef)
    g = _geom_args(dim, geom)
    nel_c = (ctypes.c_int * 3)(*(nel + [1] * (3 - dim)))
    st = _load().wqo_gradient(dim, p, nel_c, _pd(g[0]), _pd(g[1]), _pd(g[2]), _pd(_f64(G)), _pd(_f64(H)),
                              _pd(grad))
    if st:
        raise RuntimeError(f"oracle gradient failed (status {st})")
    return grad


# ------------------------------------------------------------------ maps with a full control net
def cross_rule(p: int):
    """The mixed-derivative rules of the non-separable stiffness terms (read
    as in wq_oracle.c, wqo_cross_rule): nodes y on the cardinal support
    [0, p+1] shared by kind 2 (weights w for the weight N', tests N) and
    kind 3 (weights v for the weight N, tests N').  Returns (y, w, v,
    max_residual)."""
    y = np.zeros(p + 1)
    w = np.zeros(p + 1)
    v = np.zeros(p + 1)
    res = ctypes.c_double(0.0)
    st = _load().wqo_cross_rule(p, _pd(y), _pd(w), _pd(v), ctypes.byref(res))
    if st:
        raise RuntimeError(f"oracle cross rule p={p} failed (status {st})")
    return y, w, v, res.value


def row_points_cross(p: int, nel: int, kind: int, r: int):
    """Points and weights of row r of one direction for kind 2 (weight B_r',
    tests B_s) or kind 3 (weight B_r, tests B_s')."""
    x = np.zeros(16)
    W = np.zeros(16)
    L = _load().wqo_row_points_cross(p, nel, kind, r, _pd(x), _pd(W))
    if L < 0:
        raise ValueError("bad row or kind")
    return x[:L].copy(), W[:L].copy()


def _net_args(dim, p, nel, net):
    n = [int(nel[a]) + p for a in range(dim)]
    net = _f64(net)
    if net.size != dim * int(np.prod(n)):
        raise ValueError("net must hold dim * prod(nel + p) values")
    return net


def assemble_general(dim, p, nel, net, coef=None, row_begin=0, row_end=None, mass=True, stiffness=True, threads=0):
    """Rows [row_begin, row_end) of M and K (full metric) for the map given by
    its full control net (component a of control point (i1, i2, i3) at
    net[a * prod(n) + i1 + n1 * (i2 + n2 * i3)]), with the weighted rules of
    Sec. 3 for the mass and (B', B') terms and the mixed rules (cross_rule)
    for the off-diagonal metric terms.  Returns (M, K)."""
    nel = [int(v) for v in nel]
    n = [nel[a] + p for a in range(dim)]
    nrows = int(np.prod(n))
    if row_end is None:
        row_end = nrows
    band = (2 * p + 1) ** dim
    M = np.zeros((row_end - row_begin, band)) if mass else None
    K = np.zeros((row_end - row_begin, band)) if stiffness else None
    g = _net_args(dim, p, nel, net)
    nel_c = (ctypes.c_int * 3)(*(nel + [1] * (3 - dim)))
    st = _load().wqo_assemble_general(dim, p, nel_c, _pd(g), _pd(_f64(coef)), row_begin, row_end, _pd(M), _pd(K),
                                      int(threads))
    if st:
        raise RuntimeError(f"oracle assemble_general failed (status {st})")
    return M, K


def assemble_gl_net(dim, p, nel, net, coef=None, ng=None, row_begin=0, row_end=None, threads=0):
    """assemble_gl for the map given by its full control net."""
    nel = [int(v) for v in nel]
    if ng is None:
        ng = p + 3
    n = [nel[a] + p for a in range(dim)]
    nrows = int(np.prod(n))
    if row_end is None:
        row_end = nrows
    band = (2 * p + 1) ** dim
    M = np.zeros((row_end - row_begin, band))
    K = np.zeros((row_end - row_begin, band))
    g = _net_args(dim, p, nel, net)
    nel_c = (ctypes.c_int * 3)(*(nel + [1] * (3 - dim)))
    st = _load().wqo_assemble_gl_net(dim, p, nel_c, _pd(g), _pd(_f64(coef)), ng, row_begin, row_end, _pd(M), _pd(K),
                                     int(threads))
    if st:
        raise RuntimeError(f"oracle GL assemble (net) failed (status {st})")
    return M, K
