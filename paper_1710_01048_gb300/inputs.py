"""Seeded synthetic inputs: separable geometry maps and coefficient splines.

This module holds no arithmetic of the assembly method.  It builds the inputs
that both the CUDA path and the CPU oracle consume:

* ``geometry(p, nel, amp)``: per direction a, the 1D control values
  g_{a,i} = xi*_i + amp_a * sin(pi * xi*_i) of the separable map
  x_a = sum_i g_{a,i} B_i(xhat_a), where xi*_i are the Greville abscissae
  (mean of the p interior knots of B_i).  With amp = 0 this is exactly the
  identity map (B-splines reproduce linear functions through their Greville
  abscissae), and J_aa >= 1 - amp*pi > 0 for amp < 1/pi.
* ``coefficients(nel, f, seed, sigma)``: the degree-3 coefficient spline of c
  on the same mesh, c_l = f(xi3*_l) * exp(sigma * z_l), z ~ N(0, 1) drawn
  with numpy's default_rng(seed) in x-fastest order.
* ``workload(name)``: the named synthetic workloads (sizes, geometry
  amplitude, coefficient recipe) used by the tests and the benchmark.
* ``full_net(p, nel, kind, amp)``: the full control net of a non-separable
  map (component a of control point i at net[a * prod(n) + i1 + n1 * (i2 +
  n2 * i3)]), the control points being the images of the Greville points
  under an affine map with shear ('affine', reproduced exactly) or under the
  warp xi_a + amp * (sin(pi xi_a) + sin(pi xi_b) sin(pi xi_c)), (b, c) the
  other directions ('warp'); ``net_from_separable`` writes a separable map's
  1D arrays as such a net.
"""
from __future__ import annotations

import math

import numpy as np


def open_uniform_knots(p: int, nel: int) -> np.ndarray:
    """p+1 zeros, the interior knots i/nel, p+1 ones."""
    inner = np.arange(1, nel, dtype=np.float64) / nel
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def greville(p: int, nel: int) -> np.ndarray:
    """Greville abscissae of the nel+p degree-p B-splines."""
    t = open_uniform_knots(p, nel)
    n = nel + p
    return np.array([t[i + 1:i + p + 1].mean() for i in range(n)])


def geometry(p: int, nel, amp=0.0):
    """List of 1D control arrays (one per direction) of a separable map."""
    dim = len(nel)
    amps = np.broadcast_to(np.asarray(amp, dtype=np.float64), (dim,))
    out = []
    for a in range(dim):
        xi = greville(p, int(nel[a]))
        out.append(np.ascontiguousarray(xi + amps[a] * np.sin(np.pi * xi)))
    return out


def coefficients(nel, f=None, seed=None, sigma=0.0) -> np.ndarray:
    """Degree-3 coefficient spline on the mesh `nel`, x fastest.

    f maps a tuple of Greville coordinate arrays (parameter space) to values;
    None means f = 1.  sigma > 0 multiplies by lognormal noise from
    default_rng(seed)."""
    dim = len(nel)
    xs = [greville(3, int(nel[a])) for a in range(dim)]
    grids = np.meshgrid(*xs, indexing="ij")  # grids[a][l1, l2, l3]
    if f is None:
        vals = np.ones_like(grids[0])
    else:
        vals = np.asarray(f(*grids), dtype=np.float64)
    if sigma:
        rng = np.random.default_rng(seed)
        # x fastest: draw in the storage order (l3, l2, l1) then transpose back
        z = rng.standard_normal(size=tuple(reversed(vals.shape))).transpose()
        vals = vals * np.exp(sigma * z)
    return np.ascontiguousarray(vals.transpose().reshape(-1))


def sin_cos_2d(x, y):
    """c(x, y) = 1 + 0.5 sin(2 pi x) cos(2 pi y)."""
    return 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)


def exp_sum(*xs):
    """c(x) = exp(0.3 * sum of coordinates)."""
    return np.exp(0.3 * sum(xs))


def band_random(nel, p, seed):
    """N(0, 1) band arrays with zeros on out-of-range columns (the weights
    G, H of the scalar functional J = sum G*K + sum H*M)."""
    dim = len(nel)
    n = [int(nel[a]) + p for a in range(dim)]
    nb = 2 * p + 1
    rng = np.random.default_rng(seed)
    rows = int(np.prod(n))
    A = rng.standard_normal(size=(rows, nb ** dim))
    return A * band_mask(nel, p)


def band_mask(nel, p):
    """1 where the band entry's column index is inside the mesh, else 0."""
    dim = len(nel)
    n = [int(nel[a]) + p for a in range(dim)]
    nb = 2 * p + 1
    masks = []
    for a in range(dim):
        r = np.arange(n[a])[:, None]
        d = np.arange(-p, p + 1)[None, :]
        masks.append(((r + d >= 0) & (r + d < n[a])).astype(np.float64))
    m = masks[0]  # [r1, d1]
    for a in range(1, dim):
        # rows: r1 fastest; band: d1 fastest
        m = np.einsum("ij,kl->kilj", m.reshape(-1, nb ** a), masks[a]).reshape(-1, nb ** (a + 1))
    return m


WORKLOADS = {
    # 2D C2 cubic, 32x32 elements, identity map, c = 1 + 0.5 sin(2 pi x) cos(2 pi y)
    "2d_p3_32": dict(dim=2, p=3, nel=(32, 32), amp=0.0, coef="sincos", sigma=0.0, seed=0),
    "2d_p3_32_c1": dict(dim=2, p=3, nel=(32, 32), amp=0.0, coef="one", sigma=0.0, seed=0),
    # 3D, 64^3, x + 0.05 sin(pi x) per coordinate, c = exp(0.3 (x+y+z)) * lognormal(0.1), seed 0
    "3d_p2_64": dict(dim=3, p=2, nel=(64, 64, 64), amp=0.05, coef="exp", sigma=0.1, seed=0),
    "3d_p3_64": dict(dim=3, p=3, nel=(64, 64, 64), amp=0.05, coef="exp", sigma=0.1, seed=0),
    # 3D C2 cubic, 128^3, same geometry and coefficient recipe
    "3d_p3_128": dict(dim=3, p=3, nel=(128, 128, 128), amp=0.05, coef="exp", sigma=0.1, seed=0),
    # differentiation workload, 96^3 (and the 12^3 oracle-gradient sub-instance)
    "3d_p3_96": dict(dim=3, p=3, nel=(96, 96, 96), amp=0.05, coef="exp", sigma=0.1, seed=0),
    "3d_p3_12": dict(dim=3, p=3, nel=(12, 12, 12), amp=0.05, coef="exp", sigma=0.1, seed=0),
}

# Non-separable maps (full control nets): the warp of full_net with amp 0.05,
# the same coefficient recipe
NET_WORKLOADS = {
    "3d_p3_64_warp": dict(dim=3, p=3, nel=(64, 64, 64), net="warp", amp=0.05, coef="exp", sigma=0.1, seed=0),
    "3d_p3_128_warp": dict(dim=3, p=3, nel=(128, 128, 128), net="warp", amp=0.05, coef="exp", sigma=0.1, seed=0),
    "2d_p3_32_warp": dict(dim=2, p=3, nel=(32, 32), net="warp", amp=0.05, coef="sincos", sigma=0.0, seed=0),
}


def make_net(dim, p, nel, net="warp", amp=0.05, coef="one", sigma=0.0, seed=0):
    """(net, coef) arrays for a non-separable workload description."""
    nel = tuple(int(v) for v in nel)
    _, c = make(dim, p, nel, 0.0, coef, sigma, seed)
    return full_net(p, nel, net, amp), c


def make(dim, p, nel, amp=0.0, coef="one", sigma=0.0, seed=0):
    """(geom, coef) arrays for a workload description."""
    nel = tuple(int(v) for v in nel)
    g = geometry(p, nel, amp)
    if coef == "one":
        c = coefficients(nel)
    elif coef == "sincos":
        c = coefficients(nel, sin_cos_2d)
    elif coef == "exp":
        c = coefficients(nel, exp_sum, seed=seed, sigma=sigma)
    else:
        raise ValueError(coef)
    return g, c


# a fixed sheared affine map (det > 0) and its translation, per dimension
AFFINE = {2: (np.array([[1.0, 0.35], [-0.2, 0.9]]), np.array([0.1, -0.2])),
          3: (np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]]), np.array([0.1, -0.2, 0.3]))}


def _greville_grid(p, nel):
    dim = len(nel)
    xs = [greville(p, int(nel[a])) for a in range(dim)]
    return np.meshgrid(*xs, indexing="ij")  # [a][i1, i2, i3]


def _flatten_net(comps):
    """Component arrays indexed [i1, i2, i3] -> flat net, x fastest per component."""
    return np.ascontiguousarray(np.concatenate([c.transpose().reshape(-1) for c in comps]))


def full_net(p, nel, kind="warp", amp=0.05):
    dim = len(nel)
    xi = _greville_grid(p, nel)
    if kind == "affine":
        A, b = AFFINE[dim]
        comps = [sum(A[a, c] * xi[c] for c in range(dim)) + b[a] for a in range(dim)]
    elif kind == "warp":
        comps = []
        for a in range(dim):
            others = [c for c in range(dim) if c != a]
            cross = np.ones_like(xi[0])
            for c in others:
                cross = cross * np.sin(np.pi * xi[c])
            comps.append(xi[a] + amp * (np.sin(np.pi * xi[a]) + cross))
    else:
        raise ValueError(kind)
    return _flatten_net(comps)


def net_from_separable(p, nel, geom):
    """The full net of the separable map with 1D control arrays geom."""
    dim = len(nel)
    grids = np.meshgrid(*[np.asarray(geom[a], dtype=np.float64) for a in range(dim)], indexing="ij")
    return _flatten_net(grids)


def workload(name):
    w = WORKLOADS[name]
    g, c = make(w["dim"], w["p"], w["nel"], w["amp"], w["coef"], w["sigma"], w["seed"])
    return w, g, c


def batch_patches(npatch=256, seed=0, lo=8, hi=48):
    """Independent patches: per-direction element counts log-uniform in
    [lo, hi], degree 2 or 3 with equal probability, geometry amplitude
    U[0, 0.08], coefficients exp(0.3 sum x) with lognormal(0.1) noise."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(npatch):
        nel = tuple(int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(3))
        p = int(rng.choice([2, 3]))
        amp = float(rng.uniform(0.0, 0.08))
        g, c = make(3, p, nel, amp, "exp", 0.1, seed + 1000 + i)
        out.append(dict(dim=3, p=p, nel=nel, amp=amp, geom=g, coef=c))
    return out
