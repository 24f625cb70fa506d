"""Pins of the oracle's weighted Gaussian rules for the boundary rows.

The Remark closing Sec. 3 leaves the boundary rows to the systems "modified
accordingly"; the reading (wq_oracle.c, wqo_boundary_rule): row r < p of
kind nu gets ceil(rank/2) nodes exact for B_r^(nu) B_s^(nu), s = 0..r+p
(rank = r+p+1 for the mass kind, one less for the stiffness kind), plus
B_r^(nu) (x/h)^(p-nu+1) when the rank is odd; high-side rows are the mirror
images; rows without such a rule (p = 3 stiffness row 1) keep Gauss-Legendre.

Pinned here against what does not come from the rule code:
* exactness against brute-force Gauss-Legendre moments (numpy nodes, the
  pinned Cox-de Boor B-splines) on meshes of several sizes;
* the node counts, and nodes strictly inside the support;
* closed forms: the classical 2-point Gauss rule of the weight (1-t)^2 on
  [0, 1] (p = 2 mass row 0, p = 3 stiffness row 0, from exact rational
  moments) and the 1-point rule t = 1/3 of p = 2 stiffness row 0;
* the mirror relation of the high-side rows;
* assembly with these rules on affine maps with c = 1 equals the exact
  integrals (element-wise Gauss-Legendre brute force), and the invariants.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1710_01048_gb300 import inputs

GX, GW = np.polynomial.legendre.leggauss(12)


def exact_moment(p, N, r, s, kind):
    """int B_r^(kind) B_s^(kind) over supp B_r by 12-point Gauss-Legendre per element."""
    h = 1.0 / N
    tot = 0.0
    for e in range(max(0, r - p), min(N - 1, r) + 1):
        xs = (e + 0.5 * (GX + 1.0)) * h
        f = [oracle.bspline(p, N, r, x, kind) * oracle.bspline(p, N, s, x, kind) for x in xs]
        tot += 0.5 * h * float(np.dot(GW, f))
    return tot


DEFINED = {(2, 0, 0): 2, (2, 0, 1): 2, (2, 1, 0): 1, (2, 1, 1): 2, (3, 0, 0): 2, (3, 0, 1): 3, (3, 0, 2): 3,
           (3, 1, 0): 2, (3, 1, 2): 3}


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("kind", [0, 1])
def test_boundary_rules_counts_and_support(p, kind):
    for r in range(p):
        b = oracle.boundary_rule(p, kind, r)
        key = (p, kind, r)
        if key not in DEFINED:
            assert b is None
            continue
        t, W, res = b
        assert len(t) == DEFINED[key]
        m = r + p + 1
        rank = m - 1 if kind else m
        assert len(t) == (rank + 1) // 2
        assert np.all(t > 0.0) and np.all(t < r + 1.0) and np.all(np.diff(t) > 0)
        assert res <= 1e-14


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("N", [None, 9, 31])
def test_boundary_rows_exact_on_interacting_splines(p, N):
    N = 2 * p + 1 if N is None else N
    n = N + p
    for kind in (0, 1):
        for r in list(range(p)) + [n - 1 - i for i in range(p)]:
            x, W = oracle.row_points(p, N, kind, r, "wqb")
            rm = r if r < p else n - 1 - r
            expect = DEFINED.get((p, kind, rm))
            gl = (min(N - 1, r) - max(0, r - p) + 1) * (p + 1)
            assert len(x) == (expect if expect else gl)
            scale = max(abs(exact_moment(p, N, r, s, kind)) for s in range(max(0, r - p), min(n - 1, r + p) + 1))
            for s in range(max(0, r - p), min(n - 1, r + p) + 1):
                q = float(np.dot(W, [oracle.bspline(p, N, s, xx, kind) for xx in x]))
                assert abs(q - exact_moment(p, N, r, s, kind)) <= 1e-13 * scale, (kind, r, s)


def _gauss_weight_one_minus_t_squared():
    """2-point Gauss rule of w(t) = (1-t)^2 on [0, 1]: nodes are the roots of
    the monic quadratic orthogonal to 1 and t, from the exact moments
    int (1-t)^2 t^k dt = 2 / ((k+1)(k+2)(k+3))."""
    mom = [Fraction(2, (k + 1) * (k + 2) * (k + 3)) for k in range(4)]
    # t^2 + a t + b orthogonal to 1 and t: [m1 m0; m2 m1] [a; b] = -[m2; m3]
    det = mom[1] * mom[1] - mom[0] * mom[2]
    a = (-mom[2] * mom[1] + mom[3] * mom[0]) / det
    b = (-mom[3] * mom[1] + mom[2] * mom[2]) / det
    disc = float(a * a - 4 * b)
    t = np.array([(-float(a) - disc ** 0.5) / 2, (-float(a) + disc ** 0.5) / 2])
    # weights from int w = W0 + W1 and int w t = W0 t0 + W1 t1
    A = np.array([[1.0, 1.0], [t[0], t[1]]])
    Wt = np.linalg.solve(A, [float(mom[0]), float(mom[1])])
    return t, Wt


def test_closed_forms():
    t_ref, w_ref = _gauss_weight_one_minus_t_squared()
    # p = 2 mass row 0: weight B_0 = (1-t)^2, span of the tests on [0, h] = P_2,
    # the odd rank's extra condition t^3 makes it the classical Gauss rule
    # (the Newton solve stops at residuals of ~1e-17; the nodes then agree
    # with the closed form to a few 1e-14)
    t, W, _ = oracle.boundary_rule(2, 0, 0)
    assert np.max(np.abs(t - t_ref)) <= 1e-13
    # W = omega B_0(x), B_0 = (1-t)^2: the Gauss weights of (1-t)^2 in units of h
    assert np.max(np.abs(W - w_ref)) <= 1e-13
    # p = 3 stiffness row 0: weight B_0' = -3/h (1-t)^2, the tests' derivatives
    # span P_2 (the extra condition t^3 again): int B_0' f dx = -3 sum w_k f(t_k),
    # so W = -3 w (independent of h)
    t, W, _ = oracle.boundary_rule(3, 1, 0)
    assert np.max(np.abs(t - t_ref)) <= 1e-13
    assert np.max(np.abs(W + 3.0 * w_ref)) <= 1e-13
    # p = 2 stiffness row 0: weight B_0' = -2/h (1-t), one node at the centroid 1/3
    t, W, _ = oracle.boundary_rule(2, 1, 0)
    assert len(t) == 1 and abs(t[0] - 1.0 / 3.0) <= 1e-15


@pytest.mark.parametrize("p", [2, 3])
def test_high_side_rows_mirror_the_low_side(p):
    N = 11
    n = N + p
    for kind in (0, 1):
        for r in range(p):
            xl, Wl = oracle.row_points(p, N, kind, r, "wqb")
            xh, Wh = oracle.row_points(p, N, kind, n - 1 - r, "wqb")
            o = np.argsort(1.0 - xh)
            assert np.max(np.abs((1.0 - xh)[o] - np.sort(xl))) <= 1e-15
            sign = -1.0 if kind else 1.0
            assert np.max(np.abs(sign * Wh[o] - Wl[np.argsort(xl)])) <= 4e-15 * max(1.0, np.max(np.abs(Wl)))


@pytest.mark.parametrize("dim,p,nel", [(2, 2, (5, 7)), (2, 3, (7, 9)), (3, 2, (5, 6, 5)), (3, 3, (7, 8, 7)),
                                       (3, 3, (3, 2, 4)), (2, 3, (12, 8))])
def test_assembly_with_boundary_rules_is_exact_on_affine_maps(dim, p, nel):
    # c = 1 on an affine map: every rule is exact for its integrands, so the
    # bands are the exact integrals (element-wise Gauss-Legendre brute force)
    g, _ = inputs.make(dim, p, nel, 0.0, "one")
    M, K = oracle.assemble_rule("wqb", dim, p, nel, g)
    Me, Ke = oracle.assemble_gl(dim, p, nel, g)
    for A, E in ((M, Me), (K, Ke)):
        assert np.max(np.abs(A - E)) <= 1e-13 * np.max(np.abs(E))


@pytest.mark.parametrize("dim,p,nel", [(3, 3, (8, 7, 9)), (2, 2, (9, 6)), (3, 2, (6, 7, 5))])
def test_boundary_rule_assembly_invariants(dim, p, nel):
    # any coefficient, separable non-affine map: K annihilates constants;
    # c = 1 on the identity: M's row sums are the integrals of B_r, total 1
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=3)
    M, K = oracle.assemble_rule("wqb", dim, p, nel, g, c)
    assert np.max(np.abs(K.sum(axis=1))) <= 1e-13 * np.max(np.abs(K).sum(axis=1))
    g1, _ = inputs.make(dim, p, nel, 0.0, "one")
    M1, _ = oracle.assemble_rule("wqb", dim, p, nel, g1)
    assert abs(M1.sum() - 1.0) <= 1e-13
    Mw, _, _ = oracle.assemble(dim, p, nel, g1)
    assert np.max(np.abs(M1.sum(axis=1) - Mw.sum(axis=1))) <= 1e-14
