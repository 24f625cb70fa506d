"""Pins of the oracle's mixed-derivative rules and of its assembly for maps
given by a full control net (wq_oracle.c: wqo_cross_rule, cross_row_rule,
wqo_assemble_general).

The paper gives weighted rules for the (B, B) and (B', B') pairs only
(Sec. 3.1, 3.2); a non-separable map adds to Eq. Stiffness the terms
dB_r/dxhat_a C_ab dB_s/dxhat_b, a != b, which pair the weight B_r' with the
tests B_s in direction a (kind 2) and the weight B_r with the tests B_s' in
direction b (kind 3).  The reading: one node set per interior row for both
kinds, nodes symmetric about the centre of the support, kind 2's weights
antisymmetric and kind 3's symmetric, p conditions each.

Pinned here against what does not come from the rule code:
* p = 2 in closed form.  With y in (0, 1) and N_2 = y^2/2, (-2y^2+6y-3)/2,
  (3-y)^2/2 on its three elements, kind 2's conditions d = 1, 2 read
  w (-2y^2+2y+1) = 5/6 and w (1-y)^2 = 1/12, whose ratio gives
  12 y^2 - 22 y + 9 = 0, y = (11 - sqrt 13)/12, w = 1/(12 (1-y)^2); kind
  3's read v (1-y) = 1/24 and vc/2 - v (1-2y) = 5/12.
* p = 3 (and 2) against moments computed here from the truncated-power form
  of the cardinal B-spline (independent of the oracle's Cox-de Boor), and
  against polynomial reproduction: kind 3 is exact for every spline of
  degree p-1 on the support (the span of the N'(. - d)), so
  sum v y^j = int N y^j for j < p; kind 2 for every degree-p spline, so
  sum w y^j = -j int N y^(j-1) for j <= p.
* Row rules on meshes (interior and Gauss-Legendre boundary rows) exact for
  every interacting B_s against element-wise Gauss-Legendre brute force.
* Assembly: on affine maps with shear (non-separable, constant J) and c = 1
  every rule is exact, so M and K equal the element-wise Gauss-Legendre
  integrals with the full metric, in 2D and 3D, p = 2 and 3, including
  meshes with no interior row; the total of M is |det A|; a separable net
  reproduces the separable assembly; K annihilates constants on a warped map.
"""
from math import comb, factorial, sqrt

import numpy as np
import pytest

import oracle
from paper_1710_01048_gb300 import inputs

GX, GW = np.polynomial.legendre.leggauss(12)


def card(p, y, nu=0):
    """Cardinal B-spline on 0..p+1 by the truncated-power formula."""
    y = np.asarray(y, dtype=np.float64)
    if nu == 1:
        return card(p - 1, y) - card(p - 1, y - 1.0)
    s = np.zeros_like(y)
    for i in range(p + 2):
        s += (-1) ** i * comb(p + 1, i) * np.where(y > i, y - i, 0.0) ** p
    return np.where((y >= 0) & (y <= p + 1), s / factorial(p), 0.0)


def cmoment(p, f):
    """int_0^{p+1} f(y) dy, element-wise 12-point Gauss-Legendre."""
    tot = 0.0
    for e in range(p + 1):
        y = e + 0.5 * (GX + 1.0)
        tot += 0.5 * float(np.dot(GW, f(y)))
    return tot


def test_p2_closed_form():
    y1 = (11.0 - sqrt(13.0)) / 12.0
    w1 = 1.0 / (12.0 * (1.0 - y1) ** 2)
    v1 = 1.0 / (24.0 * (1.0 - y1))
    vc = 5.0 / 6.0 + 2.0 * v1 * (1.0 - 2.0 * y1)
    y, w, v, res = oracle.cross_rule(2)
    assert np.max(np.abs(y - [y1, 1.5, 3.0 - y1])) <= 1e-15
    assert np.max(np.abs(w - [w1, 0.0, -w1])) <= 2e-15
    assert np.max(np.abs(v - [v1, vc, v1])) <= 2e-15
    assert res <= 1e-15


@pytest.mark.parametrize("p", [2, 3])
def test_exact_against_independent_moments(p):
    y, w, v, _ = oracle.cross_rule(p)
    assert len(y) == p + 1
    for k in range(p + 1):
        assert k < y[k] < k + 1  # one node per element
    assert np.max(np.abs(y + y[::-1] - (p + 1))) <= 1e-15
    assert np.max(np.abs(w + w[::-1])) <= 1e-15 and np.max(np.abs(v - v[::-1])) <= 1e-15
    for d in range(-p, p + 1):
        m2 = cmoment(p, lambda t: card(p, t, 1) * card(p, t - d))
        m3 = cmoment(p, lambda t: card(p, t) * card(p, t - d, 1))
        assert abs(np.dot(w, card(p, y - d)) - m2) <= 1e-14, d
        assert abs(np.dot(v, card(p, y - d, 1)) - m3) <= 1e-14, d


@pytest.mark.parametrize("p", [2, 3])
def test_polynomial_reproduction(p):
    y, w, v, _ = oracle.cross_rule(p)
    for j in range(p):
        assert abs(np.dot(v, y ** j) - cmoment(p, lambda t: card(p, t) * t ** j)) <= 1e-14 * (p + 1) ** j
    for j in range(p + 1):
        ref = -j * cmoment(p, lambda t: card(p, t) * t ** (j - 1)) if j else 0.0
        assert abs(np.dot(w, y ** j) - ref) <= 1e-14 * (p + 1) ** j
    assert abs(v.sum() - 1.0) <= 1e-15


def brute(p, N, r, s, nuw, nut):
    """int B_r^(nuw) B_s^(nut) over supp B_r, 12-point Gauss-Legendre per element."""
    h = 1.0 / N
    tot = 0.0
    for e in range(max(0, r - p), min(N - 1, r) + 1):
        xs = (e + 0.5 * (GX + 1.0)) * h
        f = [oracle.bspline(p, N, r, x, nuw) * oracle.bspline(p, N, s, x, nut) for x in xs]
        tot += 0.5 * h * float(np.dot(GW, f))
    return tot


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("N", [1, 4, 9, 17])
def test_row_rules_exact_on_interacting_splines(p, N):
    n = N + p
    for kind, (nuw, nut) in ((2, (1, 0)), (3, (0, 1))):
        for r in range(n):
            x, W = oracle.row_points_cross(p, N, kind, r)
            interior = p <= r <= N - 1
            assert len(x) == (p + 1 if interior else (min(N - 1, r) - max(0, r - p) + 1) * (p + 1))
            cols = range(max(0, r - p), min(n - 1, r + p) + 1)
            ex = [brute(p, N, r, s, nuw, nut) for s in cols]
            scale = max(abs(e) for e in ex)
            for s, e in zip(cols, ex):
                q = float(np.dot(W, [oracle.bspline(p, N, s, xx, nut) for xx in x]))
                assert abs(q - e) <= 1e-13 * scale, (kind, r, s)


@pytest.mark.parametrize("dim,p,nel", [(3, 3, (7, 8, 9)), (3, 2, (5, 6, 7)), (2, 3, (9, 8)), (2, 2, (6, 7)),
                                       (3, 3, (2, 3, 1)), (2, 3, (1, 2)), (3, 2, (1, 1, 1))])
def test_exact_on_sheared_affine_maps(dim, p, nel):
    net = inputs.full_net(p, nel, "affine")
    M, K = oracle.assemble_general(dim, p, nel, net)
    Me, Ke = oracle.assemble_gl_net(dim, p, nel, net)
    for A, E in ((M, Me), (K, Ke)):
        assert np.max(np.abs(A - E)) <= 1e-13 * np.max(np.abs(E))
    # the off-diagonal metric terms are not small on this map
    A, _ = inputs.AFFINE[dim]
    Ai = np.linalg.inv(A)
    G = Ai @ Ai.T
    assert np.max(np.abs(G - np.diag(np.diag(G)))) > 0.1 * np.max(np.diag(G))
    assert abs(M.sum() - abs(np.linalg.det(A))) <= 1e-13


@pytest.mark.parametrize("dim,p,nel", [(3, 3, (5, 6, 4)), (3, 2, (4, 3, 5)), (2, 3, (7, 6))])
def test_separable_net_reproduces_separable_assembly(dim, p, nel):
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=4)
    net = inputs.net_from_separable(p, nel, g)
    M0, K0, _ = oracle.assemble(dim, p, nel, g, c)
    M1, K1 = oracle.assemble_general(dim, p, nel, net, c)
    for A, B in ((M1, M0), (K1, K0)):
        assert np.max(np.abs(A - B)) <= 1e-15 * np.max(np.abs(B))
    # and the Gauss-Legendre oracle reads the net with the same layout
    Ge, He = oracle.assemble_gl(dim, p, nel, g, c)
    Gn, Hn = oracle.assemble_gl_net(dim, p, nel, net, c)
    assert np.max(np.abs(Gn - Ge)) <= 1e-15 * np.max(np.abs(Ge))
    assert np.max(np.abs(Hn - He)) <= 1e-15 * np.max(np.abs(He))


@pytest.mark.parametrize("dim,p,nel", [(3, 3, (6, 5, 7)), (2, 2, (8, 7))])
def test_warped_map_invariants(dim, p, nel):
    net, c = inputs.make_net(dim, p, nel, "warp", 0.05, "exp", 0.1, seed=2)
    M, K = oracle.assemble_general(dim, p, nel, net, c)
    assert np.max(np.abs(K.sum(axis=1))) <= 1e-13 * np.max(np.abs(K).sum(axis=1))
    # close to the exact integrals (the rules are exact only for affine maps)
    Me, Ke = oracle.assemble_gl_net(dim, p, nel, net, c, ng=8)
    assert np.max(np.abs(M - Me)) <= 2e-2 * np.max(np.abs(Me))
    assert np.max(np.abs(K - Ke)) <= 5e-2 * np.max(np.abs(Ke))
