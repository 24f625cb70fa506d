"""Pins of the oracle's row-wise assembly against what the paper and the
mathematics fix:

* exactness for constant coefficient on affine maps (Remark closing Sec. 3):
  brute-force element-wise Gauss-Legendre assembly of the exact integrals,
  including every boundary row, and closed forms of the interior entries from
  the exact moments;
* the 1D comparison of Sec. 4 (weighted vs standard Gauss, 1000 elements);
* invariants: zero row sums of K, row sums of M = integral of B_r, total mass,
  symmetry for constant coefficient on the identity map, linearity in c;
* non-constant coefficient on a non-affine map: an independent evaluation of
  the weighted sum for interior rows from the printed rules, explicit cardinal
  B-spline pieces and closed-form c and J;
* the gradient: Euler's identity, finite differences, unit coefficient vectors.
"""
import itertools

import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_1710_01048_gb300 import inputs


def rel_err(A, B):
    return np.max(np.abs(A - B)) / np.max(np.abs(B))


def band_index(d, p):
    nb = 2 * p + 1
    return sum((d[a] + p) * nb ** a for a in range(len(d)))


def row_index(r, n):
    idx, mul = 0, 1
    for a in range(len(r)):
        idx += r[a] * mul
        mul *= n[a]
    return idx


# ------------------------------------------------------------ exactness, affine
@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("nel", [(1, 1), (2, 3), (4, 4), (6, 5)])
def test_wq_equals_exact_integrals_2d_identity(p, nel):
    g = inputs.geometry(p, nel)
    M, K, off = oracle.assemble(2, p, nel, g)
    Mg, Kg = oracle.assemble_gl(2, p, nel, g, ng=p + 2)
    assert rel_err(M, Mg) < 1e-14
    assert rel_err(K, Kg) < 1e-14
    assert off < 1e-14


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("nel", [(1, 2, 1), (3, 3, 2), (4, 3, 5)])
def test_wq_equals_exact_integrals_3d_affine(p, nel):
    alpha = np.array([1.5, 0.75, 2.0])
    beta = np.array([0.25, -1.0, 3.0])
    g = [alpha[a] * gi + beta[a] for a, gi in enumerate(inputs.geometry(p, nel))]
    M, K, off = oracle.assemble(3, p, nel, g)
    Mg, Kg = oracle.assemble_gl(3, p, nel, g, ng=p + 1)
    assert rel_err(M, Mg) < 1e-14
    assert rel_err(K, Kg) < 1e-14
    assert off < 1e-14
    # scaling by the affine map: M by prod alpha, K term a by prod alpha / alpha_a^2
    M0, K0, _ = oracle.assemble(3, p, nel, inputs.geometry(p, nel))
    assert rel_err(M, np.prod(alpha) * M0) < 1e-14


@pytest.mark.parametrize("p", [2, 3])
def test_interior_entries_closed_form_3d(p):
    nel = (3 * p + 2, 3 * p + 1, 3 * p + 3)
    n = [v + p for v in nel]
    h = [1.0 / v for v in nel]
    M, K, _ = oracle.assemble(3, p, nel, inputs.geometry(p, nel))
    mom = {}
    for kind, pp, d, num, den in [r[:5] for r in read_golden("moments_exact.txt")]:
        if int(pp) == p:
            mom[(kind, int(d))] = int(num) / int(den)

    def m(d):
        return mom[("mass", abs(d))]

    def k(d):
        return mom[("stiff", abs(d))]

    checked = 0
    # rows whose every band column is an interior (cardinal) B-spline
    rng = [range(2 * p, nel[a] - p) for a in range(3)]
    for r in itertools.product(*rng):
        ri = row_index(r, n)
        for d in itertools.product(range(-p, p + 1), repeat=3):
            bi = band_index(d, p)
            Mex = h[0] * h[1] * h[2] * m(d[0]) * m(d[1]) * m(d[2])
            Kex = sum(k(d[a]) / h[a] * np.prod([h[b] * m(d[b]) for b in range(3) if b != a]) for a in range(3))
            assert abs(M[ri, bi] - Mex) < 1e-14 * np.max(np.abs(M))
            assert abs(K[ri, bi] - Kex) < 1e-14 * np.max(np.abs(K))
            checked += 1
    assert checked > 0


@pytest.mark.parametrize("p", [2, 3])
def test_sec4_1d_comparison_1000_elements(p):
    """Sec. 4: 1D, 1000 uniform elements; the weighted Gaussian and the
    standard Gauss assemblies agree to rounding."""
    nel = (1000,)
    g = inputs.geometry(p, nel)
    M, K, _ = oracle.assemble(1, p, nel, g)
    Mg, Kg = oracle.assemble_gl(1, p, nel, g, ng=p + 1)
    # the paper's figure: maximum absolute difference of order 1e-15
    assert np.max(np.abs(M - Mg)) < 1e-15
    # both sides evaluate B-splines in global coordinates, so the local
    # coordinate (x - t_i)/h carries a relative error of about N * eps
    assert rel_err(K, Kg) < 1000 * 2.2e-16 * 4


# ------------------------------------------------------------ invariants
@pytest.mark.parametrize("p", [2, 3])
def test_row_sums_and_symmetry(p):
    nel = (5, 4, 6)
    n = [v + p for v in nel]
    g0 = inputs.geometry(p, nel)
    M, K, _ = oracle.assemble(3, p, nel, g0)
    t = [inputs.open_uniform_knots(p, v) for v in nel]
    for ri, r in enumerate(itertools.product(*[range(v) for v in reversed(n)])):
        r = tuple(reversed(r))
        assert row_index(r, n) == ri
        integral = np.prod([(t[a][r[a] + p + 1] - t[a][r[a]]) / (p + 1) for a in range(3)])
        assert abs(M[ri].sum() - integral) < 1e-15
    assert abs(M.sum() - 1.0) < 1e-13
    assert np.max(np.abs(K.sum(axis=1))) < 1e-13 * np.max(np.abs(K).sum(axis=1))
    # symmetry: entry (r, d) equals entry (r + d, -d)
    grids = np.meshgrid(*[np.arange(v) for v in n], indexing="ij")
    r = [gr.transpose(2, 1, 0).reshape(-1) for gr in grids]  # row order: r1 fastest
    for A in (M, K):
        scale = np.max(np.abs(A))
        for d in itertools.product(range(-p, p + 1), repeat=3):
            s_ = [r[a] + d[a] for a in range(3)]
            ok = np.all([(s_[a] >= 0) & (s_[a] < n[a]) for a in range(3)], axis=0)
            rows = np.nonzero(ok)[0]
            srows = s_[0][ok] + n[0] * (s_[1][ok] + n[1] * s_[2][ok])
            a1 = A[rows, band_index(d, p)]
            a2 = A[srows, band_index(tuple(-x for x in d), p)]
            assert np.max(np.abs(a1 - a2)) < 1e-14 * scale


@pytest.mark.parametrize("p", [2, 3])
def test_k_row_sums_vanish_for_any_coefficient_and_map(p):
    nel = (4, 5, 3)
    g, c = inputs.make(3, p, nel, amp=0.07, coef="exp", sigma=0.3, seed=5)
    M, K, off = oracle.assemble(3, p, nel, g, c)
    assert np.max(np.abs(K.sum(axis=1))) < 1e-13 * np.max(np.abs(K).sum(axis=1))
    assert off < 1e-13  # separable map: the off-diagonal metric vanishes


def test_linearity_in_coefficient():
    p, nel = 3, (3, 4, 3)
    g = inputs.geometry(p, nel, 0.05)
    rng = np.random.default_rng(11)
    nc = int(np.prod([v + 3 for v in nel]))
    c1, c2 = rng.random(nc) + 0.5, rng.random(nc) + 0.5
    M1, K1, _ = oracle.assemble(3, p, nel, g, c1)
    M2, K2, _ = oracle.assemble(3, p, nel, g, c2)
    M3, K3, _ = oracle.assemble(3, p, nel, g, 2.0 * c1 - 0.5 * c2)
    assert rel_err(M3, 2.0 * M1 - 0.5 * M2) < 1e-14
    assert rel_err(K3, 2.0 * K1 - 0.5 * K2) < 1e-14


# ------------------------------------------------------------ non-constant C, non-affine map
def _card(p, y, nu):
    """Explicit cardinal B-spline pieces (value nu=0, derivative nu=1)."""
    if p == 2:
        pieces = [(lambda y: y * y / 2, lambda y: y), (lambda y: (-2 * y * y + 6 * y - 3) / 2, lambda y: -2 * y + 3),
                  (lambda y: (3 - y) ** 2 / 2, lambda y: y - 3)]
    else:
        pieces = [(lambda y: y ** 3 / 6, lambda y: y * y / 2),
                  (lambda y: (-3 * y ** 3 + 12 * y * y - 12 * y + 4) / 6, lambda y: (-9 * y * y + 24 * y - 12) / 6),
                  (lambda y: (3 * y ** 3 - 24 * y * y + 60 * y - 44) / 6, lambda y: (9 * y * y - 48 * y + 60) / 6),
                  (lambda y: (4 - y) ** 3 / 6, lambda y: -(4 - y) ** 2 / 2)]
    if y <= 0 or y >= p + 1:
        return 0.0
    return pieces[int(np.floor(y))][nu](y)


def _quadratic_map_ctrl(p, nel, kappa):
    """Control values of x = xhat + kappa xhat^2: Greville abscissae plus kappa
    times the polar form of xhat^2 (average of pairwise knot products)."""
    t = inputs.open_uniform_knots(p, nel)
    n = nel + p
    out = []
    for i in range(n):
        kn = t[i + 1:i + p + 1]
        pairs = [kn[j] * kn[k] for j in range(p) for k in range(j + 1, p)]
        out.append(kn.mean() + kappa * np.mean(pairs))
    return np.array(out)


@pytest.mark.parametrize("p", [2, 3])
def test_weighted_sum_independent_evaluation(p, golden_rules):
    """For interior rows far from the boundary, evaluate the weighted sum of
    Eq. GaussQuadSys / GaussQuadSysStiff in tensor form directly from the
    printed rules, the explicit cardinal pieces, c = 1 + 0.5 x - 0.3 y + 0.2 z
    (a cubic spline reproduces it through its Greville coefficients) and the
    quadratic map x_a = xhat_a + kappa_a xhat_a^2 (J_aa = 1 + 2 kappa_a xhat_a)."""
    nel = (3 * p + 2, 3 * p + 1, 3 * p + 3)  # rows 2p..N-1-p have only cardinal columns
    n = [v + p for v in nel]
    h = [1.0 / v for v in nel]
    kappa = [0.3, -0.2, 0.45]
    g = [_quadratic_map_ctrl(p, nel[a], kappa[a]) for a in range(3)]
    lin = (1.0, 0.5, -0.3, 0.2)
    c = inputs.coefficients(nel, lambda x, y, z: lin[0] + lin[1] * x + lin[2] * y + lin[3] * z)
    M, K, off = oracle.assemble(3, p, nel, g, c)
    assert off < 1e-13  # rounding of the partition-of-unity sums in the full Jacobian

    pre = {0: "mass", 1: "stiff"}

    def rule(kind):
        t1 = float(golden_rules[f"{pre[kind]}_p{p}_tau1"])
        t2 = float(golden_rules[f"{pre[kind]}_p{p}_tau2"])
        w1 = float(golden_rules[f"{pre[kind]}_p{p}_omega1"])
        w2 = float(golden_rules[f"{pre[kind]}_p{p}_omega2"])
        if p == 2:
            return [t1, t2, 3 - t1], [w1, w2, w1]
        return [t1, t2, 4 - t2, 4 - t1], [w1, w2, w2, w1]

    rules = {0: rule(0), 1: rule(1)}
    rows = [(2 * p, 2 * p, 2 * p), (nel[0] - p - 1, 2 * p, nel[2] - p - 1)]
    for r in rows:
        assert all(2 * p <= r[a] <= nel[a] - 1 - p for a in range(3))
    for r in rows:
        ri = row_index(r, n)
        Mi = np.zeros((2 * p + 1,) * 3)
        Ki = np.zeros((2 * p + 1,) * 3)
        for term in range(4):
            kinds = [1 if term == a + 1 else 0 for a in range(3)]
            for ks in itertools.product(range(p + 1), repeat=3):
                xs, wt, J = [], 1.0, []
                for a in range(3):
                    tau, om = rules[kinds[a]]
                    y = tau[ks[a]]
                    xh = (r[a] - p + y) * h[a]
                    xs.append(xh)
                    J.append(1 + 2 * kappa[a] * xh)
                    if kinds[a] == 0:
                        wt *= h[a] * om[ks[a]] * _card(p, y, 0)
                    else:
                        wt *= om[ks[a]] * _card(p, y, 1)  # h * omega * B_r'(x), B_r' = N'/h
                cval = lin[0] + lin[1] * xs[0] + lin[2] * xs[1] + lin[3] * xs[2]
                if term == 0:
                    geo = abs(J[0] * J[1] * J[2])
                else:
                    a = term - 1
                    geo = abs(J[0] * J[1] * J[2]) / J[a] ** 2
                for d in itertools.product(range(-p, p + 1), repeat=3):
                    val = wt * cval * geo
                    for a in range(3):
                        y = rules[kinds[a]][0][ks[a]]
                        if kinds[a] == 0:
                            val *= _card(p, y - d[a], 0)
                        else:
                            val *= _card(p, y - d[a], 1) / h[a]
                    if term == 0:
                        Mi[d[2] + p, d[1] + p, d[0] + p] += val
                    else:
                        Ki[d[2] + p, d[1] + p, d[0] + p] += val
        assert np.max(np.abs(M[ri] - Mi.reshape(-1))) < 1e-13 * np.max(np.abs(Mi))
        assert np.max(np.abs(K[ri] - Ki.reshape(-1))) < 1e-13 * np.max(np.abs(Ki))


# ------------------------------------------------------------ gradient
def test_gradient_euler_and_unit_vectors():
    p, nel = 2, (3, 2, 2)
    g = inputs.geometry(p, nel, 0.06)
    nc = int(np.prod([v + 3 for v in nel]))
    rng = np.random.default_rng(2)
    c = rng.random(nc) + 0.5
    G = inputs.band_random(nel, p, 7)
    H = inputs.band_random(nel, p, 8)
    grad = oracle.gradient(3, p, nel, g, G, H)
    M, K, _ = oracle.assemble(3, p, nel, g, c)
    J = np.sum(G * K) + np.sum(H * M)
    assert abs(np.dot(grad, c) - J) < 1e-13 * abs(J)
    # dJ/dc_l = J(e_l), every coefficient
    for l in range(nc):
        e = np.zeros(nc)
        e[l] = 1.0
        Me, Ke, _ = oracle.assemble(3, p, nel, g, e)
        Jl = np.sum(G * Ke) + np.sum(H * Me)
        assert abs(grad[l] - Jl) < 1e-13 * np.max(np.abs(grad))
