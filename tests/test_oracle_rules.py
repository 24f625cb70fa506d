"""Pins of the oracle's 1D building blocks against what the paper and the
mathematics fix: printed 20-digit rules, exact rational moments, closed
forms, the paper's own reduced systems, Gauss-Legendre facts, explicit
cardinal B-spline pieces, and the rejected spurious root."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import read_golden

MASS, STIFF = 0, 1


# ---------------------------------------------------------------- Gauss-Legendre
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8])
def test_gauss_legendre_exact_on_monomials(n):
    x, w = oracle.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    assert np.all(np.diff(x) > 0)


def test_gauss_legendre_closed_forms():
    x, w = oracle.gauss_legendre(2)
    ulp2 = 2.3e-16  # two units in the last place near 1
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=ulp2, rtol=0)
    x, w = oracle.gauss_legendre(3)
    assert np.allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], atol=ulp2, rtol=0)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=4 * ulp2, rtol=0)


# ---------------------------------------------------------------- B-splines
def _n2(y):
    if 0 <= y < 1:
        return y * y / 2
    if 1 <= y < 2:
        return (-2 * y * y + 6 * y - 3) / 2
    if 2 <= y <= 3:
        return (3 - y) ** 2 / 2
    return 0.0


def _n3(y):
    if 0 <= y < 1:
        return y ** 3 / 6
    if 1 <= y < 2:
        return (-3 * y ** 3 + 12 * y * y - 12 * y + 4) / 6
    if 2 <= y < 3:
        return (3 * y ** 3 - 24 * y * y + 60 * y - 44) / 6
    if 3 <= y <= 4:
        return (4 - y) ** 3 / 6
    return 0.0


@pytest.mark.parametrize("p,fn", [(2, _n2), (3, _n3)])
def test_cardinal_matches_explicit_pieces(p, fn):
    for y in np.linspace(-0.5, p + 1.5, 97):
        assert abs(oracle.cardinal(p, y) - fn(y)) < 1e-14  # monomial pieces cancel to ~2e-15
        h = 1e-6
        if all(abs(y - k) > 1e-3 for k in range(p + 2)):
            fd = (fn(y + h) - fn(y - h)) / (2 * h)
            assert abs(oracle.cardinal(p, y, 1) - fd) < 1e-8


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("nel", [1, 2, 5, 9])
def test_open_knot_partition_of_unity(p, nel):
    n = nel + p
    for x in np.linspace(0, 1, 53):
        vals = [oracle.bspline(p, nel, i, x) for i in range(n)]
        ders = [oracle.bspline(p, nel, i, x, 1) for i in range(n)]
        assert abs(sum(vals) - 1.0) < 1e-14
        assert abs(sum(ders)) < 1e-11 * nel
        assert min(vals) >= 0.0


def test_interior_bspline_is_translate_of_cardinal():
    p, nel = 3, 10
    h = 1.0 / nel
    for r in range(p, nel):
        for y in np.linspace(0.05, p + 0.95, 17):
            x = (r - p + y) * h
            assert abs(oracle.bspline(p, nel, r, x) - _n3(y)) < 1e-14


# ---------------------------------------------------------------- moments
def test_moments_exact_rationals():
    for kind, p, d, num, den in [r[:5] for r in read_golden("moments_exact.txt")]:
        exact = int(num) / int(den)
        nu = MASS if kind == "mass" else STIFF
        got = oracle.moment(int(p), nu, int(d))
        assert abs(got - exact) < 2e-16 * max(1.0, abs(exact)) * 4, (kind, p, d, got, exact)
        # beyond the overlap the moment is zero, and m(-d) = m(d)
        assert abs(oracle.moment(int(p), nu, -int(d)) - got) < 1e-16 * 4
    for p in (2, 3):
        assert oracle.moment(p, MASS, p + 1) == 0.0
        assert oracle.moment(p, STIFF, p + 1) == 0.0


def test_moments_are_degree_2p1_cardinal_at_integers():
    # m(d) = N_{2p+1}(p+1+d): evaluate the higher-degree cardinal B-spline by its
    # explicit truncated-power form with exact rationals.
    def n_card(n, x):
        s = Fraction(0)
        for j in range(n + 2):
            t = x - j
            if t > 0:
                s += (-1) ** j * math.comb(n + 1, j) * Fraction(t) ** n
        return s / math.factorial(n)

    for p in (2, 3):
        for d in range(p + 1):
            assert abs(oracle.moment(p, MASS, d) - float(n_card(2 * p + 1, p + 1 + d))) < 1e-15


# ---------------------------------------------------------------- rules
def _printed(golden, kind, p):
    pre = "mass" if kind == MASS else "stiff"
    t1 = float(golden[f"{pre}_p{p}_tau1"])
    t2 = float(golden[f"{pre}_p{p}_tau2"])
    w1 = float(golden[f"{pre}_p{p}_omega1"])
    w2 = float(golden[f"{pre}_p{p}_omega2"])
    if p == 2:
        return np.array([t1, t2, 3 - t1]), np.array([w1, w2, w1])
    return np.array([t1, t2, 4 - t2, 4 - t1]), np.array([w1, w2, w2, w1])


# Newton converges to a root whose accuracy is set by the rounding of the residual
# (a few 1e-17 for these moments) divided by the local slope of the system; the
# observed worst cases are 4 units in the last place (omega_2 of the p=2 mass rule,
# 4.4e-16).  1e-15 is far inside what the 1e-12 assembly tolerance needs.
RULE_TOL = 1e-15


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("kind", [MASS, STIFF])
def test_rule_matches_printed_values(golden_rules, p, kind):
    tau, om, res = oracle.rule(p, kind)
    pt, pw = _printed(golden_rules, kind, p)
    assert np.all(np.abs(tau - pt) < RULE_TOL * np.maximum(1.0, pt)), (tau, pt)
    assert np.all(np.abs(om - pw) < RULE_TOL * np.maximum(1.0, pw)), (om, pw)
    assert res < 1e-15
    # minimal point count: p+1 nodes, one per element of the support (Sec. 3, Eq. Reduction)
    assert len(tau) == p + 1
    for k in range(p + 1):
        assert k < tau[k] < k + 1


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("kind", [MASS, STIFF])
def test_printed_rules_pass_exactness(golden_rules, p, kind):
    pt, pw = _printed(golden_rules, kind, p)
    ok, res = oracle.rule_check(p, kind, pt, pw, 1e-15)
    assert ok, res


def test_stiffness_closed_forms():
    tau, om, _ = oracle.rule(2, STIFF)
    assert abs(tau[0] - 0.75) < 2.3e-16 and abs(om[0] - 8 / 9) < 2.3e-16
    tau, om, _ = oracle.rule(3, STIFF)
    t1 = 0.5 - math.sqrt(225 - 30 * math.sqrt(30)) / 30  # Eq. CubicStiffTau1, smaller root
    assert abs(tau[0] - t1) < RULE_TOL
    assert om[0] == 1.0
    # tau_1 solves 30 x^4 w - 60 x^3 w + 30 x^2 w - 1 = 0 with w = 1 (Eq. CubicStiffTau1W)
    x = tau[0]
    assert abs(30 * x ** 4 - 60 * x ** 3 + 30 * x ** 2 - 1) < 1e-14


def test_paper_reduced_systems_hold_at_oracle_rules():
    """The reduced symmetric systems printed in Sec. 3, evaluated at the
    oracle's rules.  The third equation of Eq. CubicQuadratureStiff is read
    with the factor (3 tau_1^2 - 2 tau_1 - 1) (the printed tau_2 leaves a
    residual of about 0.03), and the third equation of
    Eq. QuadraticQuadratureStiff holds in the form 2 omega_1 tau_1^2 = 1
    because B_j' vanishes at the middle node."""
    (t1, _, _), (w1, w2, _), _ = oracle.rule(2, MASS)
    eqs = [0.25 * w1 * t1 ** 2 * (1 - t1) ** 2 - 1 / 120,
           0.25 * w1 * t1 ** 2 * (-2 * t1 ** 2 + 2 * t1 + 1) + 3 / 32 * w2 - 13 / 60,
           0.5 * w1 * t1 ** 4 + 9 / 16 * w2 - 11 / 20]
    assert max(abs(e) for e in eqs) < 1e-15

    tau, om, _ = oracle.rule(3, MASS)
    t1, t2, w1, w2 = tau[0], tau[1], om[0], om[1]
    q = t2 ** 3 - 4 * t2 ** 2 + 4 * t2 - 4 / 3
    eqs = [w1 * t1 ** 3 * (1 - t1) ** 3 / 36 - 1 / 5040,
           w1 * t1 ** 3 * (t1 ** 3 / 12 - t1 ** 2 / 6 + 1 / 9) - w2 * (2 - t2) ** 3 * q / 12 - 1 / 42,
           -w1 * t1 ** 3 * (t1 ** 3 - t1 ** 2 - t1 - 1 / 3) / 12
           - w2 * (t2 ** 3 - 4.5 * t2 ** 2 + 6 * t2 - 1.5) * q / 3 - 397 / 1680,
           w1 * t1 ** 6 / 18 + 0.5 * w2 * q ** 2 - 151 / 315]
    assert max(abs(e) for e in eqs) < 1e-15

    (t1, _, _), (w1, w2, _), _ = oracle.rule(2, STIFF)
    # first two equations with the sign of the moment restored on the second
    eqs = [w1 * t1 * (1 - t1) - 1 / 6, w1 * t1 * (1 - 2 * t1) - (-1 / 3), 2 * w1 * t1 ** 2 - 1]
    assert max(abs(e) for e in eqs) < 1e-15

    tau, om, _ = oracle.rule(3, STIFF)
    t1, t2, w1, w2 = tau[0], tau[1], om[0], om[1]
    eqs = [0.25 * w1 * t1 ** 2 * (1 - t1) ** 2 - 1 / 120,
           0.25 * w1 * t1 ** 3 * (4 - 3 * t1) - 0.75 * w2 * (t2 - 2) ** 3 * (t2 - 2 / 3) - 1 / 5,
           0.25 * w1 * t1 ** 2 * (3 * t1 ** 2 - 2 * t1 - 1) + 3 * w2 * (t2 - 1) * (t2 - 2) ** 2 * (t2 - 2 / 3) - 1 / 8,
           0.5 * w1 * t1 ** 4 + 4.5 * w2 * (t2 - 2) ** 2 * (t2 - 2 / 3) ** 2 - 2 / 3]
    assert max(abs(e) for e in eqs) < 1e-14
    printed_third = 0.25 * w1 * t1 ** 2 * (3 * t2 ** 2 - 2 * t2 - 1) + 3 * w2 * (t2 - 1) * (t2 - 2) ** 2 * (t2 - 2 / 3) - 1 / 8
    assert abs(printed_third) > 1e-2


def test_spurious_cubic_root_rejected(golden_rules):
    t1 = float(golden_rules["spurious_p3_tau1"])
    t2 = float(golden_rules["spurious_p3_tau2"])
    w1 = float(golden_rules["spurious_p3_omega1"])
    w2 = float(golden_rules["spurious_p3_omega2"])
    ok, res = oracle.rule_check(3, MASS, [t1, t2, 4 - t2, 4 - t1], [w1, w2, w2, w1])
    assert not ok
    assert res > 1e-2  # fails true piecewise exactness, not just the node-location test


def test_paper_initial_guess_does_not_give_a_wrong_rule():
    """From the start of Eq. WQcubicIni, Newton on the true piecewise system
    either fails or finds the printed rule; it never returns a rule that
    passes the checks with a node outside its element (Sec. 3.1.2)."""
    st, tau, om, res = oracle.rule_newton(3, MASS, [1 / 3, 5 / 3, 1.0, 1.0], [0, 1, 2, 3])
    if st == 0:
        ref, _, _ = oracle.rule(3, MASS)
        assert np.max(np.abs(tau - ref)) < 1e-14


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("kind", [MASS, STIFF])
def test_rule_exact_on_interior_spline_space(p, kind):
    """The rule integrates every degree-p C^{p-1} spline on the support of
    the weight function exactly (Eq. GaussQuadSys / GaussQuadSysStiff),
    e.g. random combinations of the 2p+1 translates."""
    tau, om, _ = oracle.rule(p, kind)
    rng = np.random.default_rng(3)
    coeffs = rng.standard_normal(2 * p + 1)
    ds = np.arange(-p, p + 1)

    def f(y):
        return sum(c * oracle.cardinal(p, y - d, kind) for c, d in zip(coeffs, ds))

    quad = sum(om[k] * oracle.cardinal(p, tau[k], kind) * f(tau[k]) for k in range(p + 1))
    exact = sum(c * oracle.moment(p, kind, int(d)) for c, d in zip(coeffs, ds))
    assert abs(quad - exact) < 1e-14


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("nel", [1, 2, 3, 7])
def test_row_points_structure(p, nel):
    """Interior rows: p+1 points, one per element of supp B_r.  Boundary
    rows: p+1 Gauss-Legendre points on each element of supp B_r."""
    h = 1.0 / nel
    for kind in (MASS, STIFF):
        for r in range(nel + p):
            x, W = oracle.row_points(p, nel, kind, r)
            elo, ehi = max(0, r - p), min(nel - 1, r)
            elems = np.floor(x / h).astype(int)
            assert elems.min() >= elo and elems.max() <= ehi
            if p <= r <= nel - 1:
                assert len(x) == p + 1
                assert sorted(elems.tolist()) == list(range(r - p, r + 1))
            else:
                assert len(x) == (ehi - elo + 1) * (p + 1)
            if kind == MASS:
                # weights integrate B_r itself: sum W = int B_r = (t_{r+p+1}-t_r)/(p+1)... times 1
                t = np.concatenate([np.zeros(p + 1), np.arange(1, nel) / nel, np.ones(p + 1)])
                assert abs(W.sum() - (t[r + p + 1] - t[r]) / (p + 1)) < 1e-15
