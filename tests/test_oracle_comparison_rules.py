"""Pins of the oracle's comparison rules (the baselines timed beside the
weighted Gaussian rules):

* the Newton-Cotes-type weighted rules (Sec. 1 and Sec. 4 compare against
  them): nodes at the knots and element midpoints of the support, weights
  exact for all 2p+1 conditions against the exact rational moments, checked
  with B-spline pieces written out here; the symmetries and the total weight
  the exactness implies;
* assembly with either comparison rule equals the exact integrals (brute
  force element-wise Gauss-Legendre with more points) for constant
  coefficient on affine maps, like the weighted Gaussian rules;
* the Gauss-Legendre mode equals the element-wise Gauss-Legendre assembly
  with the same points for any coefficient and map (two code paths).
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_1710_01048_gb300 import inputs


def _pieces(p, y, nu):
    """Cardinal B-spline N_p (nu = 0) or N_p' (nu = 1), explicit polynomial pieces."""
    if p == 2:
        if 0 <= y < 1:
            return y * y / 2 if nu == 0 else y
        if 1 <= y < 2:
            return (-2 * y * y + 6 * y - 3) / 2 if nu == 0 else -2 * y + 3
        if 2 <= y <= 3:
            return (3 - y) ** 2 / 2 if nu == 0 else -(3 - y)
        return 0.0
    if 0 <= y < 1:
        return y ** 3 / 6 if nu == 0 else y * y / 2
    if 1 <= y < 2:
        return (-3 * y ** 3 + 12 * y * y - 12 * y + 4) / 6 if nu == 0 else (-9 * y * y + 24 * y - 12) / 6
    if 2 <= y < 3:
        return (3 * y ** 3 - 24 * y * y + 60 * y - 44) / 6 if nu == 0 else (9 * y * y - 48 * y + 60) / 6
    if 3 <= y <= 4:
        return (4 - y) ** 3 / 6 if nu == 0 else -((4 - y) ** 2) / 2
    return 0.0


def _moments():
    mom = {}
    for kind, p, d, num, den in [r[:5] for r in read_golden("moments_exact.txt")]:
        mom[(0 if kind == "mass" else 1, int(p), int(d))] = int(num) / int(den)
    return mom


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("kind", [0, 1])
def test_nc_rule_nodes_and_exactness(p, kind):
    y, v, res = oracle.rule_nc(p, kind)
    assert np.allclose(y, 0.5 * np.arange(1, 2 * p + 2), atol=0, rtol=0)
    assert res < 1e-14
    mom = _moments()
    for d in range(-p, p + 1):
        s = sum(v[k] * _pieces(p, y[k] - d, kind) for k in range(2 * p + 1))
        assert abs(s - mom[(kind, p, abs(d))]) < 1e-14


@pytest.mark.parametrize("p", [2, 3])
def test_nc_rule_symmetries_and_total_weight(p):
    _, vm, _ = oracle.rule_nc(p, 0)
    _, vs, _ = oracle.rule_nc(p, 1)
    # N is symmetric about the centre, N' antisymmetric
    assert np.allclose(vm, vm[::-1], rtol=0, atol=1e-15)
    assert np.allclose(vs, -vs[::-1], rtol=0, atol=1e-15)
    assert vs[p] == 0.0
    # summing the mass conditions over d: the translates sum to one on the
    # support, so the weights sum to the integral of N, which is 1
    assert abs(vm.sum() - 1.0) < 1e-15
    # the mass weights are positive
    assert np.all(vm > 0)


@pytest.mark.parametrize("mode", ["gl", "nc"])
@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("nel", [(1, 2, 1), (3, 3, 2), (8, 4, 5)])
def test_comparison_rules_exact_on_affine_maps(mode, p, nel):
    alpha = np.array([1.25, 0.5, 2.0])
    g = [alpha[a] * gi + 0.3 for a, gi in enumerate(inputs.geometry(p, nel))]
    M, K = oracle.assemble_rule(mode, 3, p, nel, g)
    Mg, Kg = oracle.assemble_gl(3, p, nel, g, ng=p + 2)
    # rounding only: entries sum up to (p+1)^6 point terms in both
    # assemblies (a few 1e-15 relative each), and the NC weights come from a
    # linear solve with condition number ~30 (p = 2) to ~600 (p = 3)
    tol = 5e-14 if mode == "gl" else 1e-13
    assert np.max(np.abs(M - Mg)) < tol * np.max(np.abs(Mg))
    assert np.max(np.abs(K - Kg)) < tol * np.max(np.abs(Kg))


@pytest.mark.parametrize("p", [2, 3])
def test_gl_mode_equals_elementwise_gauss_legendre(p):
    nel = (7, 5, 6)
    g, c = inputs.make(3, p, nel, 0.06, "exp", 0.1, seed=3)
    M, K = oracle.assemble_rule("gl", 3, p, nel, g, c)
    Mg, Kg = oracle.assemble_gl(3, p, nel, g, c, ng=p + 1)
    assert np.max(np.abs(M - Mg)) < 1e-13 * np.max(np.abs(Mg))
    assert np.max(np.abs(K - Kg)) < 1e-13 * np.max(np.abs(Kg))


@pytest.mark.parametrize("p", [2, 3])
def test_nc_differs_from_wq_for_variable_coefficient(p):
    # both approximate the same integrals: close, but not equal, for a
    # non-constant coefficient on a non-affine map (Remark closing Sec. 3)
    nel = (7, 6, 5)
    g, c = inputs.make(3, p, nel, 0.06, "exp", 0.1, seed=4)
    Mw, Kw, _ = oracle.assemble(3, p, nel, g, c)
    Mn, Kn = oracle.assemble_rule("nc", 3, p, nel, g, c)
    Mx, Kx = oracle.assemble_gl(3, p, nel, g, c, ng=p + 3)
    for A, X in ((Mw, Mx), (Mn, Mx), (Kw, Kx), (Kn, Kx)):
        e = np.max(np.abs(A - X)) / np.max(np.abs(X))
        assert 1e-12 < e < 1e-2
