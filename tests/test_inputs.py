"""The seeded synthetic inputs follow their stated recipes (CPU only).

The geometry and coefficient generators hold no arithmetic of the method,
but every parity test and the benchmark consume them, so their recipe is
checked here against the mathematics it relies on: Greville abscissae
reproduce linear maps (so amp = 0 is the identity and an affine net is the
affine map), the perturbed maps keep J_aa >= 1 - amp * pi, the coefficient
spline is f at the Greville points times lognormal noise in x-fastest order,
and the named workloads and the batch have the documented sizes."""
import math

import numpy as np
import pytest

import oracle
from paper_1710_01048_gb300 import inputs


def spline_1d(p, nel, ctrl, x, deriv=0):
    return sum(ctrl[i] * oracle.bspline(p, nel, i, x, deriv) for i in range(nel + p))


@pytest.mark.parametrize("p", [2, 3])
def test_greville_reproduces_the_identity(p):
    nel = 7
    g = inputs.geometry(p, (nel,), 0.0)[0]
    assert np.array_equal(g, inputs.greville(p, nel))
    rng = np.random.default_rng(3)
    for x in rng.uniform(0.0, 1.0, 25):
        assert abs(spline_1d(p, nel, g, x) - x) <= 1e-14
        assert abs(spline_1d(p, nel, g, x, 1) - 1.0) <= 1e-13


@pytest.mark.parametrize("p", [2, 3])
def test_perturbed_map_jacobian_bound(p):
    amp, nel = 0.08, 9
    g = inputs.geometry(p, (nel, nel), amp)
    assert np.array_equal(g[0], g[1])
    xs = np.linspace(0.0, 1.0, 301)
    J = np.array([spline_1d(p, nel, g[0], x, 1) for x in xs])
    assert J.min() >= 1.0 - amp * math.pi - 1e-12
    # the map keeps the end points and is increasing
    assert abs(spline_1d(p, nel, g[0], 0.0)) <= 1e-15 and abs(spline_1d(p, nel, g[0], 1.0) - 1.0) <= 1e-14


def test_coefficient_layout_is_x_fastest():
    nel = (3, 5, 7)
    c = inputs.coefficients(nel, lambda x, y, z: x + 10.0 * y + 100.0 * z)
    xs = [inputs.greville(3, v) for v in nel]
    n = [v + 3 for v in nel]
    assert c.shape == (n[0] * n[1] * n[2],)
    for l1, l2, l3 in [(0, 0, 0), (5, 0, 0), (0, 7, 0), (0, 0, 9), (2, 4, 6), (5, 7, 9)]:
        want = xs[0][l1] + 10.0 * xs[1][l2] + 100.0 * xs[2][l3]
        assert c[l1 + n[0] * (l2 + n[1] * l3)] == pytest.approx(want, abs=1e-14)


def test_coefficient_noise_recipe_and_seeds():
    nel = (16, 16, 16)
    c = inputs.coefficients(nel, inputs.exp_sum, seed=0, sigma=0.1)
    c_again = inputs.coefficients(nel, inputs.exp_sum, seed=0, sigma=0.1)
    c_other = inputs.coefficients(nel, inputs.exp_sum, seed=1, sigma=0.1)
    assert np.array_equal(c, c_again) and not np.array_equal(c, c_other)
    base = inputs.coefficients(nel, inputs.exp_sum)
    z = np.log(c / base) / 0.1  # the standard normal draws
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1.0) < 0.05
    # the draws follow default_rng(seed) in storage order
    assert np.allclose(z, np.random.default_rng(0).standard_normal(z.size), atol=1e-9)
    assert np.all(c > 0)


def test_named_workloads_have_the_documented_sizes():
    w = inputs.WORKLOADS
    assert (w["2d_p3_32"]["dim"], w["2d_p3_32"]["p"], w["2d_p3_32"]["nel"]) == (2, 3, (32, 32))
    assert w["2d_p3_32"]["coef"] == "sincos" and w["2d_p3_32_c1"]["coef"] == "one"
    for name, p, n in [("3d_p2_64", 2, 64), ("3d_p3_64", 3, 64), ("3d_p3_128", 3, 128), ("3d_p3_96", 3, 96),
                       ("3d_p3_12", 3, 12)]:
        assert (w[name]["dim"], w[name]["p"], w[name]["nel"]) == (3, p, (n, n, n))
        assert (w[name]["amp"], w[name]["coef"], w[name]["sigma"], w[name]["seed"]) == (0.05, "exp", 0.1, 0)
    spec, g, c = inputs.workload("3d_p3_12")
    assert [len(x) for x in g] == [15, 15, 15] and c.size == 15 ** 3


def test_batch_patch_recipe():
    specs = inputs.batch_patches(256, seed=0)
    assert len(specs) == 256
    nel = np.array([s["nel"] for s in specs])
    ps = np.array([s["p"] for s in specs])
    amps = np.array([s["amp"] for s in specs])
    assert nel.min() >= 8 and nel.max() <= 48
    # log-uniform per direction: the mean of log(nel) near the midpoint of [log 8, log 48]
    assert abs(np.log(nel).mean() - 0.5 * (math.log(8) + math.log(48))) < 0.1
    assert set(ps.tolist()) == {2, 3} and abs((ps == 3).mean() - 0.5) < 0.1
    assert amps.min() >= 0.0 and amps.max() <= 0.08
    for s in specs[:4]:
        assert [len(x) for x in s["geom"]] == [v + s["p"] for v in s["nel"]]
        assert s["coef"].size == int(np.prod([v + 3 for v in s["nel"]]))
    again = inputs.batch_patches(4, seed=0)
    assert all(np.array_equal(a["coef"], b["coef"]) and a["nel"] == b["nel"] for a, b in zip(again, specs[:4]))


@pytest.mark.parametrize("dim", [2, 3])
def test_band_mask_counts_in_range_columns(dim):
    p, nel = 3, (4, 2, 5)[:dim]
    m = inputs.band_mask(nel, p)
    n = [v + p for v in nel]
    assert m.shape == (int(np.prod(n)), (2 * p + 1) ** dim)
    per_dir = [sum(min(r + p, k - 1) - max(r - p, 0) + 1 for r in range(k)) for k in n]
    assert m.sum() == np.prod(per_dir)
    # row 0 (the corner): its diagonal entry (every offset 0) is in range, offset -p in any direction is not
    corner = m[0].reshape([2 * p + 1] * dim)
    assert corner[(p,) * dim] == 1.0
    assert corner.sum() == (p + 1) ** dim


def test_affine_net_is_the_affine_map():
    p, nel = 3, (3, 4)
    net = inputs.full_net(p, nel, "affine")
    A, b = inputs.AFFINE[2]
    n = [v + p for v in nel]
    comps = net.reshape(2, n[1], n[0])  # [a][i2][i1]
    rng = np.random.default_rng(5)
    for x, y in rng.uniform(0.0, 1.0, (10, 2)):
        B1 = np.array([oracle.bspline(p, nel[0], i, x) for i in range(n[0])])
        B2 = np.array([oracle.bspline(p, nel[1], i, y) for i in range(n[1])])
        pt = [B2 @ comps[a] @ B1 for a in range(2)]
        assert np.allclose(pt, A @ np.array([x, y]) + b, atol=1e-14)
    sep = inputs.net_from_separable(p, nel, inputs.geometry(p, nel, 0.0))
    assert np.allclose(sep.reshape(2, n[1], n[0])[0][0], inputs.greville(p, nel[0]))
