"""Host-side tests of libwq (no GPU): the C-ABI loads and exports every
symbol of include/wq.h; the host rule solver reproduces the paper's rules;
the per-row tables agree with the oracle's; bookkeeping and argument
checks."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from conftest import ROOT, read_golden
from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import build as wqbuild
from paper_1710_01048_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def built():
    wqbuild.build()


def header_functions():
    with open(os.path.join(ROOT, "include", "wq.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wq_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = wq.library()
    declared = header_functions()
    assert len(declared) >= 16
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(wq.EXPORTS) == declared


def test_status_strings():
    for s in range(10):
        assert len(wq.wq_status_string(s)) >= 2 and wq.wq_status_string(s) != "unknown status"
    assert wq.wq_version() >= 100


def _printed(golden, kind, p):
    pre = "mass" if kind == 0 else "stiff"
    t1, t2 = float(golden[f"{pre}_p{p}_tau1"]), float(golden[f"{pre}_p{p}_tau2"])
    w1, w2 = float(golden[f"{pre}_p{p}_omega1"]), float(golden[f"{pre}_p{p}_omega2"])
    if p == 2:
        return np.array([t1, t2, 3 - t1]), np.array([w1, w2, w1])
    return np.array([t1, t2, 4 - t2, 4 - t1]), np.array([w1, w2, w2, w1])


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("kind", [0, 1])
def test_host_rules_match_printed(golden_rules, p, kind):
    tau, om = wq.wq_rule_1d(p, kind)
    pt, pw = _printed(golden_rules, kind, p)
    # four units in the last place of values up to 4
    assert np.all(np.abs(tau - pt) <= 4 * np.spacing(np.maximum(pt, 1.0))), tau - pt
    assert np.all(np.abs(om - pw) <= 4 * np.spacing(np.maximum(pw, 1.0))), om - pw


def test_host_rule_bad_start_is_reported(golden_rules):
    # the start of Eq. WQcubicIni: never a wrong rule
    st, tau, om = wq.wq_rule_1d_from(3, 0, [1 / 3, 5 / 3, 1.0, 1.0])
    if st == wq.WQ_OK:
        pt, _ = _printed(golden_rules, 0, 3)
        assert np.max(np.abs(tau - pt)) < 1e-14
    else:
        assert st == wq.WQ_ERR_NO_CONVERGENCE
    # starting at the spurious root of Sec. 3.1.2 (tau_2 outside [1, 2])
    st, _, _ = wq.wq_rule_1d_from(3, 0, [float(golden_rules[k]) for k in
                                         ("spurious_p3_tau1", "spurious_p3_tau2", "spurious_p3_omega1",
                                          "spurious_p3_omega2")])
    assert st == wq.WQ_ERR_NO_CONVERGENCE
    # a start far outside: diverges or fails the checks
    st, _, _ = wq.wq_rule_1d_from(3, 0, [5.0, -3.0, 100.0, -7.0])
    assert st == wq.WQ_ERR_NO_CONVERGENCE


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("nel", [1, 2, 3, 5, 11])
def test_host_row_tables_match_oracle(p, nel):
    R = wq.Rules(2, p, (nel, 4), device=False)
    for kind in (0, 1):
        for r in range(nel + p):
            x, W, e = R.row(0, kind, r)
            xo, Wo = oracle.row_points(p, nel, kind, r)
            assert len(x) == len(xo)
            assert np.max(np.abs(x - xo)) < 1e-15
            assert np.max(np.abs(W - Wo)) < 1e-14 * max(1.0, np.max(np.abs(Wo)))
            assert np.all(e == np.floor(x * nel).astype(int))
    R.close()


def test_bookkeeping_counts():
    for p in (2, 3):
        for nel in [(4, 5), (6, 7, 8), (64, 64, 64)]:
            R = wq.Rules(len(nel), p, nel, device=False)
            n = [v + p for v in nel]
            assert R.rows == int(np.prod(n))
            assert R.band == (2 * p + 1) ** len(nel)
            assert R.nnz == int(np.prod([v * (2 * p + 1) - p * (p + 1) for v in n]))
            assert R.ncoef == int(np.prod([v + 3 for v in nel]))
            R.close()
    # 64^3 cubic: 95.4M non-zeros per matrix
    R = wq.Rules(3, 3, (64, 64, 64), device=False)
    assert R.nnz == 457 ** 3
    fl, cf = R.flops()
    # interior rows: 4 terms' sum-factorised non-zero multiply-adds
    interior = 2 * (3 * (4 * 4 * 4 * 4 + 4 * 7 * 4 * 4) + (64 + 112) + 49 * 4 * 4 * 3 + 0.5 * 49 * 4)
    assert fl > interior * R.rows * 0.9
    R.close()


def test_point_count_reduction_and_evaluation_counts():
    """Sec. 3, Eq. Reduction and the comparison values of Sec. 4: per
    direction an interior row uses p+1 points against the 2p+1 of a
    Newton-Cotes-type weighted rule; counting the non-vanishing basis
    evaluations (knots lose one function), the 2D ratios are (13/9)^2 = 2.09
    and (25/16)^2 = 2.44 for p = 2, 3."""
    printed = {int(r[0]): float(r[1]) for r in read_golden("counts_printed.txt")}
    for p in (2, 3):
        R = wq.Rules(2, p, (100, 100), device=False)
        r = 50
        x, W, e = R.row(0, 0, r)
        assert len(x) == p + 1
        wq_evals = len(x) * (p + 1)  # each point in one element: p+1 non-zero B-splines
        nc_points = 2 * p + 1  # interior knots and midpoints of supp B_r where B_r > 0
        nc_knots = p  # interior knots of the support: p non-zero B-splines there
        nc_evals = (nc_points - nc_knots) * (p + 1) + nc_knots * p
        ratio = (nc_evals / wq_evals) ** 2
        assert abs(ratio - printed[p]) < 0.01
        assert abs(((p + 1) / (2 * p + 1)) ** 2 - (len(x) / nc_points) ** 2) < 1e-15
        R.close()


def test_argument_validation():
    with pytest.raises(wq.WqError) as ei:
        wq.Rules(4, 3, (4, 4, 4), device=False)
    assert ei.value.status == wq.WQ_ERR_UNSUPPORTED
    with pytest.raises(wq.WqError) as ei:
        wq.Rules(3, 5, (4, 4, 4), device=False)
    assert ei.value.status == wq.WQ_ERR_UNSUPPORTED
    with pytest.raises(wq.WqError) as ei:
        wq.Rules(3, 3, (4, 0, 4), device=False)
    assert ei.value.status == wq.WQ_ERR_ARG
    R = wq.Rules(3, 2, (3, 3, 3), device=False)
    # assembly on a host-only object is an argument error, before any CUDA call
    st = wq.wq_assemble_mass(R.handle, [1, 1, 1], None, wq.WQ_FP64, 1, 0, 1, None)
    assert st == wq.WQ_ERR_ARG
    with pytest.raises(wq.WqError):
        R.row(3, 0, 0)
    R.close()


def test_injected_device_allocation_failure(monkeypatch):
    # the allocation-failure hook fails the device upload before any CUDA call
    monkeypatch.setenv("WQ_FAULT_DEVICE_ALLOC", "1")
    with pytest.raises(wq.WqError) as ei:
        wq.Rules(3, 3, (4, 4, 4), device=True)
    assert ei.value.status == wq.WQ_ERR_OOM
    # host tables are unaffected
    R = wq.Rules(3, 3, (4, 4, 4), device=False)
    assert R.rows == 7 ** 3
    R.close()


def test_apply_and_load_reject_host_only_rules():
    R = wq.Rules(3, 2, (3, 3, 3), device=False)
    st = wq.wq_apply_mass_stiffness(R.handle, [1, 1, 1], None, wq.WQ_FP64, 1, 1, 1, 0, 1, None)
    assert st == wq.WQ_ERR_ARG
    st = wq.wq_assemble_load(R.handle, [1, 1, 1], None, wq.WQ_FP64, 1, 0, 1, None)
    assert st == wq.WQ_ERR_ARG
    R.close()


def test_band_nnz_rows_matches_mask():
    # the closed-form CSR row pointer against the band mask's running sum
    rng = np.random.default_rng(0)
    for dim, p, nel in [(3, 3, (5, 4, 6)), (3, 2, (1, 1, 1)), (2, 3, (7, 3)), (3, 3, (12, 2, 9)), (2, 2, (1, 5))]:
        R = wq.Rules(dim, p, nel, device=False)
        m = inputs.band_mask(nel, p)
        cs = np.concatenate([[0], np.cumsum(m.sum(1))]).astype(np.int64)
        rows = m.shape[0]
        for _ in range(40):
            rb = int(rng.integers(0, rows + 1))
            re = int(rng.integers(rb, rows + 1))
            assert wq.wq_band_nnz_rows(R.handle, rb, re) == cs[re] - cs[rb]
        assert wq.wq_band_nnz_rows(R.handle, 0, rows) == R.nnz
        assert wq.wq_band_nnz_rows(R.handle, 3, 2) == -1
        R.close()


@pytest.mark.parametrize("p", [2, 3])
def test_comparison_rule_tables_match_oracle(p):
    # Newton-Cotes-type rows: nodes (r - p + y_k) h, W = h v_k (mass) or v_k
    # (stiffness), from the oracle's rule; Gauss-Legendre rows: the oracle's
    # boundary-row form on every row
    nel = 11
    h = 1.0 / nel
    gx, gw = oracle.gauss_legendre(p + 1)
    for mode in ("nc", "gl"):
        R = wq.Rules(2, p, (nel, 4), device=False, rule=mode)
        for kind in (0, 1):
            y, v, _ = oracle.rule_nc(p, kind)
            for r in range(nel + p):
                x, W, e = R.row(0, kind, r)
                if mode == "nc" and p <= r <= nel - 1:
                    assert len(x) == 2 * p + 1
                    assert np.max(np.abs(x - (r - p + y) * h)) < 1e-15
                    Wo = (h if kind == 0 else 1.0) * v
                    assert np.max(np.abs(W - Wo)) < 1e-14 * np.max(np.abs(Wo))
                    assert np.array_equal(e, r - p + np.floor(y).astype(int))
                else:
                    elo, ehi = max(0, r - p), min(nel - 1, r)
                    xs = np.concatenate([(el + 0.5 * (gx + 1.0)) * h for el in range(elo, ehi + 1)])
                    Wo = np.array([0.5 * h * gw[g % (p + 1)] * oracle.bspline(p, nel, r, xq, kind)
                                   for g, xq in enumerate(xs)])
                    assert len(x) == len(xs)
                    assert np.max(np.abs(x - xs)) < 1e-15
                    assert np.max(np.abs(W - Wo)) < 1e-13 * max(1.0, np.max(np.abs(Wo)))
        R.close()
    with pytest.raises(wq.WqError):
        wq.wq_rules_build(2, p, (4, 4), wq.WQ_RULES_GAUSS_LEGENDRE | wq.WQ_RULES_NEWTON_COTES)
    with pytest.raises(wq.WqError):
        wq.wq_rules_build(2, p, (4, 4), 16)


def test_comparison_rule_point_counts():
    # points per interior row and direction: p+1 (weighted Gaussian), 2p+1
    # (Newton-Cotes type: knots and midpoints), (p+1)^2 (Gauss-Legendre on the
    # p+1 elements of the support)
    for p in (2, 3):
        for mode, cnt in (("wq", p + 1), ("nc", 2 * p + 1), ("gl", (p + 1) ** 2)):
            R = wq.Rules(2, p, (20, 20), device=False, rule=mode)
            for kind in (0, 1):
                assert all(len(R.row(0, kind, r)[0]) == cnt for r in range(p, 20))
            R.close()


@pytest.mark.parametrize("p", [2, 3])
def test_boundary_weighted_rules_match_the_oracle(p):
    # WQ_RULES_BOUNDARY_WEIGHTED: the boundary rows' points (padding of zero
    # weight dropped) are the oracle's weighted rules, to the solves'
    # accuracy; interior rows are unchanged; the two kinds' points lie in the
    # same elements one by one (the kernels take both from one list)
    import oracle

    for N in (2 * p + 1, 13):
        n = N + p
        R = wq.Rules(2, p, (N, N), device=False, rule="wqb")
        Rw = wq.Rules(2, p, (N, N), device=False)
        for r in range(n):
            xs = []
            for kind in (0, 1):
                x, W, e = R.row(0, kind, r)
                xs.append(e)
                # padding points carry W = 0 in boundary rows (an interior
                # p = 2 stiffness rule has a genuine zero weight at its centre)
                keep = (W != 0.0) if (r < p or r > N - 1) else np.ones(len(W), bool)
                xo, Wo = oracle.row_points(p, N, kind, r, "wqb")
                o = np.argsort(x[keep])
                oo = np.argsort(xo)
                assert len(xo) == keep.sum(), (N, r, kind)
                assert np.max(np.abs(x[keep][o] - xo[oo])) <= 1e-12
                assert np.max(np.abs(W[keep][o] - Wo[oo])) <= 1e-12 * max(1.0, np.max(np.abs(Wo)))
                if p <= r <= N - 1:
                    xw, Ww, _ = Rw.row(0, kind, r)
                    assert np.array_equal(x, xw) and np.array_equal(W, Ww)
            assert np.array_equal(xs[0], xs[1])
        R.close()
        Rw.close()


def test_boundary_weighted_rules_fewer_points_and_flags():
    # p = 3: boundary rows 0 and 2 drop from 4 and 12 points to 2 and 3; the
    # flag does not combine with the comparison rules
    R = wq.Rules(3, 3, (9, 8, 7), device=False, rule="wqb")
    Rg = wq.Rules(3, 3, (9, 8, 7), device=False)
    counts = [len(R.row(0, 0, r)[0]) for r in range(3)]
    assert counts == [2, 8, 3]
    assert [len(Rg.row(0, 0, r)[0]) for r in range(3)] == [4, 8, 12]
    assert R.flops()[0] < Rg.flops()[0]
    R.close()
    Rg.close()
    m = wq.wq_mesh(3, 3, (ctypes.c_int * 3)(5, 5, 5))
    h = ctypes.c_void_p()
    for bad in (wq.WQ_RULES_BOUNDARY_WEIGHTED | wq.WQ_RULES_GAUSS_LEGENDRE,
                wq.WQ_RULES_BOUNDARY_WEIGHTED | wq.WQ_RULES_NEWTON_COTES):
        assert wq.library().wq_rules_build(ctypes.byref(m), bad, ctypes.byref(h)) == wq.WQ_ERR_ARG


@pytest.mark.parametrize("p", [2, 3])
def test_mixed_rules_match_the_oracle(p):
    y, w, v = wq.wq_rule_1d_mixed(p)
    yo, wo, vo, _ = oracle.cross_rule(p)
    assert np.max(np.abs(y - yo)) <= 1e-15
    assert np.max(np.abs(w - wo)) <= 2e-15 and np.max(np.abs(v - vo)) <= 2e-15


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("nel", [1, 2, 3, 5, 11])
def test_mixed_row_tables_match_oracle(p, nel):
    R = wq.Rules(2, p, (nel, 4), device=False)
    for kind in (wq.WQ_KIND_MIXED_DW, wq.WQ_KIND_MIXED_WD):
        for r in range(nel + p):
            x, W, e = R.row(0, kind, r)
            xo, Wo = oracle.row_points_cross(p, nel, kind, r)
            xm, _, em = R.row(0, 0, r)
            assert len(x) == len(xo) == len(xm)
            assert np.all(e == em)  # same elements point by point as the mass kind
            assert np.max(np.abs(x - xo)) < 1e-15
            assert np.max(np.abs(W - Wo)) < 1e-14 * max(1.0, np.max(np.abs(Wo)))
    R.close()


def test_mixed_kinds_only_with_the_plain_rules():
    for rule in ("gl", "nc", "wqb"):
        R = wq.Rules(3, 3, (9, 8, 7), device=False, rule=rule)
        with pytest.raises(wq.WqError) as ei:
            R.row(0, wq.WQ_KIND_MIXED_DW, 3)
        assert ei.value.status == wq.WQ_ERR_UNSUPPORTED
        R.close()
    R = wq.Rules(3, 3, (9, 8, 7), device=False)
    with pytest.raises(wq.WqError):
        R.row(0, 4, 3)
    R.close()
