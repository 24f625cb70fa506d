"""Batched assembly (wq_batch_*): per degree two persistent launches
(partial contractions, rows) for many patches, replayed from a CUDA graph,
with an autotuned launch configuration.

Every patch's bands must be bit-identical to a single-patch
wq_assemble_mass_stiffness call in the same precision (the batch runs the
same per-chunk arithmetic), whatever the chunk lengths, CTA counts or
schedule; a few patches are also compared with the oracle."""
import json

import numpy as np
import pytest

import oracle
from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = [(2, (6, 5, 4)), (3, (14, 9, 7)), (3, (1, 1, 1)), (2, (3, 12, 2)), (3, (25, 4, 6)), (2, (9, 9, 9)),
         (3, (2, 3, 11)), (3, (14, 9, 7))]  # the last shares its mesh with the second


def make_patches(specs, prec, seed=0):
    dt = torch.float32 if prec == "mixed" else torch.float64
    rules_cache, patches, host = {}, [], []
    for i, (p, nel) in enumerate(specs):
        key = (p, nel)
        if key not in rules_cache:
            rules_cache[key] = wq.Rules(3, p, nel)
        R = rules_cache[key]
        g, c = inputs.make(3, p, nel, 0.02 + 0.01 * (i % 5), "exp", 0.1, seed=seed + i)
        gd = [torch.from_numpy(x).cuda() for x in g]
        cd = torch.from_numpy(c).cuda()
        M = torch.full((R.rows, R.band), float("nan"), dtype=dt, device="cuda")
        K = torch.full((R.rows, R.band), float("nan"), dtype=dt, device="cuda")
        patches.append((R, gd, cd, M, K))
        host.append((g, c))
    return patches, host


def assert_matches_single(patches, prec):
    for R, gd, cd, M, K in patches:
        Ms, Ks = wq.assemble(R, gd, cd, prec)
        assert torch.equal(M, Ms) and torch.equal(K, Ks)


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_batch_equals_single_patch_calls(prec):
    patches, host = make_patches(SMALL, prec)
    B = wq.Batch(patches, prec)
    B.launch()
    B.check()
    assert_matches_single(patches, prec)
    if prec == "fp64":
        for k in (1, 4):
            R, _, _, M, K = patches[k]
            g, c = host[k]
            Mo, Ko, _ = oracle.assemble(3, R.degree, R.nel, g, c)
            for A, O in ((M, Mo), (K, Ko)):
                d = A.cpu().numpy() - O
                assert np.max(np.abs(d)) <= 1e-12 * np.max(np.abs(O))
    B.close()


def test_batch_configurations_and_tuner(monkeypatch):
    monkeypatch.delenv("WQ_AUTOTUNE_CACHE", raising=False)
    patches, _ = make_patches(SMALL, "fp64", seed=3)
    B = wq.Batch(patches, "fp64")
    mu, mx = B.config["max_u_ctas_per_sm"], B.config["max_ctas_per_sm"]
    assert mu >= 1 and mx >= 1
    for cfg in [(32, mu, mx, 1), (8, 1, 1, 0), (13, mu, mx, 0), (1, 1, 1, 1)]:
        for _, _, _, M, K in patches:
            M.fill_(float("nan"))
            K.fill_(float("nan"))
        B.set_config(*cfg)
        c = B.config
        assert (c["chunk"], c["u_ctas_per_sm"], c["ctas_per_sm"], c["schedule"]) == cfg
        B.launch()
        B.check()
        assert_matches_single(patches, "fp64")
    for bad in [(33, mu, mx, 0), (32, mu + 1, mx, 0), (32, mu, mx + 1, 0), (32, mu, mx, 2)]:
        with pytest.raises(wq.WqError):
            B.set_config(*bad)
    ms = B.tune(reps=1)
    assert ms > 0
    for _, _, _, M, K in patches:
        M.fill_(float("nan"))
        K.fill_(float("nan"))
    B.launch()
    B.check()
    assert_matches_single(patches, "fp64")
    B.close()


def _cfg(B):
    c = B.config
    return [c["chunk"], c["u_ctas_per_sm"], c["ctas_per_sm"], c["schedule"]]


def test_tuner_cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("WQ_AUTOTUNE_CACHE", str(path))
    patches, _ = make_patches(SMALL[:5], "mixed", seed=7)
    B = wq.Batch(patches, "mixed")
    ms = B.tune(reps=1)
    assert ms > 0
    d = json.loads(path.read_text())
    assert len(d) == 1
    key, ent = next(iter(d.items()))
    assert ent["config"] == _cfg(B) and abs(ent["ms"] - ms) <= 1e-5 * ms
    assert "|mixed|" in key and f"|sm{torch.cuda.get_device_properties(0).multi_processor_count}|" in key
    B.close()
    # plant another valid configuration and a time no run takes: a new plan of
    # the same patches comes back with both, so its tune() timed nothing
    planted = [16, 1, 1, 1 - ent["config"][3]]
    path.write_text('{\n  "%s": {"config": [%d, %d, %d, %d], "ms": 1234.5}\n}\n' % (key, *planted))
    for _, _, _, M, K in patches:
        M.fill_(float("nan"))
        K.fill_(float("nan"))
    B2 = wq.Batch(patches, "mixed")
    assert B2.tune(reps=1) == 1234.5
    assert _cfg(B2) == planted
    B2.launch()
    B2.check()
    assert_matches_single(patches, "mixed")
    B2.close()
    # another precision or another patch set is another key: timed, and added
    # beside the planted entry
    B3 = wq.Batch(patches, "fp64")
    ms3 = B3.tune(reps=1)
    assert 0 < ms3 < 1234.5
    B4 = wq.Batch(patches[:3], "mixed")
    B4.tune(reps=1)
    d = json.loads(path.read_text())
    assert len(d) == 3 and d[key] == {"config": planted, "ms": 1234.5}
    B3.close()
    B4.close()
    # a cached configuration the plan rejects is timed again and replaced
    path.write_text('{\n  "%s": {"config": [32, 999, 1, 0], "ms": 1234.5}\n}\n' % key)
    B5 = wq.Batch(patches, "mixed")
    ms5 = B5.tune(reps=1)
    assert ms5 < 1234.5
    d = json.loads(path.read_text())
    assert d[key]["config"] == _cfg(B5) and d[key]["config"][1] != 999
    B5.close()


def test_graph_replay_reads_new_inputs_and_one_shot():
    patches, _ = make_patches(SMALL[:4], "df64", seed=5)
    B = wq.Batch(patches, "df64")
    B.launch()
    # new coefficient and geometry values in the same buffers
    for R, gd, cd, M, K in patches:
        cd.mul_(1.5).add_(0.25)
        gd[0].mul_(1.1)
    B.launch()
    B.check()
    assert_matches_single(patches, "df64")
    B.close()
    for _, _, _, M, K in patches:
        M.zero_()
        K.zero_()
    wq.assemble_batch(patches, "df64")
    assert_matches_single(patches, "df64")


def test_batch_status_and_arguments():
    patches, _ = make_patches(SMALL[:3], "fp64", seed=7)
    patches[1][2][5] = float("nan")
    B = wq.Batch(patches, "fp64")
    B.launch()
    assert B.status() == wq.WQ_ERR_NONFINITE
    patches[1][2][5] = 1.0
    B.launch()
    assert B.status() == wq.WQ_OK
    B.close()
    # a 2D rules object is rejected
    R2 = wq.Rules(2, 3, (5, 5))
    g = [torch.ones(8, dtype=torch.float64, device="cuda")] * 3
    M = torch.empty((R2.rows, R2.band), dtype=torch.float64, device="cuda")
    with pytest.raises(wq.WqError) as ei:
        wq.Batch([(R2, g, None, M, M)], "fp64")
    assert ei.value.status == wq.WQ_ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_256_patches(prec):
    # 256 patches, element counts log-uniform in [8, 48] per direction,
    # degree 2 or 3, geometry amplitude U[0, 0.08]
    specs = inputs.batch_patches(256, seed=0)
    dt = torch.float32 if prec == "mixed" else torch.float64
    rules, patches = {}, []
    for s in specs:
        key = (s["p"], s["nel"])
        if key not in rules:
            rules[key] = wq.Rules(3, s["p"], s["nel"])
        R = rules[key]
        gd = [torch.from_numpy(x).cuda() for x in s["geom"]]
        cd = torch.from_numpy(s["coef"]).cuda()
        M = torch.empty((R.rows, R.band), dtype=dt, device="cuda")
        K = torch.empty((R.rows, R.band), dtype=dt, device="cuda")
        patches.append((R, gd, cd, M, K))
    B = wq.Batch(patches, prec)
    B.tune(reps=1)
    B.launch()
    B.check()
    assert_matches_single(patches, prec)
    # a seeded sample of the patches against the oracle: three x3 slabs of
    # rows each (first, middle, last), every row of the slab
    tol = 1e-6 if prec == "mixed" else 1e-12
    rng = np.random.default_rng(256)
    for k in rng.choice(len(specs), size=6, replace=False):
        s = specs[int(k)]
        R, _, _, M, K = patches[int(k)]
        n = [v + s["p"] for v in s["nel"]]
        slab = n[0] * n[1]
        for z in (0, n[2] // 2, n[2] - 1):
            rb, re = z * slab, (z + 1) * slab
            Mo, Ko, _ = oracle.assemble(3, s["p"], s["nel"], s["geom"], s["coef"], rb, re)
            for A, O in ((M, Mo), (K, Ko)):
                d = A[rb:re].double().cpu().numpy() - O
                assert np.max(np.abs(d)) <= tol * np.max(np.abs(O)), (k, z)
                assert np.linalg.norm(d) <= tol * np.linalg.norm(O), (k, z)
    B.close()


def test_batch_equals_single_calls_mixed_on_long_lines():
    # lines of several row chunks, in FP32: the persistent batch launches and
    # the per-mesh launches run the same block code, so the bits agree
    specs = [(3, (70, 5, 4)), (2, (66, 3, 4)), (3, (97, 2, 3)), (2, (33, 4, 2))]
    patches, _ = make_patches(specs, "mixed", seed=9)
    B = wq.Batch(patches, "mixed")
    B.launch()
    B.check()
    assert_matches_single(patches, "mixed")
    B.close()
