"""Benchmark: 3D cubic weighted-Gaussian mass+stiffness assembly, nnz/s.

One step = one mass+stiffness assembly call (coefficient check, geometry
fold, the partial-contraction kernel and the row kernel, all rows) of the
named synthetic workload through the C-ABI.  Default workload: 128^3
elements, C2 cubic (p = 3), separable map xhat + 0.05 sin(pi xhat) per
coordinate, c = exp(0.3 (x+y+z)) with lognormal(0.1) noise as a cubic spline
on the same mesh, FP64 arithmetic and FP64 bands (--prec fp64).  Beside it
("variants"): the same workload in double-float (FP64-accurate on the FP32
pipe) and FP32 (mixed) arithmetic, each with its error against the oracle;
the 64^3 cubic and quadratic workloads and the 2D 32^2 cubic one in every
precision; the comparison rules (Gauss-Legendre rows, Newton-Cotes-type
rule; FP64) with their quadrature point totals; the adjoint on the 96^3
cubic workload; the matrix-free apply; the 256-patch batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload 3d_p3_128] [--prec fp64|df64|mixed] [--no-cpu-baseline]

Prints one JSON line.  value = assembled non-zeros (M and K) per second over
all ranks, device time (CUDA events around each step on the launching
stream, L2 flushed before each step by writing a 256 MiB buffer); e2e = the
same through host buffers (wq_assemble_mass_stiffness_host: pinned H2D of
geometry and coefficients, D2H of both bands, inside the timed region).
Under torchrun the mesh grows along x3 with the rank count (128 x 128 x
128 N elements) and each rank assembles its own slab of x3 planes (weak
scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "3D cubic WQ mass+stiffness assembled nnz/s"
DTYPE = {"fp64": "f64", "df64": "f32x2", "mixed": "f32"}
# peaks of the ALU-bound forms (none is in MEASURED_PEAKS.json, which holds
# the HBM copy rate and dense bf16 tensor rates):
# FP64: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz = 1.259 TFLOP/s (the
# nominal FP64 rate of the part, 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 80.5
# double-float multiply-add = 12 FP32-pipe instructions (csrc/dd.cuh): FP64-equivalent peak
DF64_PEAK_TFLOPS = 152 * 128 / 12 * 2 * 2.070e9 / 1e12  # 6.71
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# capture of the current kernel (dram__bytes_read.sum + dram__bytes_write.sum);
# entries without a capture of the current kernel are absent and report null.
# "scale": the captured case's rows, when the capture was made on a smaller
# mesh of the same kernel and its traffic is scaled to the workload's rows.
_CAP64 = ("ncu --set full --clock-control none -k regex:rows_ug_kernel, python bench.py --workload 3d_p3_64 "
          "--steps 1 --warmup 3 --no-cpu-baseline --no-variants --no-e2e --prec {}; 64^3 launch scaled by rows")
TRAFFIC = {
    ("3d_p3_128", "fp64"): {"bytes": 236.140544e6 + 1.589815e9, "scale_rows": 300763,
                            "note": "rows_ug_kernel<3,32,M+K,double>: " + _CAP64.format("fp64")},
    ("3d_p3_128", "df64"): {"bytes": 236.021504e6 + 1.590448e9, "scale_rows": 300763,
                            "note": "rows_ug_kernel<3,32,M+K,dd>: " + _CAP64.format("df64")},
    ("3d_p3_128", "mixed"): {"bytes": 118.000640e6 + 767.056128e6, "scale_rows": 300763,
                             "note": "rows_ug_kernel<3,32,M+K,float>: " + _CAP64.format("mixed")},
    ("3d_p3_64", "fp64"): {"bytes": 236.140544e6 + 1.589815e9,
                           "note": "rows_ug_kernel<3,32,M+K,double>: " + _CAP64.format("fp64").split(";")[0]},
    ("3d_p3_64", "df64"): {"bytes": 236.021504e6 + 1.590448e9,
                           "note": "rows_ug_kernel<3,32,M+K,dd>: " + _CAP64.format("df64").split(";")[0]},
    ("3d_p3_64", "mixed"): {"bytes": 118.000640e6 + 767.056128e6,
                            "note": "rows_ug_kernel<3,32,M+K,float>: " + _CAP64.format("mixed").split(";")[0]},
}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def band_nnz_rows(nel, p, rows_idx):
    """Number of in-range band entries of the given rows (one matrix)."""
    import numpy as np

    dim = len(nel)
    n = [v + p for v in nel]
    cnt = np.ones_like(rows_idx)
    rest = rows_idx
    for a in range(dim):
        r = rest % n[a]
        rest = rest // n[a]
        cnt = cnt * (np.minimum(n[a] - 1, r + p) - np.maximum(0, r - p) + 1)
    return int(cnt.sum())


def cpu_sample_rows(nel, p, stride):
    """Every `stride`-th slab of rows along the last direction (interior and
    boundary rows alike)."""
    n = [v + p for v in nel]
    slab = 1
    for v in n[:-1]:
        slab *= v
    return [(s * slab, (s + 1) * slab) for s in range(0, n[-1], stride)]


def run_oracle_sample(w, g, c, stride):
    """The FP64 oracle on a sample of slabs with all host cores: (seconds,
    in-range non-zeros of M and K, the sample's rows, [(rb, re, M, K)])."""
    import numpy as np

    import oracle

    nel, p, dim = w["nel"], w["p"], w["dim"]
    ranges = cpu_sample_rows(nel, p, stride)
    nnz = 0
    outs = []
    t0 = time.perf_counter()
    for rb, re in ranges:
        M, K, _ = oracle.assemble(dim, p, nel, g, c, rb, re)
        outs.append((rb, re, M, K))
    dt = time.perf_counter() - t0
    for rb, re in ranges:
        nnz += 2 * band_nnz_rows(nel, p, np.arange(rb, re))
    rows = sum(re - rb for rb, re in ranges)
    return dt, nnz, rows, outs


def errors_vs_oracle(bands, outs):
    """Per-matrix relative max-entry and Frobenius errors of device bands on
    the oracle's sampled rows (bands: (M, K) torch tensors of all rows)."""
    import numpy as np

    res = {}
    for name, A, k in (("M", bands[0], 2), ("K", bands[1], 3)):
        dmax = omax = dsq = osq = 0.0
        for o in outs:
            rb, re, O = o[0], o[1], o[k]
            d = A[rb:re].double().cpu().numpy() - O
            dmax = max(dmax, float(np.max(np.abs(d))))
            omax = max(omax, float(np.max(np.abs(O))))
            dsq += float(np.sum(d * d))
            osq += float(np.sum(O * O))
        res[name] = {"rel_max": dmax / omax, "rel_fro": (dsq / osq) ** 0.5}
    res["max"] = max(res["M"]["rel_max"], res["K"]["rel_max"], res["M"]["rel_fro"], res["K"]["rel_fro"])
    return res


def reference_arm(args):
    """The oracle as it stands, on the host cores, for the same workload."""
    import numpy as np

    from paper_1710_01048_gb300 import inputs

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, g, c = inputs.workload(args.workload)
    nel, p, dim = w["nel"], w["p"], w["dim"]
    ranges = cpu_sample_rows(nel, p, 1)
    # each step: one slab of rows along the last direction (a bounded sample of the workload)
    import oracle

    oracle.build()
    for i in range(args.warmup):
        rb, re = ranges[i % len(ranges)]
        oracle.assemble(dim, p, nel, g, c, rb, re)
    t = []
    nnz = 0
    for i in range(args.steps):
        rb, re = ranges[(len(ranges) // 2 + i) % len(ranges)]
        t0 = time.perf_counter()
        oracle.assemble(dim, p, nel, g, c, rb, re)
        t.append(time.perf_counter() - t0)
        nnz += 2 * band_nnz_rows(nel, p, np.arange(rb, re))
    total = sum(t)
    value = nnz / total
    slab = ranges[0][1] - ranges[0][0]
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "nel": list(nel), "degree": p, "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"one slab of {slab} rows along the last direction per step"},
           "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d_p3_128")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "df64", "mixed"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-patch batch variant")
    ap.add_argument("--batch-patches", type=int, default=256,
                    help="patches of the batch variant (the workload is 256; fewer for profiling)")
    ap.add_argument("--batch-precs", default="fp64,df64,mixed", help="precisions of the batch variant")
    ap.add_argument("--adjoint-workload", default="3d_p3_96",
                    help="workload of the adjoint variant (the configuration is 3d_p3_96; smaller for profiling)")
    ap.add_argument("--adjoint-precs", default="fp64,df64,mixed", help="precisions of the adjoint variant")
    ap.add_argument("--only", default=None,
                    help="comma list of variant groups to run: precisions, workloads, rules, adjoint, apply, "
                         "general, batch (default: all)")
    ap.add_argument("--cpu-stride", type=int, default=16)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch

    from paper_1710_01048_gb300 import binding as wq
    from paper_1710_01048_gb300 import inputs, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)

    def timed(fn, n, do_flush=True):
        """Mean device time (ms) of n calls of fn, CUDA events on the stream."""
        evs = []
        for _ in range(n):
            if do_flush:
                flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    # ------------------------------------------------------------ the workload (this rank's slab)
    w = dict(inputs.WORKLOADS[args.workload])
    dim, p = w["dim"], w["p"]
    nel = list(w["nel"])
    nel[-1] *= world  # weak scaling: the mesh grows along the last direction
    nel = tuple(nel)
    g, c = inputs.make(dim, p, nel, w["amp"], w["coef"], w["sigma"], w["seed"])
    R = wq.Rules(dim, p, nel)
    rb, re = shard.shard_rows([v + p for v in nel], rank, world)
    rows, band = re - rb, R.band
    nnz_rank = wq.wq_band_nnz_rows(R.handle, rb, re)
    nnz_step = 2 * nnz_rank  # M and K
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    dt = torch.float32 if args.prec == "mixed" else torch.float64
    M = torch.empty((rows, band), dtype=dt, device="cuda")
    K = torch.empty((rows, band), dtype=dt, device="cuda")

    def step():
        wq.assemble(R, gd, cd, args.prec, out=(M, K), row_begin=rb, row_end=re, stream=stream, check=False)

    for _ in range(args.warmup):
        step()
    st = wq.wq_status_check(R.handle, wq._stream_handle(stream))
    if st != wq.WQ_OK:
        raise wq.WqError(st, "warm-up")

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    ms = timed(step, args.steps)
    barrier()
    clocks = sampler.stop()
    ms_step = float(np.mean(ms))
    st = wq.wq_status_check(R.handle, wq._stream_handle(stream))
    if st != wq.WQ_OK:
        raise wq.WqError(st, "timed steps")
    # coefficient check/convert + fold + partial contractions + rows per step
    gpu_launches = 4 * args.steps

    # ------------------------------------------------------------ end to end through host buffers
    e2e = None
    if not args.no_e2e:
        gh = [torch.from_numpy(x).pin_memory() for x in g]
        ch = torch.from_numpy(c).pin_memory()
        Mh = torch.empty((rows, band), dtype=dt, pin_memory=True)
        Kh = torch.empty((rows, band), dtype=dt, pin_memory=True)
        gdd = [torch.empty_like(x) for x in gd]
        cdd = torch.empty_like(cd)
        h2d = sum(x.numel() * 8 for x in gh) + ch.numel() * 8
        d2h = 2 * rows * band * M.element_size()
        e2e_steps = max(3, min(args.steps, 10))

        def e2e_step():
            wq.assemble_to_host(R, gh, ch, args.prec, Mh, Kh, gdd, cdd, M, K, nchunks=8, stream=stream,
                                row_begin=rb, row_end=re)

        e2e_step()
        barrier()
        e2e_ms = float(np.mean(timed(e2e_step, e2e_steps, do_flush=False)))
        barrier()
        if not torch.equal(Mh[: min(rows, 64)], M[: min(rows, 64)].cpu()):
            raise RuntimeError("end-to-end bands differ from the device bands")
        e2e = {"ms_per_step": e2e_ms, "h2d": h2d, "d2h": d2h}
        del Mh, Kh, gh, ch, gdd, cdd

    # the oracle's sampled rows (rank 0 at N = 1): CPU baseline and the
    # accuracy of every precision on those rows
    sample = None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs, snnz, srows, outs = run_oracle_sample(w, g, c, args.cpu_stride)
        sample = outs
        cpu = {"value": snnz / secs, "unit": "nnz/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{len(outs)} slabs of rows along x3 (every {args.cpu_stride}th; {srows} of {R.rows} "
                         f"rows, {snnz} non-zeros of M and K), {secs:.1f} s wall; the rate is the sample's"}
    accuracy = errors_vs_oracle((M, K), sample) if sample else None

    # max over ranks
    if dist is not None:
        ms_step, e2e_ms_max = shard.max_over_ranks([ms_step, e2e["ms_per_step"] if e2e else 0.0], dist,
                                                   device="cuda")
        if e2e:
            e2e["ms_per_step"] = e2e_ms_max
        nnz_all = shard.sum_over_ranks([nnz_step], dist, device="cuda")[0]
    else:
        nnz_all = nnz_step
    value = nnz_all / (ms_step * 1e-3)

    # roofline of the assembly call (coefficient prepare + fold + the two
    # kernels): the step's algorithmic contraction flops / the step's device time
    flops, coef_flops = R.flops(row_begin=rb, row_end=re)
    bytes_step = 2 * rows * band * M.element_size()
    if args.prec in ("fp64", "df64"):
        pk = FP64_PEAK_TFLOPS if args.prec == "fp64" else DF64_PEAK_TFLOPS
        achieved = flops / (ms_step * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                "peak_source": ("derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal FP64 1.25 TFLOP/s; "
                                "not in MEASURED_PEAKS.json)" if args.prec == "fp64" else
                                "derived: FP32 pipe 152 SMs x 128 lanes x 2.07 GHz / 12 FP32 instructions per "
                                "double-float multiply-add, x 2 flop (FP64-equivalent)"),
                "flops_per_step": flops, "band_bytes_per_step": bytes_step,
                "band_gb_s": bytes_step / (ms_step * 1e-3) / 1e9,
                "achieved_incl_coef_eval": (flops + coef_flops) / (ms_step * 1e-3) / 1e12}
    else:
        achieved = bytes_step / (ms_step * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
                else "fallback 6.8 TB/s",
                "fp32_tflops": (flops + coef_flops) / (ms_step * 1e-3) / 1e12, "fp32_peak_tflops": FP32_PEAK_TFLOPS}
    tr = TRAFFIC.get((args.workload, args.prec))
    if tr and world == 1:
        roof["traffic"] = tr["bytes"] * (R.rows / tr["scale_rows"] if tr.get("scale_rows") else 1.0)
        roof["traffic_note"] = tr["note"]
        # the dominant kernel's algorithmic bytes: the band written plus the
        # partial contractions U it reads
        roof["traffic_over_band_bytes"] = roof["traffic"] / bytes_step
    else:
        roof["traffic"] = None

    # ------------------------------------------------------------ variants (rank 0 at N = 1)
    variants = {}
    if not args.no_variants and world == 1:
        variants = run_variants(args, wq, inputs, R, w, g, gd, cd, (M, K), sample, timed, stream, peaks)

    out = {"metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
           "config": {"workload": args.workload, "nel": list(nel), "degree": p, "rows": int(R.rows),
                      "rows_per_rank": int(rows), "band": int(band), "nnz_per_matrix": int(R.nnz),
                      "precision": args.prec,
                      "l2": "256 MiB buffer written before each timed step; each step also writes "
                            f"{bytes_step / 1e9:.2f} GB of band output per rank"},
           "roofline": roof, "clocks": clocks, "gpu_launches": gpu_launches,
           "ms_per_step_min": float(np.min(ms)), "ms_per_step_max": float(np.max(ms))}
    if e2e:
        out["e2e"] = {"value": nnz_all / (e2e["ms_per_step"] * 1e-3), "unit": "nnz/s",
                      "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                      "ms_per_step": e2e["ms_per_step"],
                      "path": "wq_assemble_mass_stiffness_host (pinned host buffers, 8 overlapped row ranges)"}
    if cpu:
        out["cpu_baseline"] = cpu
    if accuracy:
        out["max_rel_err_vs_oracle"] = accuracy["max"]
        out["error_vs_oracle"] = {k: accuracy[k] for k in ("M", "K")}
    out["variants"] = variants
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    R.close()
    return 0


def general_counts(Rg, dim, p, nel, has_coef):
    """Algorithmic work of one assembly for a map given by a full control net
    (wq_assemble_general): (flops of the row contractions, flops of the
    per-point metric, factor points, HBM bytes of FP32 data flow).

    Rows: per row and term, the sum-factorised contractions over the band's
    non-zero structure, each 1D weight-test row touching p+1 band columns:
    3D 2 L1 L2 L3 (p+1) + 2 L1 L2 (2p+1)(p+1) per term (10 terms) and
    2 L1 (2p+1)^2 (p+1) per direction-1 group (5 groups); 2D 2 L1 L2 (p+1)
    per term (5) and 2 L1 (2p+1)(p+1) per group (5).  Summed over rows these
    factor into the per-direction point counts.  Metric: per point of each
    grid the Jacobian (p+1 multiply-adds per entry), the coefficient (4
    multiply-adds) and the
    metric entry (determinant 15 flops, an off-diagonal or stiffness entry 31
    in 3D; 5 and 13 in 2D); the partial contractions of the net that feed the
    Jacobian are not counted."""
    import numpy as np
    NP, NB = p + 1, 2 * p + 1
    n = [nel[a] + p for a in range(dim)]
    np_ = [sum(len(Rg.row(a, 0, r)[0]) for r in range(n[a])) for a in range(dim)]
    if dim == 3:
        rows_fl = 10 * (2 * NP * np_[0] * np_[1] * np_[2] + 2 * NB * NP * np_[0] * np_[1] * n[2]) \
            + 5 * 2 * NB * NB * NP * np_[0] * n[1] * n[2]
        pts = np_[0] * np_[1] * np_[2]
        per_pt_j = 2 * (3 * NP + 3 * NP + 3 * NP)
        met = pts * (7 * per_pt_j + (7 * 8 if has_coef else 0) + 15 + 6 * 31)
        grids = 7
    else:
        rows_fl = 5 * 2 * NP * np_[0] * np_[1] + 5 * 2 * NB * NP * np_[0] * n[1]
        pts = np_[0] * np_[1]
        per_pt_j = 2 * (2 * NP + 2 * NP)
        met = pts * (4 * per_pt_j + (4 * 8 if has_coef else 0) + 5 + 3 * 13)
        grids = 4
    ntot = int(np.prod(n))
    ncoef = int(np.prod([nel[a] + 3 for a in range(dim)]))
    rows = int(np.prod(n))
    nband = NB ** dim
    bytes32 = (8 * dim * ntot + 2 * 4 * dim * dim * ntot + (12 * ncoef if has_coef else 0)
               + 2 * 4 * grids * pts + 2 * 4 * rows * nband)
    return float(rows_fl), float(met), int(grids * pts), float(bytes32)


def run_variants(args, wq, inputs, R, w, g, gd, cd, bands, sample, timed, stream, peaks):
    """The other precisions of the headline workload (with their errors on the
    oracle's sampled rows), the other workloads of the same method, the
    comparison rules, the adjoint, the matrix-free apply and the batch."""
    import numpy as np
    import torch

    hbm = peaks.get("hbm_gbs", 6800.0)
    variants = {}
    reps = max(3, min(args.steps, 10))
    groups = None if args.only is None else set(args.only.split(","))
    want = lambda k: groups is None or k in groups  # noqa: E731

    def assemble_timed(Rv, gdv, cdv, prec, out, n):
        fn = lambda: wq.assemble(Rv, gdv, cdv, prec, out=out, stream=stream, check=False)  # noqa: E731
        for _ in range(3):
            fn()
        ms = float(np.mean(timed(fn, n)))
        st = wq.wq_status_check(Rv.handle, wq._stream_handle(stream))
        if st != wq.WQ_OK:
            raise wq.WqError(st, "variant")
        return ms

    def roofline(Rv, prec, ms, nbytes):
        fl, _ = Rv.flops()
        if prec == "mixed":
            bw = nbytes / (ms * 1e-3) / 1e9
            return {"bound": "hbm", "achieved": bw, "peak": hbm, "unit": "GB/s", "frac": bw / hbm,
                    "fp32_tflops": fl / (ms * 1e-3) / 1e12}
        pk = FP64_PEAK_TFLOPS if prec == "fp64" else DF64_PEAK_TFLOPS
        tf = fl / (ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s", "frac": tf / pk}

    # the other precisions of the headline workload, errors on the oracle's rows
    if want("precisions"):
        for vp in ("fp64", "df64", "mixed"):
            if vp == args.prec:
                continue
            vdt = torch.float32 if vp == "mixed" else torch.float64
            if vdt == bands[0].dtype:
                Mv, Kv = bands  # the headline's errors are already taken: reuse its buffers
            else:
                Mv = torch.empty((R.rows, R.band), dtype=vdt, device="cuda")
                Kv = torch.empty((R.rows, R.band), dtype=vdt, device="cuda")
            vm = assemble_timed(R, gd, cd, vp, (Mv, Kv), reps)
            ev = {"ms_per_step": vm, "value": 2 * R.nnz / (vm * 1e-3), "unit": "nnz/s", "dtype": DTYPE[vp],
                  "roofline": roofline(R, vp, vm, 2 * R.rows * R.band * Mv.element_size())}
            if sample:
                ev["error_vs_oracle"] = errors_vs_oracle((Mv, Kv), sample)
            variants[vp] = ev
            del Mv, Kv
        torch.cuda.empty_cache()

    # the other workloads: 64^3 cubic and quadratic, 2D 32^2 cubic (c as
    # named, and c = 1), every precision, errors on oracle rows
    if want("workloads"):
        others = [("3d_p3_64", 16), ("3d_p2_64", 16), ("2d_p3_32", 1), ("2d_p3_32_c1", 1)]
        for name, stride in others:
            if name == args.workload:
                continue
            wv, gv, cv = inputs.workload(name)
            Rv = wq.Rules(wv["dim"], wv["p"], wv["nel"])
            gdv = [torch.from_numpy(x).cuda() for x in gv]
            cdv = torch.from_numpy(cv).cuda()
            _, _, _, outs = run_oracle_sample(wv, gv, cv, stride)
            ent = {"workload": name, "nel": list(wv["nel"]), "degree": wv["p"], "rows": int(Rv.rows),
                   "nnz_per_matrix": int(Rv.nnz),
                   "oracle_rows": int(sum(o[1] - o[0] for o in outs))}
            for vp in ("fp64", "df64", "mixed"):
                vdt = torch.float32 if vp == "mixed" else torch.float64
                Mv = torch.empty((Rv.rows, Rv.band), dtype=vdt, device="cuda")
                Kv = torch.empty((Rv.rows, Rv.band), dtype=vdt, device="cuda")
                vm = assemble_timed(Rv, gdv, cdv, vp, (Mv, Kv), reps)
                ent[vp] = {"ms_per_step": vm, "value": 2 * Rv.nnz / (vm * 1e-3), "unit": "nnz/s",
                           "roofline": roofline(Rv, vp, vm, 2 * Rv.rows * Rv.band * Mv.element_size()),
                           "error_vs_oracle": errors_vs_oracle((Mv, Kv), outs)}
                del Mv, Kv
            variants[name] = ent
            Rv.close()
        torch.cuda.empty_cache()

    # the comparison rules (FP64, same kernel's general-points class) on the
    # 64^3 cubic workload: Gauss-Legendre on every element of each row's
    # support, and the Newton-Cotes-type weighted rules; and the weighted
    # Gaussian rules with the boundary rows on their own weighted rules
    # ('wqb', the default kernels); with the quadrature-point counts
    if want("rules") or want("apply"):
        wc, gc, cc = inputs.workload("3d_p3_64")
        gdc = [torch.from_numpy(x).cuda() for x in gc]
        cdc = torch.from_numpy(cc).cuda()
    if want("rules"):
        points = {}
        Mv = Kv = None
        for mode in ("wq", "wqb", "nc", "gl"):
            Rm = wq.Rules(3, wc["p"], wc["nel"], rule=mode)
            total = 1
            for a in range(3):
                total *= sum(len(Rm.row(a, 0, r)[0]) for r in range(wc["nel"][a] + wc["p"]))
            points[mode] = {"points_per_interior_row_and_direction": len(Rm.row(0, 0, wc["p"])[0]),
                            "rule_points_total": total}
            if Mv is None:
                Mv = torch.empty((Rm.rows, Rm.band), dtype=torch.float64, device="cuda")
                Kv = torch.empty((Rm.rows, Rm.band), dtype=torch.float64, device="cuda")
            vm = assemble_timed(Rm, gdc, cdc, "fp64", (Mv, Kv), max(3, min(args.steps, 5)))
            variants["3d_p3_64_fp64_" + mode + "_rule"] = {"ms_per_step": vm, "value": 2 * Rm.nnz / (vm * 1e-3),
                                                            "unit": "nnz/s", "dtype": "f64", **points[mode]}
            Rm.close()
        variants["rule_points_3d_p3_64"] = points
        del Mv, Kv
        torch.cuda.empty_cache()

    # the adjoint (coefficient gradient of sum G*K + H*M) on the 96^3 cubic workload
    if want("adjoint"):
        w3, g3, c3 = inputs.workload(args.adjoint_workload)
        R3 = wq.Rules(3, w3["p"], w3["nel"])
        gd3 = [torch.from_numpy(x).cuda() for x in g3]
        gen = torch.Generator(device="cuda").manual_seed(96)
        adj = {"workload": args.adjoint_workload, "ncoef": R3.ncoef}
        for vp in args.adjoint_precs.split(","):
            vdt = torch.float32 if vp == "mixed" else torch.float64
            G = torch.randn((R3.rows, R3.band), dtype=vdt, device="cuda", generator=gen)
            H = torch.randn((R3.rows, R3.band), dtype=vdt, device="cuda", generator=gen)
            grad = torch.empty(R3.ncoef, dtype=torch.float64, device="cuda")
            fn = lambda: wq.assemble_adjoint(R3, gd3, G, H, vp, out=grad, stream=stream, check=False)  # noqa: E731
            for _ in range(3):
                fn()
            vm = float(np.mean(timed(fn, max(3, min(args.steps, 5)))))
            fl, _ = R3.flops()
            # per step the adjoint reads both weight bands (band entries per
            # second); its transposed stages do the forward contraction's
            # multiply-adds, counted as its algorithmic flops
            pk = {"fp64": FP64_PEAK_TFLOPS, "df64": DF64_PEAK_TFLOPS, "mixed": FP32_PEAK_TFLOPS}[vp]
            tf = fl / (vm * 1e-3) / 1e12
            adj[vp] = {"ms_per_step": vm, "value": 2 * R3.nnz / (vm * 1e-3), "unit": "nnz/s (weights read)",
                       "weights_gb_s": 2 * R3.rows * R3.band * G.element_size() / (vm * 1e-3) / 1e9,
                       "roofline": {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s", "frac": tf / pk,
                                    "flops_per_gradient": fl,
                                    "weight_bytes_per_gradient": 2 * R3.rows * R3.band * G.element_size()}}
            del G, H, grad
            torch.cuda.empty_cache()
        st = wq.wq_status_check(R3.handle, wq._stream_handle(stream))
        if st != wq.WQ_OK:
            raise wq.WqError(st, "adjoint variant")
        variants["adjoint_" + args.adjoint_workload] = adj
        R3.close()

    # matrix-free apply y = M x, y = K x (the band never stored) and the load
    # vector, on the 64^3 cubic workload
    if want("apply"):
        Ra = wq.Rules(3, wc["p"], wc["nel"])
        gen = torch.Generator(device="cuda").manual_seed(64)
        app = {"workload": "3d_p3_64", "nnz_per_step": 2 * Ra.nnz}
        for vp in ("df64", "fp64", "mixed"):
            vdt = torch.float32 if vp == "mixed" else torch.float64
            xv = torch.randn(Ra.rows, dtype=torch.float64, device="cuda", generator=gen).to(vdt)
            yM = torch.empty(Ra.rows, dtype=vdt, device="cuda")
            yK = torch.empty(Ra.rows, dtype=vdt, device="cuda")
            fn = lambda: wq.apply(Ra, gdc, xv, cdc, vp, out=(yM, yK), stream=stream, check=False)  # noqa: E731
            for _ in range(3):
                fn()
            vm = float(np.mean(timed(fn, reps)))
            # the contractions plus one multiply-add per band entry and matrix
            fl_apply = Ra.flops()[0] + 2 * 2 * Ra.nnz
            pk = {"fp64": FP64_PEAK_TFLOPS, "df64": DF64_PEAK_TFLOPS, "mixed": FP32_PEAK_TFLOPS}[vp]
            tf = fl_apply / (vm * 1e-3) / 1e12
            app[vp] = {"ms_per_step": vm, "value": 2 * Ra.nnz / (vm * 1e-3), "unit": "nnz/s (applied)",
                       "roofline": {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s", "frac": tf / pk}}
            if vp == "df64":
                bl = torch.empty(Ra.rows, dtype=vdt, device="cuda")
                fl_ = lambda: wq.assemble_load(Ra, gdc, cdc, vp, out=bl, stream=stream, check=False)  # noqa: E731
                for _ in range(3):
                    fl_()
                app["load_vector_df64_ms"] = float(np.mean(timed(fl_, 5)))
                del bl
            del xv, yM, yK
        sta = wq.wq_status_check(Ra.handle, wq._stream_handle(stream))
        if sta != wq.WQ_OK:
            raise wq.WqError(sta, "apply variant")
        variants["apply_3d_p3_64"] = app
        Ra.close()

    # maps given by a full control net (the off-diagonal metric terms with the
    # mixed-derivative rules): the warped 64^3 cubic workload, FP64 and FP32
    # (parity with the oracle is tested, not timed here)
    if want("general"):
        gen_out = {}
        for gname in ("3d_p3_64_warp",):
            wn = inputs.NET_WORKLOADS[gname]
            netn, cnn = inputs.make_net(wn["dim"], wn["p"], wn["nel"], wn["net"], wn["amp"], wn["coef"], wn["sigma"],
                                        wn["seed"])
            Rg = wq.Rules(wn["dim"], wn["p"], wn["nel"])
            ndg, cdg = torch.from_numpy(netn).cuda(), torch.from_numpy(cnn).cuda()
            rows_fl, met_fl, npts, b32 = general_counts(Rg, wn["dim"], wn["p"], wn["nel"], True)
            ent = {"workload": gname, "nel": list(wn["nel"]), "degree": wn["p"], "rows": int(Rg.rows),
                   "nnz_per_matrix": int(Rg.nnz), "metric_points": npts, "flops_rows": rows_fl, "flops_metric": met_fl,
                   "fp32_algorithmic_bytes": b32}
            for vp in ("fp64", "mixed"):
                vdt = torch.float32 if vp == "mixed" else torch.float64
                Mv = torch.empty((Rg.rows, Rg.band), dtype=vdt, device="cuda")
                Kv = torch.empty((Rg.rows, Rg.band), dtype=vdt, device="cuda")
                fn = lambda: wq.assemble_general(Rg, ndg, cdg, vp, out=(Mv, Kv), stream=stream,  # noqa: E731
                                                 check=False)
                for _ in range(3):
                    fn()
                vm = float(np.mean(timed(fn, max(3, min(args.steps, 5)))))
                stg = wq.wq_status_check(Rg.handle, wq._stream_handle(stream))
                if stg != wq.WQ_OK:
                    raise wq.WqError(stg, "general variant")
                tf = (rows_fl + met_fl) / (vm * 1e-3) / 1e12
                if vp == "fp64":
                    roof = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": tf / FP64_PEAK_TFLOPS}
                else:
                    bw = b32 / (vm * 1e-3) / 1e9
                    roof = {"bound": "hbm", "achieved": bw, "peak": hbm, "unit": "GB/s", "frac": bw / hbm,
                            "fp32_tflops": tf, "fp32_frac": tf / FP32_PEAK_TFLOPS}
                ent[vp] = {"ms_per_step": vm, "value": 2 * Rg.nnz / (vm * 1e-3), "unit": "nnz/s", "dtype": DTYPE[vp],
                           "roofline": roof}
                del Mv, Kv
                torch.cuda.empty_cache()
            gen_out[gname] = ent
            Rg.close()
        variants["general_map"] = gen_out

    # the batch of 256 independent patches (8..48 elements per direction, p in {2, 3}):
    # one graph of two persistent launches, tuned, against one call per patch
    if want("batch"):
        if not args.no_batch:
            specs = inputs.batch_patches(args.batch_patches, seed=0)
            rules_cache, base = {}, []
            for sp in specs:
                key = (sp["p"], sp["nel"])
                if key not in rules_cache:
                    rules_cache[key] = wq.Rules(3, sp["p"], sp["nel"])
                base.append((rules_cache[key], [torch.from_numpy(x).cuda() for x in sp["geom"]],
                             torch.from_numpy(sp["coef"]).cuda()))
            bnnz = 2 * sum(Rb.nnz for Rb, _, _ in base)
            bflops = sum(Rb.flops()[0] for Rb, _, _ in base)
            bat = {"workload": f"batch_{args.batch_patches}", "patches": args.batch_patches, "nnz_per_step": bnnz, "flops_per_step": bflops}
            for vp in args.batch_precs.split(","):
                vdt = torch.float32 if vp == "mixed" else torch.float64
                pts = [(Rb, gb, cb, torch.empty((Rb.rows, Rb.band), dtype=vdt, device="cuda"),
                        torch.empty((Rb.rows, Rb.band), dtype=vdt, device="cuda")) for Rb, gb, cb in base]
                Bp = wq.Batch(pts, vp)
                Bp.tune(reps=1, stream=stream)
                Bp.launch(stream)
                tb = float(np.mean(timed(lambda: Bp.launch(stream), 5)))
                stb = Bp.status(stream)
                if stb != wq.WQ_OK:
                    raise wq.WqError(stb, "batch")

                def seq():
                    for Rb, gb, cb, Mb, Kb in pts:
                        wq.assemble(Rb, gb, cb, vp, out=(Mb, Kb), stream=stream, check=False)

                seq()
                ts = float(np.mean(timed(seq, 2)))
                # the same algorithmic counts as the single-mesh line: contraction
                # flops against the FP64 (df64) pipe, the band bytes against HBM for FP32
                if vp == "mixed":
                    bw = bnnz * 4 / (tb * 1e-3) / 1e9
                    broof = {"bound": "hbm", "achieved": bw, "peak": hbm, "unit": "GB/s", "frac": bw / hbm}
                else:
                    pk = FP64_PEAK_TFLOPS if vp == "fp64" else DF64_PEAK_TFLOPS
                    tf = bflops / (tb * 1e-3) / 1e12
                    broof = {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s", "frac": tf / pk}
                bat[vp] = {"ms_per_step": tb, "value": bnnz / (tb * 1e-3), "unit": "nnz/s",
                           "ms_one_call_per_patch": ts, "config": Bp.config, "roofline": broof}
                Bp.close()
                del pts
                torch.cuda.empty_cache()
            variants[f"batch_{args.batch_patches}"] = bat
            for Rb in rules_cache.values():
                Rb.close()
            del base
    return variants


if __name__ == "__main__":
    sys.exit(main())
