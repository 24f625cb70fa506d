"""Benchmark: 3D cubic weighted-Gaussian mass+stiffness assembly, nnz/s.

One step = one mass+stiffness assembly call (coefficient check, geometry
fold, the partial-contraction kernel and the row kernel, all rows) of the
named synthetic workload through the C-ABI.  Default workload: 64^3 elements, C2 cubic (p = 3), separable map
xhat + 0.05 sin(pi xhat) per coordinate, c = exp(0.3 (x+y+z)) with
lognormal(0.1) noise as a cubic spline on the same mesh, FP64-accurate bands
(double output, <= 1e-12 relative to the FP64 oracle) computed in
double-float arithmetic on the FP32 pipe (--prec df64).  Timed beside it
("variants"): the plain FP64 form, the FP32 mixed mode, the comparison rules
(Gauss-Legendre rows, Newton-Cotes-type rule; FP64) with their quadrature
point totals, the 128^3 cubic workload in every precision, the adjoint on
the 96^3 cubic workload and the 256-patch batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload 3d_p3_64] [--prec df64|fp64|mixed] [--no-cpu-baseline]

Prints one JSON line.  value = assembled non-zeros (M and K) per second over
all ranks, device time (CUDA events around each step on the launching
stream, L2 flushed before each step by writing a 256 MiB buffer); e2e = the
same through host buffers (pinned H2D of geometry and coefficients, D2H of
both bands, inside the timed region).  Under torchrun every rank assembles
its own copy of the workload (weak scaling, no data-path collective).
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
# peaks
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz = 1.259
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 80.5
# double-float multiply-add = 12 FP32-pipe instructions (csrc/dd.cuh): FP64-equivalent peak
DF64_PEAK_TFLOPS = 152 * 128 / 12 * 2 * 2.070e9 / 1e12  # 6.71
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# capture of the current kernel (profiles/split_kernels_3d_p3_64_df64.md);
# absent entries report null
TRAFFIC = {("3d_p3_64", "df64"): {"bytes": 1.590632e9 + 0.236710e9, "kernel": "rows_ug_kernel<3, 32, M+K, dd>",
                                  "algorithmic_bytes": 2 * 300763 * 343 * 8}}


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

    n = [v + p for v in nel]
    r1 = rows_idx % n[0]
    r2 = (rows_idx // n[0]) % n[1]
    r3 = rows_idx // (n[0] * n[1])
    cnt = np.ones_like(rows_idx)
    for r, m in ((r1, n[0]), (r2, n[1]), (r3, n[2])):
        cnt = cnt * (np.minimum(m - 1, r + p) - np.maximum(0, r - p) + 1)
    return int(cnt.sum())


def cpu_sample_rows(nel, p, stride):
    """Every `stride`-th x3-slab of rows (interior and boundary rows alike)."""
    n = [v + p for v in nel]
    slab = n[0] * n[1]
    return [(s * slab, (s + 1) * slab) for s in range(0, n[2], stride)]


def run_cpu_baseline(w, g, c, stride, max_slabs=None):
    """Times the FP64 oracle on a sample of slabs with all host cores."""
    import numpy as np

    import oracle

    nel, p = w["nel"], w["p"]
    ranges = cpu_sample_rows(nel, p, stride)
    if max_slabs:
        ranges = ranges[:max_slabs]
    nnz = 0
    t0 = time.perf_counter()
    outs = []
    for rb, re in ranges:
        M, K, _ = oracle.assemble(3, p, nel, g, c, rb, re)
        outs.append((rb, re, M, K))
        nnz += 2 * band_nnz_rows(nel, p, np.arange(rb, re))
    dt = time.perf_counter() - t0
    rows = sum(re - rb for rb, re in ranges)
    return {"value": nnz / dt, "unit": "nnz/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(ranges)} x3-slabs (every {stride}th, {rows} rows of {int(np.prod([v + p for v in nel]))}), "
                      f"{dt:.1f} s wall"}, outs


def reference_arm(args):
    """The oracle as it stands, on the host cores, for the same workload."""
    import numpy as np

    from paper_1710_01048_gb300 import inputs

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, g, c = inputs.workload(args.workload)
    nel, p = w["nel"], w["p"]
    n = [v + p for v in nel]
    slab = n[0] * n[1]
    # each step: one x3-slab of rows (a bounded sample of the workload)
    import oracle

    oracle.build()
    for i in range(args.warmup):
        oracle.assemble(3, p, nel, g, c, slab * (i % n[2]), slab * (i % n[2] + 1))
    t = []
    nnz = 0
    for i in range(args.steps):
        s = (n[2] // 2 + i) % n[2]
        t0 = time.perf_counter()
        oracle.assemble(3, p, nel, g, c, slab * s, slab * (s + 1))
        t.append(time.perf_counter() - t0)
        nnz += 2 * band_nnz_rows(nel, p, np.arange(slab * s, slab * (s + 1)))
    total = sum(t)
    value = nnz / total
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "nel": list(nel), "degree": p, "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"one x3-slab ({slab} rows) per step"},
           "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d_p3_64")
    ap.add_argument("--prec", default="df64", choices=["fp64", "df64", "mixed"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-128", action="store_true", help="skip the 128^3 and adjoint variants")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-patch batch variant")
    ap.add_argument("--cpu-stride", type=int, default=8)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch

    from paper_1710_01048_gb300 import binding as wq
    from paper_1710_01048_gb300 import inputs

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

    w, g, c = inputs.workload(args.workload)
    dim, p, nel = w["dim"], w["p"], w["nel"]
    R = wq.Rules(dim, p, nel)
    rows, band = R.rows, R.band
    nnz_step = 2 * R.nnz  # M and K
    gd = [torch.from_numpy(x).cuda() for x in g]
    cd = torch.from_numpy(c).cuda()
    dt = torch.float32 if args.prec == "mixed" else torch.float64
    M = torch.empty((rows, band), dtype=dt, device="cuda")
    K = torch.empty((rows, band), dtype=dt, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        wq.assemble(R, gd, cd, args.prec, out=(M, K), stream=stream, check=False)

    for _ in range(args.warmup):
        step()
    st = wq.wq_status_check(R.handle, wq._stream_handle(stream))
    if st != wq.WQ_OK:
        raise wq.WqError(st, "warm-up")

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for e0, e1 in evs:
        flush.fill_(1)
        e0.record(stream)
        step()
        e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    ms_step = float(np.mean(ms))
    st = wq.wq_status_check(R.handle, wq._stream_handle(stream))
    if st != wq.WQ_OK:
        raise wq.WqError(st, "timed steps")
    # coefficient check/convert + fold + interior-line rows + boundary-line rows per step
    gpu_launches = 4 * args.steps

    # end to end through host buffers: pinned inputs H2D, both bands D2H
    # (measured before the variants, whose large allocations would otherwise
    # precede it)
    gh = [torch.from_numpy(x).pin_memory() for x in g]
    ch = torch.from_numpy(c).pin_memory()
    Mh = torch.empty((rows, band), dtype=dt).pin_memory()
    Kh = torch.empty((rows, band), dtype=dt).pin_memory()
    h2d = sum(x.numel() * 8 for x in gh) + ch.numel() * 8
    d2h = 2 * rows * band * M.element_size()
    e2e_steps = max(3, min(args.steps, 10))

    def e2e_step():
        # inputs to the device, then the assembly with its band copies to the
        # host overlapped range by range (binding.assemble_to_host)
        for dst, src in zip(gd, gh):
            dst.copy_(src, non_blocking=True)
        cd.copy_(ch, non_blocking=True)
        wq.assemble_to_host(R, gd, cd, args.prec, Mh, Kh, M, K, nchunks=8, stream=stream)

    e2e_step()
    barrier()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    t1e.record(stream)
    barrier()
    e2e_ms = t0e.elapsed_time(t1e) / e2e_steps

    # the other precisions on the same workload, a few steps each
    variants = {}
    peaks = measured_peaks()
    if not args.no_variants:
        for vp in ("fp64", "df64", "mixed"):
            if vp == args.prec:
                continue
            vdt = torch.float32 if vp == "mixed" else torch.float64
            Mv = torch.empty((rows, band), dtype=vdt, device="cuda")
            Kv = torch.empty((rows, band), dtype=vdt, device="cuda")
            for _ in range(3):
                wq.assemble(R, gd, cd, vp, out=(Mv, Kv), stream=stream, check=False)
            vms = []
            for _ in range(max(3, min(args.steps, 10))):
                flush.fill_(1)
                v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                v0.record(stream)
                wq.assemble(R, gd, cd, vp, out=(Mv, Kv), stream=stream, check=False)
                v1.record(stream)
                vms.append((v0, v1))
            torch.cuda.synchronize()
            vm = float(np.mean([x.elapsed_time(y) for x, y in vms]))
            ev = {"ms_per_step": vm, "value": world * nnz_step / (vm * 1e-3), "unit": "nnz/s",
                  "dtype": {"fp64": "f64", "df64": "f32x2", "mixed": "f32"}[vp]}
            if vp == "mixed":
                # accuracy of the FP32 bands against this run's FP64-accurate bands
                ev["max_rel_err_vs_fp64_bands"] = max(
                    float(((Mv.double() - M.double()).abs().max() / M.double().abs().max()).item()),
                    float(((Kv.double() - K.double()).abs().max() / K.double().abs().max()).item()))
            variants[vp] = ev
            del Mv, Kv
        torch.cuda.empty_cache()

        # the comparison rules (FP64, same kernel's general-points class):
        # Gauss-Legendre on every element of each row's support, and the
        # Newton-Cotes-type weighted rules; with the quadrature-point counts
        Mv = torch.empty((rows, band), dtype=torch.float64, device="cuda")
        Kv = torch.empty((rows, band), dtype=torch.float64, device="cuda")
        points = {}
        for mode in ("wq", "nc", "gl"):
            Rm = R if mode == "wq" else wq.Rules(dim, p, nel, rule=mode)
            total = 1
            for a in range(dim):
                total *= sum(len(Rm.row(a, 0, r)[0]) for r in range(nel[a] + p))
            points[mode] = {"points_per_interior_row_and_direction": len(Rm.row(0, 0, p)[0]),
                            "rule_points_total": total}
            if mode == "wq":
                continue
            for _ in range(3):
                wq.assemble(Rm, gd, cd, "fp64", out=(Mv, Kv), stream=stream, check=False)
            vms = []
            for _ in range(max(3, min(args.steps, 5))):
                flush.fill_(1)
                v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                v0.record(stream)
                wq.assemble(Rm, gd, cd, "fp64", out=(Mv, Kv), stream=stream, check=False)
                v1.record(stream)
                vms.append((v0, v1))
            torch.cuda.synchronize()
            vm = float(np.mean([x.elapsed_time(y) for x, y in vms]))
            variants["fp64_" + mode + "_rule"] = {"ms_per_step": vm, "value": world * nnz_step / (vm * 1e-3),
                                                  "unit": "nnz/s", "dtype": "f64", **points[mode]}
            Rm.close()
        variants["rule_points"] = points
        del Mv, Kv
        torch.cuda.empty_cache()

        # the 128^3 cubic workload (the precision configuration), every precision
        if args.workload == "3d_p3_64" and not args.no_128:
            w2, g2, c2 = inputs.workload("3d_p3_128")
            R2 = wq.Rules(3, w2["p"], w2["nel"])
            gd2 = [torch.from_numpy(x).cuda() for x in g2]
            cd2 = torch.from_numpy(c2).cuda()
            fl2, _ = R2.flops()
            big = {"workload": "3d_p3_128", "nel": list(w2["nel"]), "nnz_per_matrix": R2.nnz}
            for vp in ("df64", "fp64", "mixed"):
                vdt = torch.float32 if vp == "mixed" else torch.float64
                Mv = torch.empty((R2.rows, R2.band), dtype=vdt, device="cuda")
                Kv = torch.empty((R2.rows, R2.band), dtype=vdt, device="cuda")
                for _ in range(3):
                    wq.assemble(R2, gd2, cd2, vp, out=(Mv, Kv), stream=stream, check=False)
                vms = []
                for _ in range(max(3, min(args.steps, 5))):
                    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    v0.record(stream)
                    wq.assemble(R2, gd2, cd2, vp, out=(Mv, Kv), stream=stream, check=False)
                    v1.record(stream)
                    vms.append((v0, v1))
                torch.cuda.synchronize()
                vm = float(np.mean([x.elapsed_time(y) for x, y in vms]))
                ent = {"ms_per_step": vm, "value": world * 2 * R2.nnz / (vm * 1e-3), "unit": "nnz/s"}
                if vp == "mixed":
                    bw = 2 * R2.rows * R2.band * 4 / (vm * 1e-3) / 1e9
                    ent["roofline"] = {"bound": "hbm", "achieved": bw, "peak": peaks.get("hbm_gbs", 6800.0),
                                       "unit": "GB/s", "frac": bw / peaks.get("hbm_gbs", 6800.0)}
                else:
                    pk = FP64_PEAK_TFLOPS if vp == "fp64" else DF64_PEAK_TFLOPS
                    tf = fl2 / (vm * 1e-3) / 1e12
                    ent["roofline"] = {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s", "frac": tf / pk}
                big[vp] = ent
                del Mv, Kv
                torch.cuda.empty_cache()
            st2 = wq.wq_status_check(R2.handle, wq._stream_handle(stream))
            if st2 != wq.WQ_OK:
                raise wq.WqError(st2, "128^3 variant")
            variants["3d_p3_128"] = big
            R2.close()
            del gd2, cd2

        # the adjoint (coefficient gradient of sum G*K + H*M) on the 96^3 cubic workload
        if args.workload == "3d_p3_64" and not args.no_128:
            w3, g3, c3 = inputs.workload("3d_p3_96")
            R3 = wq.Rules(3, w3["p"], w3["nel"])
            gd3 = [torch.from_numpy(x).cuda() for x in g3]
            gen = torch.Generator(device="cuda").manual_seed(96)
            adj = {"workload": "3d_p3_96", "ncoef": R3.ncoef}
            for vp in ("fp64", "df64", "mixed"):
                vdt = torch.float32 if vp == "mixed" else torch.float64
                G = torch.randn((R3.rows, R3.band), dtype=vdt, device="cuda", generator=gen)
                H = torch.randn((R3.rows, R3.band), dtype=vdt, device="cuda", generator=gen)
                grad = torch.empty(R3.ncoef, dtype=torch.float64, device="cuda")
                for _ in range(3):
                    wq.assemble_adjoint(R3, gd3, G, H, vp, out=grad, stream=stream, check=False)
                vms = []
                for _ in range(max(3, min(args.steps, 5))):
                    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    v0.record(stream)
                    wq.assemble_adjoint(R3, gd3, G, H, vp, out=grad, stream=stream, check=False)
                    v1.record(stream)
                    vms.append((v0, v1))
                torch.cuda.synchronize()
                vm = float(np.mean([x.elapsed_time(y) for x, y in vms]))
                # per step the adjoint reads both weight bands: report band entries per second
                adj[vp] = {"ms_per_step": vm, "value": 2 * R3.nnz / (vm * 1e-3), "unit": "nnz/s (weights read)",
                           "weights_gb_s": 2 * R3.rows * R3.band * G.element_size() / (vm * 1e-3) / 1e9}
                del G, H, grad
                torch.cuda.empty_cache()
            variants["adjoint_3d_p3_96"] = adj
            R3.close()

        # matrix-free apply y = M x, y = K x (the band never stored) and the
        # load vector, on the same workload as the headline
        if args.workload == "3d_p3_64":
            gen = torch.Generator(device="cuda").manual_seed(64)
            app = {"workload": args.workload, "nnz_per_step": nnz_step}
            for vp in ("df64", "fp64", "mixed"):
                vdt = torch.float32 if vp == "mixed" else torch.float64
                xv = torch.randn(rows, dtype=torch.float64, device="cuda", generator=gen).to(vdt)
                yM = torch.empty(rows, dtype=vdt, device="cuda")
                yK = torch.empty(rows, dtype=vdt, device="cuda")
                for _ in range(3):
                    wq.apply(R, gd, xv, cd, vp, out=(yM, yK), stream=stream, check=False)
                vms = []
                for _ in range(max(3, min(args.steps, 10))):
                    flush.fill_(1)
                    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    v0.record(stream)
                    wq.apply(R, gd, xv, cd, vp, out=(yM, yK), stream=stream, check=False)
                    v1.record(stream)
                    vms.append((v0, v1))
                torch.cuda.synchronize()
                vm = float(np.mean([x.elapsed_time(y) for x, y in vms]))
                # the contractions plus one multiply-add per band entry and matrix
                fl_apply = R.flops()[0] + 2 * 2 * R.nnz
                pk = {"fp64": FP64_PEAK_TFLOPS, "df64": DF64_PEAK_TFLOPS, "mixed": FP32_PEAK_TFLOPS}[vp]
                tf = fl_apply / (vm * 1e-3) / 1e12
                app[vp] = {"ms_per_step": vm, "value": world * nnz_step / (vm * 1e-3), "unit": "nnz/s (applied)",
                           "roofline": {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s",
                                        "frac": tf / pk}}
                if vp == "df64":
                    bl = torch.empty(rows, dtype=vdt, device="cuda")
                    for _ in range(3):
                        wq.assemble_load(R, gd, cd, vp, out=bl, stream=stream, check=False)
                    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    v0.record(stream)
                    for _ in range(5):
                        wq.assemble_load(R, gd, cd, vp, out=bl, stream=stream, check=False)
                    v1.record(stream)
                    torch.cuda.synchronize()
                    app["load_vector_df64_ms"] = v0.elapsed_time(v1) / 5
                    del bl
                del xv, yM, yK
            sta = wq.wq_status_check(R.handle, wq._stream_handle(stream))
            if sta != wq.WQ_OK:
                raise wq.WqError(sta, "apply variant")
            variants["apply_3d_p3_64"] = app

        # the batch of 256 independent patches (8..48 elements per direction, p in {2, 3}):
        # one graph of two persistent launches, tuned, against one call per patch
        if not args.no_batch:
            specs = inputs.batch_patches(256, seed=0)
            rules_cache, base = {}, []
            for sp in specs:
                key = (sp["p"], sp["nel"])
                if key not in rules_cache:
                    rules_cache[key] = wq.Rules(3, sp["p"], sp["nel"])
                base.append((rules_cache[key], [torch.from_numpy(x).cuda() for x in sp["geom"]],
                             torch.from_numpy(sp["coef"]).cuda()))
            bnnz = 2 * sum(Rb.nnz for Rb, _, _ in base)
            bat = {"workload": "batch_256", "patches": 256, "nnz_per_step": bnnz}
            for vp in ("fp64", "df64", "mixed"):
                vdt = torch.float32 if vp == "mixed" else torch.float64
                pts = [(Rb, gb, cb, torch.empty((Rb.rows, Rb.band), dtype=vdt, device="cuda"),
                        torch.empty((Rb.rows, Rb.band), dtype=vdt, device="cuda")) for Rb, gb, cb in base]
                Bp = wq.Batch(pts, vp)
                Bp.tune(reps=1, stream=stream)

                def timed(fn, n):
                    fn()
                    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    v0.record(stream)
                    for _ in range(n):
                        fn()
                    v1.record(stream)
                    torch.cuda.synchronize()
                    return v0.elapsed_time(v1) / n

                tb = timed(lambda: Bp.launch(stream), 5)
                stb = Bp.status(stream)
                if stb != wq.WQ_OK:
                    raise wq.WqError(stb, "batch")

                def seq():
                    for Rb, gb, cb, Mb, Kb in pts:
                        wq.assemble(Rb, gb, cb, vp, out=(Mb, Kb), stream=stream, check=False)

                ts = timed(seq, 2)
                bat[vp] = {"ms_per_step": tb, "value": bnnz / (tb * 1e-3), "unit": "nnz/s",
                           "ms_one_call_per_patch": ts, "config": Bp.config}
                Bp.close()
                del pts
                torch.cuda.empty_cache()
            variants["batch_256"] = bat
            for Rb in rules_cache.values():
                Rb.close()
            del base


    # max over ranks
    if dist is not None:
        from paper_1710_01048_gb300 import shard

        ms_step, e2e_ms = shard.max_over_ranks([ms_step, e2e_ms], dist, device="cuda")

    value = world * nnz_step / (ms_step * 1e-3)
    e2e_value = world * nnz_step / (e2e_ms * 1e-3)

    # roofline of the assembly call (fold + the two row launches; the fold is
    # a few microseconds): algorithmic contraction flops / device time
    flops, coef_flops = R.flops()
    if args.prec == "fp64":
        achieved = flops / (ms_step * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (not in MEASURED_PEAKS.json)",
                "achieved_incl_coef_eval": (flops + coef_flops) / (ms_step * 1e-3) / 1e12}
    elif args.prec == "df64":
        achieved = flops / (ms_step * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": DF64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / DF64_PEAK_TFLOPS,
                "traffic": TRAFFIC.get((args.workload, "df64"), {}).get("bytes"),
                "traffic_note": TRAFFIC.get((args.workload, "df64")),
                "peak_source": "derived: FP32 pipe 152 SMs x 128 lanes x 2.07 GHz / 12 FP32 instructions per "
                               "double-float multiply-add, x 2 flop (FP64-equivalent)",
                "achieved_incl_coef_eval": (flops + coef_flops) / (ms_step * 1e-3) / 1e12}
    else:
        bytes_step = 2 * rows * band * 4
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = bytes_step / (ms_step * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
                else "fallback 6.8 TB/s",
                "fp32_tflops": (flops + coef_flops) / (ms_step * 1e-3) / 1e12, "fp32_peak_tflops": FP32_PEAK_TFLOPS}

    out = {"metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {"fp64": "f64", "df64": "f32x2", "mixed": "f32"}[args.prec],
           "data": "synthetic",
           "config": {"workload": args.workload, "nel": list(nel), "degree": p, "rows": rows, "band": band,
                      "nnz_per_matrix": R.nnz, "precision": args.prec,
                      "l2": "256 MiB buffer written before each timed step; each step also writes "
                            f"{2 * rows * band * M.element_size() / 1e9:.2f} GB of band output"},
           "roofline": roof,
           "e2e": {"value": e2e_value, "unit": "nnz/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
           "clocks": clocks, "gpu_launches": gpu_launches, "ms_per_step_min": float(np.min(ms)),
           "variants": variants}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, outs = run_cpu_baseline(w, g, c, args.cpu_stride, max_slabs=None)
        out["cpu_baseline"] = cpu
        # accuracy of this run's bands on the sampled rows against the oracle
        emax = 0.0
        for rb, re, Mo, Ko in outs:
            for A, O in ((M[rb:re], Mo), (K[rb:re], Ko)):
                d = A.double().cpu().numpy() - O
                emax = max(emax, float(np.max(np.abs(d)) / np.max(np.abs(O))))
        out["max_rel_err_vs_oracle"] = emax
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    R.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
