#!/usr/bin/env python
"""Benchmark of the SIP-DG Stokes solver library on one GB300.

Metric: Stokes solves per second to a 1e-8 relative residual on the
single-inclusion workload (128 x 128 elements, k = 3, a square inclusion of
viscosity 1e4 and density 1.2 in a unit medium, Neumann top / Navier
elsewhere, Q^2_1 coarse space + 3 h-coarsenings, 2+2 element-block-Jacobi /
Chebyshev steps), FP64 form; the mixed-precision form, the SIP-apply
bandwidth and the p50/p99 step latency are reported beside it.

One step = a complete solve of a fresh viscosity field: copy of eta, the
whole multigrid set-up (block-Jacobi inverses, eigenvalue estimates,
Galerkin coarse operators, coarsest inverse), the load vector and the
block-preconditioned FGMRES solve, with every input resident in HBM.  L2 is
flushed (a 256 MB write) before every timed step.

``--impl reference`` times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload on the host cores.
Under torchrun (N > 1) every rank solves its own instance (replicas,
weak scaling); rank 0 prints the JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "stokes_solves_per_s_to_1e-8_residual"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner-rtol", type=float, default=1e-3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-precision", default="fp64", choices=["fp64", "mixed"],
                    help="form timed by --profile-only")
    ap.add_argument("--profile-n", type=int, default=128,
                    help="mesh side of the --profile-only run (same physics)")
    ap.add_argument("--profile-k", type=int, default=3,
                    help="polynomial degree of the --profile-only run")
    ap.add_argument("--inner-loop", default="device", choices=["device", "host"],
                    help="inner PCG loop on the device (one graph launch per inner solve) or "
                         "driven from the host (for profilers that cannot see kernels inside "
                         "graphs with conditional nodes)")
    ap.add_argument("--profile-only", action="store_true",
                    help="run only the warm-up and timed FP64 steps (for ncu launch lists)")
    ap.add_argument("--mode", default="solve",
                    choices=["solve", "batch", "serve", "coarse", "sinkers", "checkerboard",
                             "kernel"],
                    help="solve: the headline line; batch / serve: the batched and served "
                         "forms on bounded samples of their workloads; coarse: the four "
                         "coarse-space preconditioners; sinkers / checkerboard: the "
                         "six-sinker and checkerboard iteration sweeps (extra lines); "
                         "kernel: a few launches of one operator on a small case, the "
                         "command the ncu captures under profiles/ run")
    ap.add_argument("--kernel", default="apply_f64",
                    choices=["apply_f64", "apply_f32", "vcycle_f32"],
                    help="operator run by --mode kernel: the FP64 or FP32 SIP apply on a "
                         "random viscosity field, or one FP32 V-cycle of the many-discs field")
    ap.add_argument("--apply-code", default="",
                    help="--mode kernel and --profile-only: pinned SIP apply schedule codes "
                         "'FP64[,FP32]' (1 elem2, 2 elem1, 3 tile, 4 staged 2 rows, 5 staged "
                         "4 rows, 6 warp-row (FP32 only); empty leaves the tuner's choice, which timings taken "
                         "under a profiler can mislead)")
    ap.add_argument("--count", type=int, default=32,
                    help="instances (batch) or requests (serve) in the bounded sample")
    ap.add_argument("--sinker-inner", default="gcr",
                    choices=["gcr", "pcg-true", "pcg-preconditioned"],
                    help="inner Krylov method of the six-sinker sweep: GCR (the paper's, "
                         "Sec. 7.3) or PCG with either stopping test")
    ap.add_argument("--sinker-outer", default="gcr", choices=["gcr", "fgmres"],
                    help="outer Krylov method of the six-sinker sweep (the paper's: GCR)")
    ap.add_argument("--checker-inner", default="pcg-true",
                    choices=["pcg-true", "pcg-preconditioned", "gcr"],
                    help="inner Krylov method and stopping test of the checkerboard sweep")
    ap.add_argument("--refine", type=int, default=4,
                    help="batch: iterative refinement with a double-double residual, the "
                         "most correction solves (0: off), in both arms")
    ap.add_argument("--serve-refine", type=int, default=0,
                    help="serve: the same for the served requests and their FP64 arm")
    ap.add_argument("--serve-max-log-contrast", type=float, default=5.0,
                    help="serve: contrasts 10^U[0, this]")
    ap.add_argument("--sinker-refine", type=int, default=0,
                    help="iterative refinement with a double-double residual in the "
                         "six-sinker sweep: the most correction solves (0: off)")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline line only: no many-disc, batched or served samples")
    ap.add_argument("--c3-max-inner", type=int, default=20,
                    help="inner iteration cap of the many-disc sample")
    ap.add_argument("--batch-count", type=int, default=16,
                    help="instances of the batched sample in the headline line")
    ap.add_argument("--serve-count", type=int, default=12,
                    help="requests of each served sample in the headline line")
    ap.add_argument("--sinker-min-eta", type=float, default=1e3,
                    help="smallest viscosity contrast of the six-sinker sweep")
    ap.add_argument("--sinker-max-eta", type=float, default=1e8,
                    help="largest viscosity contrast of the six-sinker sweep")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ ranks
def max_over_ranks(value, world, device=None):
    """Largest per-rank value over all ranks (the slowest rank's time);
    identity on one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps, world, total_ms):
    """Solves per second of the whole job: every rank solves ``steps``
    independent instances; the job takes as long as its slowest rank."""
    return world * steps / (total_ms / 1000.0)


# ------------------------------------------------------------------ ours
def algorithmic_apply(prob_k, ne, word):
    """Algorithmic bytes and flops of one SIP apply, per element: read x,
    write y (2 n^2 coefficients each) and read eta_K; 16 n^3 flops for the
    volume terms by sum-factorisation plus 128 n^2 for the face terms
    (n = k + 1).  Neighbour re-reads are not algorithmic."""
    n = prob_k + 1
    nb = 2 * n * n
    bytes_ = ne * (2 * nb * word + word)
    flops = ne * (16 * n ** 3 + 128 * n * n)
    return bytes_, flops


def headline_config(args):
    """The headline workload's configuration, shared by both arms: the
    128^2, k = 3 box inclusion (eta 1e4) with Q^2_1 + 3 h-levels, FP64,
    FGMRES to 1e-8 with PCG stopped on the residual at inner_rtol."""
    from paper_1607_03777_gb300 import synth
    wl = synth.single_box_inclusion()
    return {"workload": "single_box_inclusion_128x128_k3_eta1e4_Q1+3h",
            "nx": wl.nx, "ny": wl.ny, "k": wl.k, "n_hlevels": wl.n_hlevels, "rtol": wl.rtol,
            "inner_rtol": args.inner_rtol, "inner_norm": "true", "inner_krylov": "pcg",
            "precision": "fp64"}


def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_1607_03777_gb300 import api, synth

    dev = torch.device("cuda", rank % max(1, torch.cuda.device_count()))
    torch.cuda.set_device(dev)
    ctx = api.Context(dev.index)
    wl = synth.single_box_inclusion(
        n=args.profile_n, k=args.profile_k,
        n_hlevels=synth.levels_to_17(args.profile_n)) if args.profile_only \
        else synth.single_box_inclusion()
    n, k = wl.nx, wl.k
    eta_d, rho_d = ctx.rasterise_inclusions(n, n, wl.shapes)
    eta_h = eta_d.cpu().numpy()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def make(precision):
        prob = api.Problem(ctx, n, n, k, eta_h, bc=wl.bc, n_hlevels=wl.n_hlevels, seed=1,
                           precision=precision)
        if args.profile_only and apply_codes(args):
            prob.set_schedule(apply=apply_codes(args))
        f = torch.empty(prob.n_u, dtype=torch.float64, device=dev)
        u = torch.empty_like(f)
        p = torch.empty(prob.n_p, dtype=torch.float64, device=dev)
        return prob, f, u, p

    # The library default and the paper's configuration (Sec. 7.1): PCG
    # stopped on the residual.  The preconditioned-residual test is timed
    # beside it (the host-driven loop implements only the residual test).
    head_norm = "true"
    alt_norm = None if args.inner_loop == "host" else "preconditioned"

    def step(prob, f, u, p, inner_norm=head_norm):
        prob.update_eta(eta_d)
        prob.rhs_body_force(rho_d, synth.GRAVITY, f)
        return prob.solve(f, u, p, rtol=wl.rtol, inner_rtol=args.inner_rtol, max_outer=1000,
                          inner_loop=args.inner_loop, inner_norm=inner_norm,
                          check=not args.profile_only)

    def timed(precision, steps, warmup, clocks=None, inner_norm=head_norm, profiler_range=False):
        prob, f, u, p = make(precision)
        for _ in range(warmup):
            step(prob, f, u, p, inner_norm)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        times, reps = [], []
        if clocks:
            clocks.start()
        if profiler_range:
            torch.cuda.profiler.start()
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reps.append(step(prob, f, u, p, inner_norm))
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        clocks_out = clocks.stop() if clocks else None
        torch.cuda.synchronize()
        if profiler_range:
            torch.cuda.profiler.stop()
        return prob, f, u, p, times, reps, clocks_out

    clocks = ClockSampler(dev.index)
    if args.profile_only:   # one form only, for profiler launch lists
        # (the timed steps are the CUDA profiler range: ncu --profile-from-start off)
        _, _, _, _, tp, rp, _ = timed(args.profile_precision, args.steps, args.warmup,
                                      profiler_range=True)
        return {"metric": METRIC, "value": whole_job_rate(args.steps, 1, sum(tp)), "unit": UNIT,
                "profile_only": True, "precision": args.profile_precision,
                "solve_report": rp[-1]}
    prob64, f64, u64, p64, t64, r64, clk = timed("fp64", args.steps, args.warmup, clocks)
    total_ms = max_over_ranks(sum(t64), world, dev)
    value = whole_job_rate(args.steps, world, total_ms)

    # mixed-precision form on the same workload
    prob32, f32, u32, p32, t32, r32, _ = timed("mixed", args.steps, max(1, args.warmup - 1))
    err_mixed = float(torch.linalg.norm(u32 - u64) / torch.linalg.norm(u64))
    sched_mixed = prob32.schedule()
    del prob32

    # the preconditioned-residual inner test on the same workload
    td, rd = [], []
    if alt_norm:
        probd, _, _, _, td, rd, _ = timed("fp64", args.steps, max(1, args.warmup - 1),
                                          inner_norm=alt_norm)
        del probd

    # end to end through the public API with host buffers (pinned)
    eta_pin = torch.from_numpy(eta_h).pin_memory()
    rho_pin = rho_d.cpu().pin_memory()
    u_pin = torch.empty(prob64.n_u, dtype=torch.float64).pin_memory()
    p_pin = torch.empty(prob64.n_p, dtype=torch.float64).pin_memory()
    eta_dd = torch.empty_like(eta_d)
    rho_dd = torch.empty_like(rho_d)
    e2e_ms = []
    for i in range(args.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eta_dd.copy_(eta_pin, non_blocking=True)
        rho_dd.copy_(rho_pin, non_blocking=True)
        prob64.update_eta(eta_dd)
        prob64.rhs_body_force(rho_dd, synth.GRAVITY, f64)
        prob64.solve(f64, u64, p64, rtol=wl.rtol, inner_rtol=args.inner_rtol, max_outer=1000,
                     inner_norm=head_norm)
        u_pin.copy_(u64, non_blocking=True)
        p_pin.copy_(p64, non_blocking=True)
        torch.cuda.synchronize()
        if i > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1000.0)
    e2e_value = world * len(e2e_ms) / (sum(e2e_ms) / 1000.0)

    # live timing of the dominant kernel, the FP64 SIP apply, on this
    # stream: one event pair per launch, L2 flushed between launches
    x = torch.randn(prob64.n_u, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    for _ in range(5):
        prob64.apply_A(x, y, stream=stream)
    reps_apply = 50
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps_apply)]
    for e0, e1 in ev:
        with torch.cuda.stream(stream):
            flush.add_(1.0)
        e0.record(stream)
        prob64.apply_A(x, y, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    apply_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / reps_apply
    ab, af = algorithmic_apply(k, n * n, 8)
    sched64 = prob64.schedule()
    dominant = kernel_name(sched64["apply"][0], k, 8)
    peaks = measured_alu_peaks(dev)
    f32_lines = apply_f32_rooflines(ctx, dev, flush, stream, peaks)

    launches = sum(r["kernel_launches"] for r in r64)
    lat = sorted(t64)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(headline_config(args),
                       step="eta copy + multigrid set-up + load vector + FGMRES solve",
                       l2="flushed (256 MB write) before every timed step"),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "solve_report": {key: r64[-1][key] for key in ("outer_its", "inner_avg", "inner_max",
                                                       "rel_residual", "setup_ms", "solve_ms")},
        "mixed": {"value": world * args.steps / (sum(t32) / 1000.0), "unit": UNIT,
                  "ms_per_step": sum(t32) / args.steps,
                  "rel_residual": r32[-1]["rel_residual"], "outer_its": r32[-1]["outer_its"],
                  "inner_avg": r32[-1]["inner_avg"], "u_rel_diff_vs_fp64": err_mixed},
        "fp64_preconditioned_inner_test": None if not td else {
            "value": world * args.steps / (sum(td) / 1000.0), "unit": UNIT,
            "inner_norm": alt_norm, "ms_per_step": sum(td) / args.steps,
            "outer_its": rd[-1]["outer_its"], "inner_avg": rd[-1]["inner_avg"]},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(eta_h.nbytes + rho_pin.numel() * 8),
                "d2h_bytes_per_step": int((prob64.n_u + prob64.n_p) * 8)},
        "gpu_launches": int(launches),
        "schedule": {"fp64": sched64, "mixed": sched_mixed},
        "clocks": clk,
        "sip_apply": {"kernel": dominant, "ms": apply_ms,
                      "GB_per_s": ab / apply_ms / 1e6, "GFLOP_per_s": af / apply_ms / 1e6,
                      "dof_per_s": prob64.n_u / (apply_ms / 1e3)},
    }
    traffic = captured_traffic(dominant)
    out["roofline"] = roofline(ab, af, apply_ms, dominant, traffic, peaks)
    out["sip_apply_f32"] = f32_lines
    out["alu_peaks_TFLOP_per_s"] = peaks
    if not args.no_extras and rank == 0:
        # bounded samples of the many-disc, batched and served workloads
        # (outside the timed region; sample sizes stated in each object)
        out["c3"] = c3_sample(ctx, args.c3_max_inner, refine=4)
        out["batch"] = batch_sample(ctx, args.batch_count, refine=4)
        out["batch_small"] = batch_small_sample(ctx)
        hi = serve_sample(ctx, args.serve_count, refine=4, max_log_contrast=6.0)
        # offered load at half the throughput measured at 200 / s: latency
        # there is service time, not backlog
        lo = serve_sample(ctx, args.serve_count, refine=4, max_log_contrast=6.0,
                          rate=max(0.05, 0.5 * hi["value"]))
        out["serve"] = {"at_200_per_s": hi, "below_capacity": lo}
    return out


# FP64 peak of one GB300, derived from unit counts and clocks: 152 SMs x
# 2 FP64 FMA per SM per clock x 2 FLOP x 2.07 GHz (maximum SM clock)
# = 1.259 TFLOP/s (NVIDIA's figure: 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# the same count for FP32: 128 FMA per SM per clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def kernel_name(code, k, word):
    """The SIP apply kernel that sip_problem_schedule's code selects."""
    n, t = k + 1, "double" if word == 8 else "float"
    return {1: f"k_apply_elem2<{n},{t},1>", 2: f"k_apply_elem<{n},{t}>",
            3: f"k_apply_sip<{n},{t}>", 4: f"k_apply_stage<{n},{t},{t},2,1,0>",
            5: f"k_apply_stage<{n},{t},{t},4,1,0>", 6: f"k_apply_warp<{n},1>"}.get(code, f"code {code}")


def measured_alu_peaks(dev):
    """FP64 and FP32 arithmetic peaks measured on this GPU by library GEMMs
    (torch.matmul, 8192^3, FP32 without TF32), best of 5 CUDA-event timings:
    the denominators of the ALU-bound rooflines."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
            n = 8192
            a = torch.randn(n, n, dtype=dt, device=dev)
            b = torch.randn(n, n, dtype=dt, device=dev)
            c = a @ b
            best = 1e30
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def hbm_peak():
    """Measured copy bandwidth of the GB300s (GB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s"


def time_launches(fn, flush, stream, reps=30):
    """Mean device time (ms) of one launch of fn on `stream`, L2 flushed
    (a 256 MB write) before every launch, CUDA events around each launch."""
    import torch
    for _ in range(3):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for e0, e1 in ev:
        with torch.cuda.stream(stream):
            flush.add_(1.0)
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in ev) / reps


def apply_f32_rooflines(ctx, dev, flush, stream, peaks):
    """The FP32 SIP apply (the operator of the mixed V-cycle) on 512^2
    meshes, k = 3 and 4, the kernel the autotuner picks: algorithmic bytes
    and FLOPs per launch over its CUDA-event time, against the measured HBM
    copy bandwidth and the measured FP32 GEMM rate.  The algorithmic
    intensity (16 n^3 + 128 n^2 FLOP per 2 (2 n^2) + 1 words) is 11.8 FLOP/B
    at k = 3 and 12.9 at k = 4, above the FP32 ridge point (peak FLOP/s over
    HBM B/s), so both fractions are reported."""
    import torch
    from paper_1607_03777_gb300 import api, synth
    hbm, hbm_src = hbm_peak()
    out = []
    for k in (3, 4):
        n = 512
        pr = api.Problem(ctx, n, n, k, synth.random_eta(n * n, 1, (0.0, 3.0)), n_hlevels=5,
                         seed=1, precision="mixed", mixed_fp64_ratio=0.0)
        pr.setup()   # autotunes the FP32 kernel for this mesh
        x = torch.randn(pr.n_u, dtype=torch.float32, device=dev)
        y = torch.empty_like(x)
        ms = time_launches(lambda: pr.apply_A_f32(x, y, stream=stream), flush, stream)
        ab, af = algorithmic_apply(k, n * n, 4)
        code = pr.schedule()["apply"][1]
        kernel = kernel_name(code, k, 4)
        out.append({"elements": f"{n}x{n}", "k": k, "kernel": kernel,
                    "traffic": captured_traffic(kernel),
                    "ms": ms, "GB_per_s": ab / ms / 1e6, "hbm_frac": ab / ms / 1e6 / hbm,
                    "TFLOP_per_s": af / ms / 1e9, "fp32_frac": af / ms / 1e9 / peaks["fp32"],
                    "algorithmic_bytes": ab, "algorithmic_flops": af,
                    "hbm_peak_GB_per_s": hbm, "hbm_peak_source": hbm_src,
                    "fp32_peak_TFLOP_per_s": peaks["fp32"],
                    "fp32_peak_source": "measured: cuBLAS SGEMM 8192^3 (torch.matmul, no TF32)"})
        del pr
    return out


# committed ncu summaries of kernels in their current form: the FP64 staged apply on the
# 128^2, k = 3 workload and the FP32 warp-row apply on 512^2 (a kernel without one
# reports traffic null)
TRAFFIC_PROFILES = {
    "k_apply_stage<4,double,double,4,1,0>": os.path.join(
        ROOT, "profiles", "k_apply_stage4_fp64_128x128_k3.md"),
    # the warp-row FP32 apply on the 512^2 meshes of sip_apply_f32
    "k_apply_warp<4,1>": os.path.join(ROOT, "profiles", "k_apply_warp_fp32_512x512_k3.md"),
    "k_apply_warp<5,1>": os.path.join(ROOT, "profiles", "k_apply_warp_fp32_512x512_k4.md"),
}


def captured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from its committed ncu summary
    (dram__bytes_read.sum + dram__bytes_write.sum), or None."""
    path = TRAFFIC_PROFILES.get(kernel)
    if not path or not os.path.exists(path):
        return None
    vals = {}
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    for line in open(path):
        for key in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            if f"`{key}`" in line:
                cells = [c.strip() for c in line.strip().strip("|").split("|")]
                vals[key] = float(cells[1]) * scale.get(cells[2], 1.0)
    if len(vals) != 2:
        return None
    return vals["dram__bytes_read.sum"] + vals["dram__bytes_write.sum"]


def roofline(ab, af, apply_ms, kernel, traffic, peaks):
    """FP64 on GB300 is bound by the FP64 pipe, not HBM: achieved FP64
    FLOP/s of the SIP apply (algorithmic FLOPs / live launch time) against the
    FP64 peak measured by cuBLAS DGEMM on this GPU (the unit-count figure
    beside it)."""
    achieved = af / apply_ms / 1e9
    peak = peaks["fp64"]
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": kernel, "algorithmic_bytes": ab, "algorithmic_flops": af,
            "hbm_GB_per_s": ab / apply_ms / 1e6,
            "peak_source": "measured: cuBLAS DGEMM 8192^3 (torch.matmul), best of 5",
            "peak_derived": FP64_PEAK_TFLOPS,
            "peak_derived_source": "152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz",
            "frac_of_derived": achieved / FP64_PEAK_TFLOPS}


# ------------------------------------------------------------------ oracle
ORACLE_SIZES = (16, 24, 32)   # meshes of the timed oracle samples (3 h-coarsenings each)


def oracle_sample(n):
    """One FP64 oracle solve of the headline physics (box inclusion 1e4,
    k = 3, Q^2_1 + 3 h-coarsenings, FGMRES to 1e-8 with PCG stopped on the
    residual at 1e-3) on an n x n mesh: assembly, multigrid set-up and solve,
    single-threaded SciPy.  Returns (seconds, outer iterations)."""
    import numpy as np
    from oracle import krylov, materials, multigrid, sip
    from paper_1607_03777_gb300 import synth
    wl = synth.single_box_inclusion(n=n, n_hlevels=3)
    eta, rho = materials.rasterise_inclusions(n, n, wl.shapes)
    t0 = time.perf_counter()
    pr = sip.Problem(n, n, wl.k, eta, bc=wl.bc)
    A, B = sip.assemble_A(pr), sip.assemble_B(pr)
    f = sip.rhs_body_force(pr, rho)
    mg = multigrid.HPMultigrid(pr, A, 3, seed=1)
    Pc = krylov.BlockPreconditioner(A, B, sip.schur_mass(pr), mg, 1e-3)   # residual inner test
    K = krylov.stokes_matrix(A, B)
    b = np.concatenate([f, np.zeros(B.shape[1])])
    x, its, _ = krylov.fgmres(lambda v: K @ v, Pc, b, 1e-8, maxit=1000)
    return time.perf_counter() - t0, its


# BLAS thread counts of the oracle's processes: one each, so that a process
# uses one host core (numpy is first imported in the spawned child)
_BLAS_THREADS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                 "BLIS_NUM_THREADS")


def _oracle_worker(n, reps, q):
    q.put((n, [oracle_sample(n) for _ in range(reps)]))


def run_oracle_processes(jobs):
    """Oracle samples in spawned processes, one per (n, reps) job, each with
    single-threaded BLAS; returns {n: [(seconds, outer iterations), ...]}."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    saved = {k: os.environ.get(k) for k in _BLAS_THREADS}
    os.environ.update({k: "1" for k in _BLAS_THREADS})
    try:
        procs = [ctx.Process(target=_oracle_worker, args=(n, reps, q)) for n, reps in jobs]
        for p in procs:
            p.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    got = {}
    for _ in procs:
        n, res = q.get()
        got[n] = res
    for p in procs:
        p.join()
    return got


def oracle_scaling():
    """The oracle timed on several mesh sizes at once (one spawned process
    each, one host core each), and the growth of its time in the element
    count fitted to them by least squares in log-log; the 128^2 time is that
    fit evaluated at 128^2 (an extrapolation, labelled as such)."""
    import math
    res = run_oracle_processes([(n, 1) for n in ORACLE_SIZES])
    got = {n: res[n][0] for n in ORACLE_SIZES}
    xs = [math.log(n * n) for n in ORACLE_SIZES]
    ys = [math.log(got[n][0]) for n in ORACLE_SIZES]
    mx, my = sum(xs) / len(xs), sum(ys) / len(ys)
    alpha = sum((x - mx) * (y - my) for x, y in zip(xs, ys)) / sum((x - mx) ** 2 for x in xs)
    t128 = math.exp(my + alpha * (math.log(128 * 128) - mx))
    return {"samples": {f"{n}x{n}": {"s": got[n][0], "outer_its": got[n][1]} for n in ORACLE_SIZES},
            "exponent": alpha, "extrapolated_s_128x128": t128,
            "cores": len(ORACLE_SIZES), "host_cpus": os.cpu_count()}


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    A step is one oracle solve of the headline physics on a 16 x 16 mesh
    (the full 128 x 128 solve takes the oracle minutes): the line's value
    and ms_per_step are what was timed; the 128 x 128 estimate is beside
    them."""
    n0 = ORACLE_SIZES[0]
    runs = run_oracle_processes([(n0, args.warmup + args.steps)])[n0]   # one core
    per = [dt for dt, _ in runs[args.warmup:]]
    its = runs[-1][1]
    value = len(per) / sum(per)
    cfg = dict(headline_config(args),
               workload=f"single_box_inclusion_{n0}x{n0}_k3_eta1e4_Q1+3h (oracle sample of the "
                        "128x128 workload)",
               nx=n0, ny=n0, sample_of="single_box_inclusion_128x128_k3_eta1e4_Q1+3h",
               step=f"one FP64 oracle solve of the same physics on a {n0}x{n0} mesh "
                    "(assembly, set-up, FGMRES)")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(per) / len(per), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cpus": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{n0}x{n0} mesh of the headline physics per step, "
                                       f"{its} outer iterations; one spawned process, "
                                       "single-threaded BLAS"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def cpu_baseline():
    sc = oracle_scaling()
    t = sc["extrapolated_s_128x128"]
    meshes = ", ".join(f"{n}x{n}" for n in ORACLE_SIZES)
    return {"value": 1.0 / t, "unit": UNIT, "cores": sc["cores"], "host_cpus": sc["host_cpus"],
            "kind": "oracle",
            "sample": f"oracle solves of the headline physics on {meshes} meshes (3 "
                      "h-coarsenings each), one spawned process per mesh with single-threaded "
                      "BLAS; value = 1 / (the 128x128 time of the least-squares fit "
                      "of log time against log element count): an extrapolation",
            "measured": sc["samples"], "exponent": sc["exponent"],
            "extrapolated_s_128x128": t}


def _instance(ctx, wl, precision, seed):
    """A problem with its load vector and output buffers on the device."""
    import torch
    from paper_1607_03777_gb300 import api, synth
    eta, rho = ctx.rasterise_inclusions(wl.nx, wl.ny, wl.shapes)
    pr = api.Problem(ctx, wl.nx, wl.ny, wl.k, eta.cpu().numpy(), bc=wl.bc,
                     n_hlevels=wl.n_hlevels, seed=seed, precision=precision)
    f = torch.empty(pr.n_u, dtype=torch.float64, device="cuda")
    pr.rhs_body_force(rho, synth.GRAVITY, f)
    u = torch.empty_like(f)
    p = torch.empty(pr.n_p, dtype=torch.float64, device="cuda")
    return pr, f, u, p


def batch_sample(ctx, count, refine, log10_contrast=(2.0, 6.0)):
    """Batched form on the first ``count`` instances of the seeded list
    (side in {32, 64, 128, 256}, k in {2..5}, the six inclusions of Sec. 7.3
    jittered, one contrast 10^U[2,6] each), mixed precision (FP32 V-cycle,
    FP64 Krylov), sip_solve_batch with one stream per instance (their solves
    overlap on the device), set-up inside the timed region; against the plain
    FP64 form solved one at a time.  Both arms refine with a double-double residual (``refine``
    correction solves at most).  Every result's residual is the library's
    (double-double with refinement); the difference from the FP64 arm is
    reported per instance."""
    import torch
    from paper_1607_03777_gb300 import api, synth
    insts = synth.batch_instances(128, log10_contrast=log10_contrast)[:count]
    mixed = [_instance(ctx, wl, "mixed", 4) for wl in insts]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, reps = api.solve_batch(ctx, [m[0] for m in mixed], [m[1] for m in mixed],
                               [m[2] for m in mixed], [m[3] for m in mixed], n_streams=count,
                               rtol=1e-8, refine=refine)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    plain = []
    for wl in insts:
        pr, f, u, p = _instance(ctx, wl, "fp64", 4)
        rep = pr.solve(f, u, p, rtol=1e-8, refine=refine, check=False)
        plain.append((rep, u))
        del pr
    torch.cuda.synchronize()
    dt1 = time.perf_counter() - t1
    err = [float(torch.linalg.norm(m[2] - u) / torch.linalg.norm(u)) for m, (_, u) in zip(mixed, plain)]
    return {"metric": "batched_stokes_solves_per_s", "value": len(insts) / dt, "unit": UNIT,
            "fp64_one_at_a_time": len(insts) / dt1, "instances": len(insts), "status": st,
            "converged": sum(1 for r in reps if r["status"] == 0),
            "fp64_converged": sum(1 for r, _ in plain if r["status"] == 0),
            "max_rel_residual": max(r["rel_residual"] for r in reps),
            "fp64_max_rel_residual": max(r["rel_residual"] for r, _ in plain),
            "u_rel_diff_vs_fp64": {"max": max(err), "median": float(sorted(err)[len(err) // 2])},
            "config": {"workload": "batch_instances(seed 4): sides 32-256, k 2-5, jittered six "
                                   f"inclusions, contrast 1e{log10_contrast[0]:g}-"
                                   f"1e{log10_contrast[1]:g}",
                       "sample": f"first {len(insts)} of the 128 instances",
                       "precision": "mixed",
                       "form": f"sip_solve_batch, {len(insts)} concurrent streams",
                       "rtol": 1e-8, "refine": refine}}


def c3_sample(ctx, max_inner, refine, forms=("fp64", "mixed"), n=512, k=4, slack=2.0):
    """The many-disc workload (64 discs of radius 0.02 at seeded random
    centres, log10 eta ~ U[0, 6] per disc, rho 1.2; Neumann top, Navier
    elsewhere; Q^2_1 + 5 h-coarsenings) solved once per form to 1e-8 with
    refinement by a double-double residual; the inner solve capped at
    ``max_inner`` iterations (the flexible outer FGMRES absorbs the rest).
    The forms after the first get ``slack`` times the first one's time
    (sip_solve_opts.time_limit_ms): a form that has not converged by then is
    slower than FP64 and stops with SIP_ERR_TIMEOUT at its last residual.
    Reports solves/s, iteration counts, the residual (double-double) and the
    difference of each form's velocity from the FP64 one."""
    import torch
    from paper_1607_03777_gb300 import api, synth
    wl = synth.many_discs(n=n, k=k, n_hlevels=synth.levels_to_17(n))
    eta, rho = ctx.rasterise_inclusions(n, n, wl.shapes)
    eh = eta.cpu().numpy()
    out, u64, limit = {}, None, 0.0
    for form in forms:
        pr = api.Problem(ctx, n, n, k, eh, bc=wl.bc, n_hlevels=wl.n_hlevels, seed=1,
                         precision=form)
        f = torch.empty(pr.n_u, dtype=torch.float64, device="cuda")
        pr.rhs_body_force(rho, synth.GRAVITY, f)
        u = torch.empty_like(f)
        p = torch.empty(pr.n_p, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = pr.solve(f, u, p, rtol=1e-8, max_outer=2000, max_inner=max_inner, refine=refine,
                       time_limit_ms=limit, check=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if not limit:
            limit = slack * dt * 1e3
        # the residual of the returned FP64 arrays, evaluated in double-double:
        # at this contrast ||K|| eps_64 ||x|| ~ 1e-7 ||b||, so rounding the
        # refined iterate to FP64 lifts it above rtol (sip_solve_dd returns
        # the iterate itself)
        xu = torch.stack([u, torch.zeros_like(u)], 1).reshape(-1)
        xp = torch.stack([p, torch.zeros_like(p)], 1).reshape(-1)
        ru, rp = torch.empty_like(xu), torch.empty_like(xp)
        pr.residual_dd(f, xu, xp, ru, rp)
        ru, rp = ru.view(-1, 2).sum(1), rp.view(-1, 2).sum(1)
        rel_fp64 = float(torch.sqrt(torch.sum(ru * ru) + torch.sum(rp * rp)) /
                         torch.linalg.norm(f))
        del xu, xp, ru, rp
        rec = {"value": 1.0 / dt, "unit": UNIT, "s": dt, "status": rep["status"],
               "outer_its": rep["outer_its"], "inner_avg": rep["inner_avg"],
               "inner_max": rep["inner_max"], "rel_residual": rep["rel_residual"],
               "rel_residual_of_fp64_output": rel_fp64,
               "refine_steps": rep["refine_steps"], "setup_ms": rep["setup_ms"],
               "time_limit_ms": limit if form != forms[0] else 0.0,
               "schedule": pr.schedule()}
        if form == "fp64":
            u64 = u.clone()
        elif u64 is not None:
            rec["u_rel_diff_vs_fp64"] = float(torch.linalg.norm(u - u64) / torch.linalg.norm(u64))
        out[form] = rec
        del pr
    return {"metric": "stokes_solves_per_s_to_1e-8_residual", "forms": out,
            "config": {"workload": f"many_discs_{n}x{n}_k{k}: 64 discs r 0.02, log10 eta "
                                   "U[0,6], Q1+5h", "rtol": 1e-8, "refine": refine,
                       "max_inner": max_inner, "inner_rtol": 1e-3,
                       "residual": "rel_residual: of the double-double iterate (refinement); "
                                   "rel_residual_of_fp64_output: of the FP64 arrays sip_solve "
                                   "returns, evaluated in double-double"}}


def batch_small_sample(ctx, count=48, side=32):
    """Many small problems (``count`` meshes of side x side elements, k 2 or
    3, the six jittered inclusions of Sec. 7.3 at contrast 10^U[1,3]): the
    launch-bound regime.  Solved three ways, mixed precision, to 1e-8: the
    grouped engine (all inner solves in one batched graph) and concurrent
    streams with 8 and 32 solves in flight."""
    import numpy as np
    import torch
    from paper_1607_03777_gb300 import api, synth
    g = np.random.Generator(np.random.PCG64(21))
    specs = [(int(g.integers(2, 4)), synth.jittered_sinkers(int(g.integers(0, 2 ** 31)), (1.0, 3.0)))
             for _ in range(count)]
    out = {}
    for label, grouped, width in (("grouped", True, count), ("streams_8", False, 8),
                                  ("streams_32", False, 32)):
        ms = []
        for k, shapes in specs:
            eta, rho = ctx.rasterise_inclusions(side, side, shapes)
            pr = api.Problem(ctx, side, side, k, eta.cpu().numpy(), bc=synth.SINKER_BC,
                             n_hlevels=synth.levels_to_17(side), seed=4, precision="mixed")
            f = torch.empty(pr.n_u, dtype=torch.float64, device="cuda")
            pr.rhs_body_force(rho, synth.GRAVITY, f)
            pr.setup()
            ms.append((pr, f, torch.empty_like(f),
                       torch.empty(pr.n_p, dtype=torch.float64, device="cuda")))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, reps = api.solve_batch(ctx, [m[0] for m in ms], [m[1] for m in ms],
                                   [m[2] for m in ms], [m[3] for m in ms], n_streams=width,
                                   rtol=1e-8, grouped=grouped)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[label] = {"value": count / dt, "unit": UNIT, "status": st,
                      "converged": sum(1 for r in reps if r["status"] == 0),
                      "max_rel_residual": max(r["rel_residual"] for r in reps)}
        del ms
    return {"metric": "batched_stokes_solves_per_s", "forms": out,
            "config": {"workload": f"{count} meshes of {side}x{side}, k 2-3, jittered six "
                                   "inclusions, contrast 1e1-1e3 (seed 21)",
                       "precision": "mixed", "rtol": 1e-8, "set_up": "before the timed region"}}


def run_batch(args):
    import torch  # noqa: F401
    from paper_1607_03777_gb300 import api
    return batch_sample(api.Context(0), args.count, args.refine)


def serve_sample(ctx, count, refine, max_log_contrast, rate=None):
    """Served form on the first ``count`` requests of the seeded Poisson
    stream (side log-uniform in [32, 512], k in {2..6}, the six inclusions of
    Sec. 7.3 jittered, contrast 10^U[0, max_log_contrast]) replayed in real
    time into the server (mixed precision, 8 slots, HBM admission budget =
    free HBM - 10%) at the stream's 200 requests/s, or at ``rate``; latency =
    submit to result on the host.  Against the same requests solved one at a
    time in plain FP64."""
    import numpy as np
    import torch
    from paper_1607_03777_gb300 import api, synth
    arrivals, wls = synth.request_stream(log10_contrast=(0.0, max_log_contrast))
    arrivals, wls = arrivals[:count], wls[:count]
    if rate:
        arrivals = arrivals * (200.0 / rate)
    free, _ = torch.cuda.mem_get_info()
    srv = api.Server(ctx, budget_bytes=int(free * 0.9), max_slots=8)
    eta_rho = []
    for wl in wls:   # element materials on the device, copied to the host once
        eta, rho = ctx.rasterise_inclusions(wl.nx, wl.ny, wl.shapes)
        eta_rho.append((eta.cpu().numpy(), rho.cpu().numpy()))
    keep = []
    t0 = time.perf_counter()
    for i, (ta, wl) in enumerate(zip(arrivals, wls)):
        wait = t0 + ta - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        eta, rho = eta_rho[i]
        keep.append(srv.submit(i, wl.nx, wl.ny, wl.k, eta, rho, g=synth.GRAVITY, bc=wl.bc,
                               n_hlevels=wl.n_hlevels, seed=5, precision="mixed",
                               opts={"rtol": 1e-8, "refine": refine}))
    srv.drain()
    dt = time.perf_counter() - t0
    done = srv.poll(cap=max(256, len(wls)))
    srv.close()
    lat = np.array([r["solve_ms"] for _, r in done])
    ok = sum(1 for _, r in done if r["status"] == 0)
    t1 = time.perf_counter()
    base_lat, base_ok, base_u = [], 0, []
    for wl in wls:
        ts = time.perf_counter()
        pr, f, u, p = _instance(ctx, wl, "fp64", 5)
        rep = pr.solve(f, u, p, rtol=1e-8, refine=refine, check=False)
        torch.cuda.synchronize()
        base_lat.append((time.perf_counter() - ts) * 1e3)
        base_ok += rep["status"] == 0
        base_u.append(u)
        del pr
    dt1 = time.perf_counter() - t1
    err = []
    for (st_i, u_srv, _), u64 in zip(keep, base_u):
        ref = u64.cpu().numpy()
        err.append(float(np.linalg.norm(u_srv - ref) / np.linalg.norm(ref)))
    return {"metric": "served_stokes_solves_per_s", "value": len(done) / dt, "unit": UNIT,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "offered_rate_per_s": rate or 200.0,
            "requests": len(done), "converged": ok,
            "u_rel_diff_vs_fp64": {"max": max(err), "median": float(np.median(err))},
            "fp64_one_at_a_time": {"value": len(wls) / dt1, "unit": UNIT,
                                   "solve_ms_p50": float(np.percentile(base_lat, 50)),
                                   "solve_ms_p99": float(np.percentile(base_lat, 99)),
                                   "converged": int(base_ok)},
            "config": {"workload": "request_stream(seed 5): sides 32-512, k 2-6, jittered six "
                                   f"inclusions, contrast 1-1e{max_log_contrast:g}",
                       "sample": f"first {len(wls)} requests", "slots": 8, "precision": "mixed",
                       "rtol": 1e-8, "refine": refine}}


def run_serve(args):
    from paper_1607_03777_gb300 import api
    return serve_sample(api.Context(0), args.count, args.serve_refine,
                        args.serve_max_log_contrast)


def run_coarse(args):
    """Coarse-space comparison (Sec. 7.1 table of the four preconditioners):
    A_p(Q^2_0), A_hp(Q^2_0), A_p(Q^2_1), A_hp(Q^2_1) on the box-inclusion
    problem (eta 1e4) with k = 2, FP64, rtol 1e-8; element-wise constant
    spaces on odd meshes (n + 1 elements per side) as the paper does, direct
    coarse solves only where the coarse problem has at most 8192 elements.
    Each solve includes its multigrid set-up; best of three."""
    import torch
    from paper_1607_03777_gb300 import api, synth
    ctx = api.Context(0)
    k = 2
    rows = []
    for n in (64, 128, 256):
        for coarse, hp in (("q0", False), ("q0", True), ("q1", False), ("q1", True)):
            m = n + 1 if coarse == "q0" else n
            if not hp and m * m > 8192:
                continue
            nh = synth.levels_to_17(m - 1 if coarse == "q0" else m) if hp else 0
            wl = synth.single_box_inclusion(n=m, k=k)
            eta, rho = ctx.rasterise_inclusions(m, m, wl.shapes)
            pr = api.Problem(ctx, m, m, k, eta.cpu().numpy(), bc=wl.bc, n_hlevels=nh, seed=1,
                             coarse=coarse)
            f = torch.empty(pr.n_u, dtype=torch.float64, device="cuda")
            u = torch.empty_like(f)
            p = torch.empty(pr.n_p, dtype=torch.float64, device="cuda")
            pr.rhs_body_force(rho, synth.GRAVITY, f)
            best, rep = 1e30, None
            for _ in range(3):
                pr.update_eta(eta)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = pr.solve(f, u, p, rtol=1e-8, max_outer=1000, check=False)
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            name = ("A_hp" if hp else "A_p") + ("(Q2_0)" if coarse == "q0" else "(Q2_1)")
            rows.append({"preconditioner": name, "elements": f"{m}x{m}", "n_hlevels": nh,
                         "status": rep["status"], "outer_its": rep["outer_its"],
                         "inner_avg": round(rep["inner_avg"], 2), "inner_max": rep["inner_max"],
                         "rel_residual": rep["rel_residual"], "ms": round(best * 1e3, 2),
                         "solves_per_s": round(1.0 / best, 3)})
            del pr
    return {"metric": "coarse_space_comparison", "unit": UNIT, "rows": rows,
            "config": {"workload": "single_box_inclusion eta 1e4, k = 2, FP64, rtol 1e-8",
                       "precision": "fp64"}}


def run_sinkers(args):
    """The six sedimenting inclusions of Sec. 7.3 (positions and radii as
    listed there, rho 1.2 against 1, Neumann top, Navier elsewhere),
    A_hp(Q^2_1) with 2, 3, 4 h-coarsenings at 64^2, 128^2, 256^2, k = 1..3,
    contrasts 1e3, 1e6, 1e8, FP64, outer rtol 1e-6 and inner rtol 1e-3 as in
    the paper.  The paper ran GCR for both solves, the defaults here; the
    outer method can be FGMRES instead and the inner one PCG with either
    stopping test."""
    import torch
    from paper_1607_03777_gb300 import api, synth
    ctx = api.Context(0)
    inner = {"gcr": dict(inner_krylov="gcr", inner_norm="true"),
             "pcg-true": dict(inner_krylov="pcg", inner_norm="true"),
             "pcg-preconditioned": dict(inner_krylov="pcg", inner_norm="preconditioned")}
    ikw = dict(inner[args.sinker_inner], outer_krylov=args.sinker_outer,
               refine=args.sinker_refine)
    rows = []
    for eta_in in [e for e in (1e3, 1e6, 1e8, 1e10)
                   if args.sinker_min_eta <= e <= args.sinker_max_eta]:
        for n in (64, 128, 256):
            for k in (1, 2, 3):
                wl = synth.six_sinkers(n=n, k=k, eta_in=eta_in, n_hlevels=synth.levels_to_17(n))
                eta, rho = ctx.rasterise_inclusions(n, n, wl.shapes)
                pr = api.Problem(ctx, n, n, k, eta.cpu().numpy(), bc=wl.bc,
                                 n_hlevels=wl.n_hlevels, seed=1)
                f = torch.empty(pr.n_u, dtype=torch.float64, device="cuda")
                u = torch.empty_like(f)
                p = torch.empty(pr.n_p, dtype=torch.float64, device="cuda")
                pr.rhs_body_force(rho, synth.GRAVITY, f)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = pr.solve(f, u, p, rtol=1e-6, max_outer=500, check=False, **ikw)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                rows.append({"eta": eta_in, "elements": f"{n}x{n}", "k": k, "status": rep["status"],
                             "outer_its": rep["outer_its"], "inner_avg": round(rep["inner_avg"], 1),
                             "inner_max": rep["inner_max"], "rel_residual": rep["rel_residual"],
                             "refine_steps": rep["refine_steps"], "ms": round(dt * 1e3, 1)})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)   # progress
                del pr
    return {"metric": "six_sinkers_iterations", "unit": "iterations", "rows": rows,
            "config": {"workload": "six sinkers (Sec. 7.3), A_hp(Q2_1), FP64, rtol 1e-6",
                       "precision": "fp64", "outer": args.sinker_outer,
                       "inner": args.sinker_inner, "refine": args.sinker_refine}}


def run_checkerboard(args):
    """The 2 x 2 viscosity checkerboard of Sec. 7.2 (jumps at x = 1/2 and
    y = 1/2, contrasts 1e3, 1e6, 1e8, Navier on every side) with our own
    forcing (a dense disc in a unit-viscosity quadrant; the SolCx forcing is
    only cited), A_hp(Q^2_1) with 3 / 4 / 5 h-coarsenings at 64^2, 128^2,
    256^2 as for SolCx, k = 1..3, FP64, FGMRES to 1e-6 with the inner solve
    to 1e-3 (Sec. 7.1 settings).  Caps: 200 outer, 100 inner iterations."""
    import torch
    from paper_1607_03777_gb300 import api, synth
    ctx = api.Context(0)
    inner = {"gcr": dict(inner_krylov="gcr", inner_norm="true"),
             "pcg-true": dict(inner_krylov="pcg", inner_norm="true"),
             "pcg-preconditioned": dict(inner_krylov="pcg", inner_norm="preconditioned")}
    ikw = inner[args.checker_inner]
    rows = []
    for eta_hi in (1e3, 1e6, 1e8):
        for n in (64, 128, 256):
            for k in (1, 2, 3):
                wl = synth.checkerboard(n=n, k=k, eta_hi=eta_hi,
                                        n_hlevels=synth.levels_to_17(n) + 1)
                eta, rho = ctx.rasterise_inclusions(n, n, wl.shapes)
                pr = api.Problem(ctx, n, n, k, eta.cpu().numpy(), bc=wl.bc,
                                 n_hlevels=wl.n_hlevels, seed=1)
                f = torch.empty(pr.n_u, dtype=torch.float64, device="cuda")
                u = torch.empty_like(f)
                p = torch.empty(pr.n_p, dtype=torch.float64, device="cuda")
                pr.rhs_body_force(rho, synth.GRAVITY, f)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rep = pr.solve(f, u, p, rtol=wl.rtol, max_outer=200, max_inner=100, check=False,
                               **ikw)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                rows.append({"eta": eta_hi, "elements": f"{n}x{n}", "k": k, "status": rep["status"],
                             "outer_its": rep["outer_its"], "inner_avg": round(rep["inner_avg"], 1),
                             "inner_max": rep["inner_max"], "rel_residual": rep["rel_residual"],
                             "ms": round(dt * 1e3, 1)})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)   # progress
                del pr
    return {"metric": "checkerboard_iterations", "unit": "iterations", "rows": rows,
            "config": {"workload": "2x2 viscosity checkerboard (Sec. 7.2) with a dense disc, "
                                   "A_hp(Q2_1), FP64, rtol 1e-6",
                       "precision": "fp64", "outer": "fgmres", "inner": args.checker_inner}}


def apply_codes(args):
    """--apply-code 'a[,b]' as the [FP64, FP32] pair set_schedule takes."""
    if not args.apply_code:
        return None
    c = [int(v) for v in args.apply_code.split(",")]
    return [c[0], c[-1]]


def run_kernel(args):
    """A few launches of one operator on a small case (--profile-n, --profile-k),
    timed with CUDA events: the command behind the ncu captures of single
    kernels. apply_f64 / apply_f32: y = A x (Eq. 6 form) on a random viscosity
    field log-uniform over three decades; vcycle_f32: one FP32 V-cycle of the
    many-discs field (the high-contrast workload, split-precision parts
    included) with the fused smoother step off, so the block-Jacobi kernel
    launches on its own."""
    import torch
    from paper_1607_03777_gb300 import api, synth
    ctx = api.Context(0)
    n, k = args.profile_n, args.profile_k
    if args.kernel == "vcycle_f32":
        wl = synth.many_discs(n=n, k=k, n_hlevels=synth.levels_to_17(n))
        eta, _ = ctx.rasterise_inclusions(n, n, wl.shapes)
        pr = api.Problem(ctx, n, n, k, eta.cpu().numpy(), bc=wl.bc, n_hlevels=wl.n_hlevels,
                         seed=1, precision="mixed")
        pr.set_schedule(fused=[0, 0])
        pr.setup()
        x = torch.randn(pr.n_u, dtype=torch.float32, device="cuda")
        fn = pr.vcycle_f32
    else:
        dt = torch.float32 if args.kernel == "apply_f32" else torch.float64
        pr = api.Problem(ctx, n, n, k, synth.random_eta(n * n, 1, (0.0, 3.0)))
        x = torch.randn(pr.n_u, dtype=dt, device="cuda")
        fn = pr.apply_A_f32 if dt == torch.float32 else pr.apply_A
    if apply_codes(args):
        pr.set_schedule(apply=apply_codes(args))
    y = torch.empty_like(x)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(max(args.warmup, 1)):
        fn(x, y)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()   # ncu --profile-from-start off captures from here
    ev[0].record()
    for _ in range(args.steps):
        fn(x, y)
    ev[1].record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    return {"mode": "kernel", "kernel": args.kernel, "n": n, "k": k,
            "schedule": pr.schedule(), "ms_per_call": ev[0].elapsed_time(ev[1]) / args.steps,
            "finite": bool(torch.isfinite(y).all().item())}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.mode != "solve":
        if rank == 0:
            out = {"batch": run_batch, "serve": run_serve, "coarse": run_coarse,
                   "sinkers": run_sinkers, "checkerboard": run_checkerboard,
                   "kernel": run_kernel}[args.mode](args)
            print(json.dumps(out), flush=True)
        return 0
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    out = run_ours(args, local, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
