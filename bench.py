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
    ap.add_argument("--steps", type=int, default=5)
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
                    choices=["solve", "batch", "serve", "coarse", "sinkers", "checkerboard"],
                    help="solve: the headline line; batch / serve: the batched and served "
                         "forms on bounded samples of their workloads; coarse: the four "
                         "coarse-space preconditioners; sinkers / checkerboard: the "
                         "six-sinker and checkerboard iteration sweeps (extra lines)")
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

    def timed(precision, steps, warmup, clocks=None, inner_norm=head_norm):
        prob, f, u, p = make(precision)
        for _ in range(warmup):
            step(prob, f, u, p, inner_norm)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        times, reps = [], []
        if clocks:
            clocks.start()
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
        return prob, f, u, p, times, reps, clocks_out

    clocks = ClockSampler(dev.index)
    if args.profile_only:   # one form only, for profiler launch lists
        _, _, _, _, tp, rp, _ = timed(args.profile_precision, args.steps, args.warmup)
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
        "schedule": {"fp64": prob64.schedule(), "mixed": sched_mixed},
        "clocks": clk,
        "sip_apply": {"kernel": DOMINANT, "ms": apply_ms,
                      "GB_per_s": ab / apply_ms / 1e6, "GFLOP_per_s": af / apply_ms / 1e6,
                      "dof_per_s": prob64.n_u / (apply_ms / 1e3)},
    }
    out["roofline"] = roofline(out, ab, af, apply_ms)
    return out


# FP64 peak of one GB300, derived from unit counts and clocks: 152 SMs x
# 2 FP64 FMA per SM per clock x 2 FLOP x 2.07 GHz (maximum SM clock)
# = 1.259 TFLOP/s (NVIDIA's figure: 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# the kernel sip_apply_A launches for k = 3 in FP64 (component split,
# 16-byte vector accesses; SIP_APPLY_KERNEL=elem1 / tile select the others)
DOMINANT = {"elem1": "k_apply_elem<4,double>", "tile": "k_apply_sip<4,double>"}.get(
    os.environ.get("SIP_APPLY_KERNEL", ""), "k_apply_elem2<4,double,true>")
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_apply_elem2_fp64_128x128_k3.md")


def captured_traffic():
    """DRAM bytes per launch of the dominant kernel from its committed ncu
    summary (dram__bytes_read.sum + dram__bytes_write.sum), or None."""
    if not os.path.exists(TRAFFIC_PROFILE):
        return None
    vals = {}
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    for line in open(TRAFFIC_PROFILE):
        for key in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            if f"`{key}`" in line:
                cells = [c.strip() for c in line.strip().strip("|").split("|")]
                vals[key] = float(cells[1]) * scale.get(cells[2], 1.0)
    if len(vals) != 2:
        return None
    return vals["dram__bytes_read.sum"] + vals["dram__bytes_write.sum"]


def roofline(out, ab, af, apply_ms):
    """FP64 on GB300 is bound by the FP64 pipe, not HBM: achieved FP64
    FLOP/s of the SIP apply (algorithmic FLOPs / live launch time) against the
    FP64 peak derived from unit counts and clocks."""
    achieved = af / apply_ms / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": captured_traffic(),
            "kernel": DOMINANT, "algorithmic_bytes": ab, "algorithmic_flops": af,
            "hbm_GB_per_s": ab / apply_ms / 1e6,
            "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz"}


# ------------------------------------------------------------------ oracle
def oracle_sample(seconds_hint=20.0):
    """Time the FP64 oracle on a bounded sample of the workload: the same
    physics (box inclusion 1e4, k = 3, Q^2_1 + h-levels, rtol 1e-8) on a
    16 x 16 mesh, scaled by the element count (128^2 / 16^2 = 64) to an
    estimate for the full workload (the solver is O(n) per iteration)."""
    import numpy as np
    from oracle import krylov, materials, multigrid, sip
    from paper_1607_03777_gb300 import synth
    n = 16
    wl = synth.single_box_inclusion(n=n, n_hlevels=0)
    eta, rho = materials.rasterise_inclusions(n, n, wl.shapes)
    t0 = time.perf_counter()
    pr = sip.Problem(n, n, wl.k, eta, bc=wl.bc)
    A, B = sip.assemble_A(pr), sip.assemble_B(pr)
    f = sip.rhs_body_force(pr, rho)
    mg = multigrid.HPMultigrid(pr, A, 1, seed=1)
    Pc = krylov.BlockPreconditioner(A, B, sip.schur_mass(pr), mg, 1e-3)   # residual inner test
    K = krylov.stokes_matrix(A, B)
    b = np.concatenate([f, np.zeros(B.shape[1])])
    x, its, _ = krylov.fgmres(lambda v: K @ v, Pc, b, 1e-8, maxit=1000)
    dt = time.perf_counter() - t0
    scale = (128 * 128) / (n * n)
    return dt, scale, its


def run_reference(args):
    per = []
    for i in range(args.warmup + args.steps):
        dt, scale, its = oracle_sample()
        if i >= args.warmup:
            per.append(dt * scale)
    value = len(per) / sum(per)
    cores = 1
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(per) / len(per), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": dict(headline_config(args),
                           step="oracle solve of a 16x16 mesh of the same physics, time x 64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "16x16 mesh of the same physics per step, time x 64 "
                                       "(element-count ratio)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def cpu_baseline():
    dt, scale, its = oracle_sample()
    return {"value": 1.0 / (dt * scale), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one oracle solve of the same physics on a 16x16 mesh ({dt:.1f} s, "
                      f"{its} outer its), time x {scale:.0f} (element-count ratio); "
                      "SciPy sparse kernels, single-threaded"}


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


def run_batch(args):
    """Batched form: the first ``--count`` instances of the seeded list
    (side in {32, 64, 128, 256}, k in {2..5}, the six inclusions of Sec. 7.3
    jittered, contrast 10^U[2,6]), mixed precision (FP32 V-cycle, FP64
    Krylov), solved concurrently on 8 streams; against the plain FP64 form
    solved one at a time.  Both arms refine with a double-double residual
    (``--refine``).  Set-up is inside both timed regions."""
    import torch
    from paper_1607_03777_gb300 import api, synth
    ctx = api.Context(0)
    insts = synth.batch_instances(128)[:args.count]
    mixed = [_instance(ctx, wl, "mixed", 4) for wl in insts]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for pr, _, _, _ in mixed:
        pr.setup()
    st, reps = api.solve_batch(ctx, [m[0] for m in mixed], [m[1] for m in mixed],
                               [m[2] for m in mixed], [m[3] for m in mixed], n_streams=8,
                               rtol=1e-8, refine=args.refine)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    plain = []
    for wl in insts:
        pr, f, u, p = _instance(ctx, wl, "fp64", 4)
        rep = pr.solve(f, u, p, rtol=1e-8, refine=args.refine, check=False)
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
            "u_rel_diff_vs_fp64": {"max": max(err), "median": float(sorted(err)[len(err) // 2])},
            "config": {"workload": "batch_instances(seed 4): sides 32-256, k 2-5, "
                                   "jittered six inclusions, contrast 1e2-1e6",
                       "count": len(insts), "precision": "mixed", "streams": 8, "rtol": 1e-8,
                       "refine": args.refine}}


def run_serve(args):
    """Served form: the first ``--count`` requests of the seeded Poisson
    stream (200 requests/s, side log-uniform in [32, 512], k in {2..6}, the
    six inclusions of Sec. 7.3 jittered, contrast 10^U[0,5] by default) replayed in real
    time into the server (mixed precision, 8 slots, HBM admission budget =
    free HBM - 10%); latency = submit to result on the host.  Against the
    same requests solved one at a time in plain FP64.  ``--serve-refine``
    turns on refinement with a double-double residual in both arms."""
    import numpy as np
    import torch
    from paper_1607_03777_gb300 import api, synth
    ctx = api.Context(0)
    arrivals, wls = synth.request_stream(log10_contrast=(0.0, args.serve_max_log_contrast))
    arrivals, wls = arrivals[:args.count], wls[:args.count]
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
                               opts={"rtol": 1e-8, "refine": args.serve_refine}))
    srv.drain()
    dt = time.perf_counter() - t0
    done = srv.poll(cap=max(256, len(wls)))
    srv.close()
    lat = np.array([r["solve_ms"] for _, r in done])
    ok = sum(1 for _, r in done if r["status"] == 0)
    # baseline: the same requests, one at a time, plain FP64, arrival times ignored
    t1 = time.perf_counter()
    base_lat, base_ok, base_u = [], 0, []
    for wl in wls:
        ts = time.perf_counter()
        pr, f, u, p = _instance(ctx, wl, "fp64", 5)
        rep = pr.solve(f, u, p, rtol=1e-8, refine=args.serve_refine, check=False)
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
            "requests": len(done), "converged": ok,
            "u_rel_diff_vs_fp64": {"max": max(err), "median": float(np.median(err))},
            "fp64_one_at_a_time": {"value": len(wls) / dt1, "unit": UNIT,
                                   "solve_ms_p50": float(np.percentile(base_lat, 50)),
                                   "solve_ms_p99": float(np.percentile(base_lat, 99)),
                                   "converged": int(base_ok)},
            "config": {"workload": "request_stream(seed 5): 200 req/s, sides 32-512, k 2-6, "
                                   "jittered six inclusions, contrast "
                                   f"1-1e{args.serve_max_log_contrast:g}",
                       "count": len(wls), "slots": 8, "precision": "mixed", "rtol": 1e-8,
                       "refine": args.serve_refine}}


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


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.mode != "solve":
        if rank == 0:
            out = {"batch": run_batch, "serve": run_serve, "coarse": run_coarse,
                   "sinkers": run_sinkers, "checkerboard": run_checkerboard}[args.mode](args)
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
