#!/usr/bin/env python
"""ManiDSDP on one GB300: solve time to KKT residual <= 1e-8.

Workload: the order-2 moment relaxation of a dense binary quadratic program
min x'Qx + c'x over x in {-1,1}^80 (Section 6.1): moment matrix 3241 x 3241,
1,666,981 classes (monomials of degree <= 4), Q and c iid N(0,1) from seed 0,
p_0 = ceil(ln m) = 15 (Section 6.1 sets p_0 = ceil(log m)).

A step is one pass of the whole hot path: one ALM outer iteration of Algorithm 1
(the RTR solve of the subproblem with its tCG Hessian-vector products, the
multiplier update, the Lanczos certificate check, the rank and sigma updates), in
the mixed-precision form (FP32 Hessian-vector products, df64 cost and gradient,
FP64 multiplier, KKT residuals and Lanczos).  The W warm-up steps are the first W
outer iterations of a fresh solve from the seeded start; the K timed steps are
the next K outer iterations of the same solve (warm start: factor, multiplier
and penalty carried over).  Inputs sit in HBM before the timed region; the
working set (index map 42 MB, N x N FP64 multiplier and G 168 MB) exceeds the
129 MB L2, so no flush is needed between steps.  Beside the headline the line
reports a full solve to eta_max <= 1e-8 of the q = 60 instance (N = 1831) and
the same q = 40 instance solved by the mixed and by the plain FP64 form.

Under torchrun (N > 1) each rank runs its own replica (the single-instance path
has no exchange step); value = max-over-ranks time / (K x ranks), the job's time
per outer iteration.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (its Hessian-vector product, cost-plus-gradient
evaluation and certificate matvec) and scales it to one outer iteration by the
operation counts of an outer iteration (see the JSON's cpu_baseline.sample).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "solve time to KKT≤1e-8 (mixed vs FP64 GPU); Hess-vec GB/s or TC % of roofline"
UNIT = "s/ALM-outer-iteration"

# Operation counts of one outer iteration of this workload (means over the timed
# steps of a GPU run), used to scale the sampled oracle timings to one outer
# iteration when no GPU run precedes them.  The GPU arm uses the counts of its
# own timed steps.
DEFAULT_COUNTS = dict(hessvecs=6622, evals=164, grads=170, lanczos_matvecs=115, p=49)

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum over the kernels of one
# Hess-vec) from one ncu capture at q = 80 and the p of the timed steps, per gather-GEMM
# engine of the mixed form.  "current" is False when kernels of the Hess-vec changed
# after the capture; the line then reports traffic null and the capture as context.
HV_TRAFFIC = {
    "fma": {"p": 51, "bytes": 191.1e6, "current": False,
            "note": "captured before the FP32 Gram moved to 32-row splits on a side stream"},
    "tc": {"p": 51, "bytes": 183.4e6, "current": False,
           "note": "captured before the tensor-core kernel rounded both TF32 halves and issued "
                   "four products per step (same loads)"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--q", type=int, default=80)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--engine", choices=["fma", "tc"], default="tc",
                    help="gather GEMM of the FP32 Hessian-vector product: FP32 FMA kernel or "
                         "tensor cores (tcgen05 kind::tf32, two-term TF32 operand split)")
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--hv-reps", type=int, default=30)
    ap.add_argument("--solve-q", type=int, default=60,
                    help="instance size of the full solve reported beside the headline (0 skips)")
    ap.add_argument("--compare-q", type=int, default=40,
                    help="instance size for the mixed-vs-FP64 solve comparison (0 skips it)")
    ap.add_argument("--tcg-host", action="store_true",
                    help="launch the tCG kernels from the host instead of the device-driven graph "
                         "(same kernels; for profilers that list kernels one launch at a time)")
    ap.add_argument("--hv-only", type=int, default=0,
                    help="only time the Hessian-vector product at this p (profiling)")
    ap.add_argument("--hv-stages", action="store_true",
                    help="with --hv-only: per-stage CUDA events (params.profile = 2, which "
                         "serialises the side stream) and the mean time of each stage")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


def bench_config(args, world):
    """The workload description shared by both arms."""
    q = args.q
    N = 1 + q + q * (q - 1) // 2
    m = sum(math.comb(q, d) for d in range(5))
    return {"workload": f"dense BQP order-2 moment relaxation, q={q}, seed={args.seed}",
            "N": N, "m": m, "p0": int(math.ceil(math.log(m))), "precision": args.precision,
            "hessvec_gemm": ("tensor cores (tcgen05 kind::tf32, operands split into two TF32 "
                             "halves)" if args.engine == "tc" else "FP32 FMA"),
            "step": "one ALM outer iteration of Algorithm 1, continuing one solve",
            "l2": "working set > L2 (idx 42 MB + N x N FP64 multiplier and G, 84 MB each), no flush",
            "parallelism": f"replicas{world}"}


def reduce_over_ranks(ms, steps_done, world, device):
    """Replicas: the job's timed-region length is the slowest rank's, and its
    work is the sum of the outer iterations all ranks completed."""
    if world <= 1:
        return ms, steps_done
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([steps_done], device=device, dtype=torch.float64)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(n.item()))


def job_value(ms_max, total_steps):
    """Seconds per outer iteration of the whole job."""
    return ms_max / 1e3 / max(1, total_steps)


def workload(q, seed):
    import paper_2512_04406_gb300 as mds
    from synthetic import bqp_instance
    Q, c = bqp_instance(q, seed)
    N, m, idx = mds.manidsdp_bqp_index_map(q, 2)
    b = mds.manidsdp_bqp_rhs(q, Q, c, 2)
    p0 = int(math.ceil(math.log(m)))
    return Q, c, N, m, idx, b, p0


def hessvec_bytes(N, m, n_entries, n_pieces, p, fp_bytes):
    """Algorithmic DRAM bytes of one Hessian-vector product (Proposition 4.2) in
    the tiled form: the class-sum pass reads the slot map (4 B per upper-triangle
    entry), writes and re-reads the class-ordered buffer (2 x fp_bytes per upper
    entry), reads the piece table (8 B per piece) and writes w (fp_bytes per
    class); the gather GEMM reads G (fp_bytes per entry) and the index map (4 B
    per entry); Y, U are read and HU written once (8 B each, FP64 I/O)."""
    return ((4 + 2 * fp_bytes) * n_entries + 8 * n_pieces + fp_bytes * m
            + (fp_bytes + 4) * N * N + 3 * 8 * N * p)


def measure_hessvec(mds, torch, ctx, N, p, reps, precision, seed=11):
    """Mean device time of one Hessian-vector product at a random unit-row Y
    (CUDA events on the library's stream, params.profile path)."""
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((N, p)); Y /= np.linalg.norm(Y, axis=1)[:, None]
    U = rng.standard_normal((N, p))
    Yd = torch.tensor(Y, device="cuda"); Ud = torch.tensor(U, device="cuda")
    HU = torch.empty_like(Yd)
    mds.manidsdp_set_state(ctx, None, 1.0)
    mds.manidsdp_subproblem_eval(ctx, Yd, p)
    for _ in range(3):
        mds.manidsdp_hessvec(ctx, Yd, Ud, p, HU, precision)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        mds.manidsdp_hessvec(ctx, Yd, Ud, p, HU, precision)
        e1.record(s)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def cpu_baseline(q, seed, counts, budget_s):
    """The FP64 oracle, as it stands, on this host: time its Hessian-vector
    product, cost-plus-gradient evaluation and certificate matvec at the
    workload's size, then scale by the operation counts of one outer iteration."""
    from oracle import manidsdp as om, moment, operators as ops, subproblem as sp
    from synthetic import bqp_instance, gaussian_factor
    t_setup = time.perf_counter()
    Q, c = bqp_instance(q, seed)
    idx = moment.index_map(q)
    m = moment.num_monomials(q)
    prob = om.make_problem(idx, moment.multiplicities(idx, m), moment.rhs(q, Q, c))
    t_setup = time.perf_counter() - t_setup
    N = idx.shape[0]
    p = max(2, int(round(counts["p"])))
    Y = gaussian_factor(N, p, seed)
    Y /= np.linalg.norm(Y, axis=1)[:, None]
    Xt = np.zeros((N, N))
    U = sp.proj_tangent(Y, np.random.default_rng(1).standard_normal((N, p)))
    deadline = time.perf_counter() + budget_s
    t_hv, t_ev, t_mv = [], [], []
    G = sp.egrad_S(Y, prob, Xt, 1.0)
    X = Xt + prob["D"] - np.diag(sp.rowdot(G @ Y, Y))
    v = np.ones(N) / math.sqrt(N)
    while time.perf_counter() < deadline or not t_hv:
        t0 = time.perf_counter(); sp.rhess(Y, U, prob, Xt, 1.0, G); t_hv.append(time.perf_counter() - t0)
        t0 = time.perf_counter(); sp.cost(Y, prob, Xt, 1.0); sp.rgrad(Y, prob, Xt, 1.0)
        t_ev.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        for _ in range(10):
            v = X @ v; v /= np.linalg.norm(v)
        t_mv.append((time.perf_counter() - t0) / 10)
    hv, ev, mv = statistics.median(t_hv), statistics.median(t_ev), statistics.median(t_mv)
    proj = hv * counts["hessvecs"] + ev * counts["evals"] + mv * counts["lanczos_matvecs"]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {
        "value": proj, "unit": UNIT, "cores": cores, "kind": "oracle",
        "sample": (f"oracle FP64 at q={q} (N={N}, m={m}, p={p}): {len(t_hv)} Hessian-vector products "
                   f"({hv:.3f} s each), {len(t_ev)} cost+gradient evaluations ({ev:.3f} s), "
                   f"{10 * len(t_mv)} certificate matvecs ({mv * 1e3:.1f} ms); value projects one "
                   f"outer iteration from its counts (hessvecs={counts['hessvecs']:.0f}, "
                   f"evals={counts['evals']:.0f}, lanczos matvecs={counts['lanczos_matvecs']:.0f}); "
                   f"index-map setup {t_setup:.1f} s not included"),
    }


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps = []
    cb = None
    budget = max(2.0, min(args.cpu_sample_s, 60.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(args.q, args.seed, DEFAULT_COUNTS, budget)
        if i >= args.warmup:
            steps.append(cb["value"])
    value = statistics.mean(steps)
    cb["value"] = value
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded N(0,1) Q, c)",
        "config": bench_config(args, world),
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    import paper_2512_04406_gb300 as mds
    from synthetic import gaussian_factor

    rank, world, local = dist_env()
    assert torch.cuda.is_available(), "bench.py needs a CUDA GPU"
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = mds.PREC_MIXED if args.precision == "mixed" else mds.PREC_FP64
    Q, c, N, m, idx, b, p0 = workload(args.q, args.seed)
    prm = mds.manidsdp_default_params()
    prm.precision_mode = prec
    prm.p_max = 256
    prm.profile = 2 if (args.hv_only and args.hv_stages) else 1
    prm.tensor_cores = 1 if args.engine == "tc" else 0
    if args.tcg_host:
        prm.tcg_device = 0
    stream = torch.cuda.current_stream()
    ctx = mds.manidsdp_setup(N, m, idx, b, params=prm, stream=stream.cuda_stream)
    if args.hv_only:
        p = args.hv_only
        mds.manidsdp_hessvec_stage_ms(ctx, True)
        ms = measure_hessvec(mds, torch, ctx, N, p, args.hv_reps, prec)
        stages = mds.manidsdp_hessvec_stage_ms(ctx, True)
        calls = args.hv_reps + 3  # measure_hessvec's warm-up calls are staged too
        fp_bytes = 4 if prec == mds.PREC_MIXED else 8
        byt = hessvec_bytes(N, m, N * (N + 1) // 2, m, p, fp_bytes)
        out = {"hv_only": True, "q": args.q, "N": N, "p": p, "precision": args.precision,
               "engine": args.engine,
               "ms": ms, "gbs": byt / (ms * 1e-3) / 1e9,
               "tflops": 6.0 * N * N * p / (ms * 1e-3) / 1e12}
        if args.hv_stages:
            out["stages_us"] = {k: round(v / calls * 1e3, 1) for k, v in stages.items()}
        print(json.dumps(out), flush=True)
        mds.manidsdp_destroy(ctx)
        return
    Y0 = torch.tensor(gaussian_factor(N, p0, args.seed + rank), device="cuda")
    # warm-up: the first W outer iterations of a fresh solve
    prm.max_outer = args.warmup
    prm.warm_start = 0
    mds.manidsdp_set_params(ctx, prm)
    rep_w, _ = mds.manidsdp_solve(ctx, Y0, p0)
    prm.max_outer = args.steps
    prm.warm_start = 1
    mds.manidsdp_set_params(ctx, prm)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = mds.manidsdp_launch_count()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler restrict itself to the timed steps
    rep, p_fin = mds.manidsdp_solve(ctx, Y0, p0)
    torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = mds.manidsdp_launch_count() - l0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    steps_done = max(1, rep.outer)
    ms, total_steps = reduce_over_ranks(ms, steps_done, world, "cuda")
    value = job_value(ms, total_steps)

    # dominant kernel: the Hessian-vector product, live (phase events inside the
    # timed solves) and in isolation at p = p_0
    hv_ms_live = rep.ms_hessvec / max(1, rep.hessvecs)
    p_avg = rep.hessvec_p_sum / max(1, rep.hessvecs)
    fp_bytes = 4 if prec == mds.PREC_MIXED else 8
    n_entries = N * (N + 1) // 2
    n_pieces = m + 2 * (args.q - 1) * 2 + (N + 31) // 32  # classes + extra pieces of long classes
    bytes_live = hessvec_bytes(N, m, n_entries, n_pieces, p_avg, fp_bytes)
    flops_live = 6.0 * N * N * p_avg
    hv_ms_iso = measure_hessvec(mds, torch, ctx, N, p0, args.hv_reps, prec)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    if prec == mds.PREC_MIXED:
        tr = HV_TRAFFIC.get(args.engine)
        roof = {"bound": "hbm", "achieved": bytes_live / (hv_ms_live * 1e-3) / 1e9, "peak": hbm_peak,
                "unit": "GB/s", "traffic": tr["bytes"] if tr and tr["current"] else None,
                "traffic_last_capture": tr, "peak_source": peak_src,
                "kernel": "Hessian-vector product (FP32 class means + gather GEMM + epilogue)",
                "avg_ms": hv_ms_live, "p_avg": p_avg,
                "isolated_ms_at_p0": hv_ms_iso,
                "isolated_gbs_at_p0": hessvec_bytes(N, m, n_entries, n_pieces, p0, 4) / (hv_ms_iso * 1e-3) / 1e9,
                "alu_tflops": flops_live / (hv_ms_live * 1e-3) / 1e12}
    else:
        fp64_peak = 1.19  # TFLOP/s: 152 SMs x 2 DFMA/clk x 2 flop x ~1.95 GHz, probe-measured
        roof = {"bound": "alu", "achieved": flops_live / (hv_ms_live * 1e-3) / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "traffic": None, "peak_source": "FP64 FMA probe on GB300",
                "kernel": "Hessian-vector product (FP64)", "avg_ms": hv_ms_live, "p_avg": p_avg}
    roof["frac"] = roof["achieved"] / roof["peak"]

    e2e = None
    if not args.no_e2e:
        # the user's call from host memory: setup from the host index map and b, a
        # solve of W + K outer iterations from a host start, host outputs; all host
        # buffers pinned, inputs generated before the timed region
        pe = mds.manidsdp_default_params()
        pe.precision_mode = prec
        pe.tensor_cores = prm.tensor_cores
        pe.max_outer = args.warmup + args.steps
        idx_h = torch.from_numpy(idx).pin_memory()
        b_h = torch.from_numpy(b).pin_memory()
        Y0h = torch.from_numpy(gaussian_factor(N, p0, args.seed + rank)).pin_memory()
        y_host = torch.empty(m, dtype=torch.float64).pin_memory()
        Yout = torch.empty(N * pe.p_max, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2 = mds.manidsdp_setup(N, m, idx_h, b_h, params=pe, stream=stream.cuda_stream)
        rep2, p2 = mds.manidsdp_solve(ctx2, Y0h, p0, Y_out=Yout, y_out=y_host)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        mds.manidsdp_destroy(ctx2)
        steps2 = max(1, rep2.outer)
        e2e = {"value": t_e2e / steps2, "unit": UNIT,
               "h2d_bytes_per_step": int((idx.nbytes + b.nbytes + Y0h.numel() * 8) / steps2),
               "d2h_bytes_per_step": int((m * 8 + N * p2 * 8) / steps2),
               "includes": f"setup (index-map validation, inverse map, H2D) + {rep2.outer} outer "
                           "iterations from a pinned host start + D2H of y and Y into pinned "
                           "buffers, per outer iteration"}

    solve60 = None
    if rank == 0 and args.solve_q > 0:
        Qs, cs, Ns, ms_, idxs, bs, p0s = workload(args.solve_q, args.seed)
        ps = mds.manidsdp_default_params()
        ps.precision_mode = prec
        ps.tensor_cores = prm.tensor_cores
        cs_ = mds.manidsdp_setup(Ns, ms_, idxs, bs, params=ps, stream=stream.cuda_stream)
        Y0s = torch.tensor(gaussian_factor(Ns, p0s, args.seed), device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rs, _ = mds.manidsdp_solve(cs_, Y0s, p0s)
        torch.cuda.synchronize()
        solve60 = {"q": args.solve_q, "N": Ns, "m": ms_, "s": time.perf_counter() - t0,
                   "eta_max": rs.eta_max, "value": rs.value, "outer": rs.outer,
                   "hessvecs": rs.hessvecs, "converged": rs.status == mds.OK}
        mds.manidsdp_destroy(cs_)

    compare = None
    if rank == 0 and args.compare_q > 0:
        # the same instance solved by the mixed form and by the plain FP64 form
        Qc, cc_, Nc, mc, idxc, bc, p0c = workload(args.compare_q, args.seed)
        Y0c = torch.tensor(gaussian_factor(Nc, p0c, args.seed), device="cuda")
        compare = {"q": args.compare_q, "N": Nc}
        for name, pm in (("mixed", mds.PREC_MIXED), ("fp64", mds.PREC_FP64)):
            pc = mds.manidsdp_default_params()
            pc.precision_mode = pm
            pc.tensor_cores = prm.tensor_cores
            cx = mds.manidsdp_setup(Nc, mc, idxc, bc, params=pc, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, _ = mds.manidsdp_solve(cx, Y0c, p0c)
            torch.cuda.synchronize()
            compare[name] = {"s": time.perf_counter() - t0, "eta_max": rc.eta_max,
                             "value": rc.value, "outer": rc.outer, "hessvecs": rc.hessvecs}
            mds.manidsdp_destroy(cx)
        compare["speedup_mixed_over_fp64"] = compare["fp64"]["s"] / compare["mixed"]["s"]
        compare["value_rel_diff"] = abs(compare["fp64"]["value"] - compare["mixed"]["value"]) / abs(
            compare["fp64"]["value"])

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        counts = dict(hessvecs=rep.hessvecs / steps_done, evals=rep.evals / steps_done,
                      grads=rep.grads / steps_done, lanczos_matvecs=rep.lanczos_matvecs / steps_done,
                      p=p_avg)
        cb = cpu_baseline(args.q, args.seed, counts, args.cpu_sample_s)

    mds.manidsdp_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / steps_done, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64 (FP32 Hessian-vector products, FP64 elsewhere)" if prec == mds.PREC_MIXED else "f64",
            "data": "synthetic (seeded N(0,1) Q, c; seeded Gaussian start)",
            "config": bench_config(args, world),
            "steps_done": steps_done, "eta_max_after": rep.eta_max, "value_after": rep.value,
            "outer_total": args.warmup + rep.outer, "full_solve": solve60,
            "rtr_iters": rep.rtr_iters, "hessvecs": rep.hessvecs, "p_final": rep.p,
            "phase_ms": {"hessvec": rep.ms_hessvec, "eval": rep.ms_eval, "grad": rep.ms_grad,
                         "lanczos_wall": rep.ms_lanczos},
            "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": int(launches),
            "mixed_vs_fp64": compare,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
