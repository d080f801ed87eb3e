#!/usr/bin/env python
"""ManiDSDP on one GB300: solve time to KKT residual <= 1e-8.

Workload: the order-2 moment relaxation of a dense binary quadratic program
min x'Qx + c'x over x in {-1,1}^80 (Section 6.1): moment matrix 3241 x 3241,
1,666,981 classes (monomials of degree <= 4), Q and c iid N(0,1) from seed 0,
p_0 = ceil(ln m) = 15 (Section 6.1 sets p_0 = ceil(log m)).

A step is one complete solve of Algorithm 1 from the seeded start to
eta_max <= 1e-8 (every ALM outer iteration: the RTR solve of the subproblem with
its tCG Hessian-vector products, the multiplier update, the Lanczos certificate
check, the rank and sigma updates, the rank-one rounding), in the
mixed-precision form (tensor-core FP32 Hessian-vector products, df64 cost and
gradient, FP64 multiplier, KKT residuals and Lanczos).  Every step restarts from
the same seeded factor with a zero multiplier, so all steps do the same work.
The inputs (index map, b) sit in HBM before the timed region; the working set
(index map 42 MB, N x N FP64 multiplier and G 84 MB each, the tensor-core
operand pairs 168 MB) exceeds the 129 MB L2, so no flush is needed between
steps.  value = CUDA-event time of the K timed solves / K, in s per solve.

Beside the headline the line reports the same comparison for the plain FP64
GPU form (`mixed_vs_fp64`, at --fp64-q, default 40; the FP64 form at q = 80
takes minutes), the Hess-vec's rate against the tensor pipe (`roofline`), an
end-to-end solve through the C ABI from pinned host buffers (`e2e`) and the FP64
oracle timed on the host cores (`cpu_baseline`).

The `batched` object times the batched persistent solver on its own workload:
4096 independent BQP relaxations (3072 first-order with n in [16, 64], 1024
second-order with n in [6, 14]) solved to KKT <= 1e-8 in one launch, in
solves/s, against the per-context FP64 form on a sample (--no-batched skips it).

Under torchrun (N > 1) each rank solves its own replica (the single-instance
path has no exchange step); value = max-over-ranks time / (K x ranks).

`--impl reference` times the FP64 CPU oracle, as it stands, on the host cores:
each step executes a bounded sample of the same workload (Hessian-vector
products, cost-plus-gradient evaluations and certificate matvecs at the factor
width the GPU solve averages) and scales it to one solve by the operation
counts of the GPU solve (see the JSON's cpu_baseline.sample).
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
UNIT = "s/solve"

# Operation counts of one solve of this workload in the mixed form with the
# tensor-core engine (GB300 run of this bench), used to scale the oracle's
# sampled timings to one solve when no GPU run precedes them (the reference arm).
# The GPU arm uses the counts of its own timed solves.
DEFAULT_COUNTS = dict(hessvecs=20885, evals=820, lanczos_matvecs=21230, p=298,
                      outer=36)

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum over the kernels of one
# Hess-vec) from one ncu capture at q = 80, per p; "current" is False when the
# kernels changed after the capture (the line then reports traffic null).
HV_TRAFFIC = {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--q", type=int, default=80)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--engine", choices=["fma", "tc"], default="tc",
                    help="FP32 Hessian-vector product: FP32 FMA kernels or the TMA-fed "
                         "tcgen05 engine (TF32 pairs, three products per step)")
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--hv-reps", type=int, default=30)
    ap.add_argument("--fp64-q", type=int, default=40,
                    help="instance size of the mixed-vs-FP64 solve comparison (0 skips it)")
    ap.add_argument("--tcg-host", action="store_true",
                    help="launch the tCG kernels from the host instead of the device-driven graph "
                         "(same kernels; for profilers that list kernels one launch at a time)")
    ap.add_argument("--hv-only", type=int, default=0,
                    help="only time the Hessian-vector product at this p (profiling)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-solver line (4096 small relaxations in one launch)")
    ap.add_argument("--batched-steps", type=int, default=3)
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched solver (profiling)")
    ap.add_argument("--batched-uniform", type=str, default="",
                    help="with --batched-only: 'n,count' -- count second-order relaxations at this n "
                         "(seeds 5000 + i) in place of the 4096-instance mix, 256 threads per CTA, "
                         "one launch, no tuner")
    ap.add_argument("--formulation-curve", type=str, default="",
                    help="comma-separated q values: solve each dense BQP relaxation with the "
                         "projected (DSDP') and the direct (DSDP) formulation and print one JSON "
                         "line per q (the paper's DSDP'-versus-DSDP comparison)")
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
            "hessvec_engine": ("tensor cores (TMA-fed tcgen05 kind::tf32, TF32 operand pairs, "
                               "three products per step)" if args.engine == "tc" else "FP32 FMA"),
            "step": "one full solve of Algorithm 1 from the seeded start to eta_max <= 1e-8",
            "l2": "working set > L2 (idx 42 MB, N x N FP64 multiplier and G 84 MB each, "
                  "tensor-core operand pairs 168 MB), no flush",
            "parallelism": f"replicas{world}"}


def reduce_over_ranks(ms, steps_done, world, device):
    """Replicas: the job's timed-region length is the slowest rank's, and its
    work is the sum of the steps all ranks completed."""
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
    """Seconds per step (one solve) of the whole job."""
    return ms_max / 1e3 / max(1, total_steps)


def workload(q, seed):
    import paper_2512_04406_gb300 as mds
    from synthetic import bqp_instance
    Q, c = bqp_instance(q, seed)
    N, m, idx = mds.manidsdp_bqp_index_map(q, 2)
    b = mds.manidsdp_bqp_rhs(q, Q, c, 2)
    p0 = int(math.ceil(math.log(m)))
    return Q, c, N, m, idx, b, p0


def hessvec_flops(N, p):
    """Algorithmic flops of one Hessian-vector product (Proposition 4.2): the
    SDDMM W = Y U' + U Y' on the N(N+1)/2 upper-triangle entries (2p multiply-adds
    each) and the gather GEMM [G | A*(w)] [U ; Y] (2N multiply-adds per output):
    2 N^2 p + 4 N^2 p."""
    return 6.0 * N * N * p


def hessvec_bytes(N, p, fp_bytes):
    """Algorithmic DRAM bytes of one Hessian-vector product in its stored-G form:
    G once (fp_bytes per entry) and the index map once per pass (4 bytes per
    entry for the class sums over the upper triangle, 4 per entry for the
    gather), w, Y, U L2-resident, HU written once (8 bytes per row element)."""
    return (fp_bytes + 4) * N * N + 4 * N * (N + 1) / 2 + 8 * N * p


def measure_hessvec(mds, torch, ctx, N, p, reps, precision, seed=11):
    """Mean device time of one Hessian-vector product at a random unit-row Y
    (CUDA events on the library's stream)."""
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
    workload's size and the GPU solve's mean factor width, then scale by the
    operation counts of one solve."""
    from oracle import manidsdp as om, moment, subproblem as sp
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
                   f"solve from the GPU solve's counts (hessvecs={counts['hessvecs']:.0f}, "
                   f"evals={counts['evals']:.0f}, lanczos matvecs={counts['lanczos_matvecs']:.0f}, "
                   f"mean p={counts['p']:.0f}); index-map setup {t_setup:.1f} s not included"),
    }


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps, walls = [], []
    cb = None
    # each step a bounded sample: the whole run stays within a few minutes
    budget = max(1.0, min(args.cpu_sample_s, 120.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(args.q, args.seed, DEFAULT_COUNTS, budget)
        if i >= args.warmup:
            steps.append(cb["value"])
            walls.append(time.perf_counter() - t0)
    value = statistics.mean(steps)
    cb["value"] = value
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        # the executed part of each step: a bounded sample whose operation times
        # `value` scales to one solve (cpu_baseline.sample says how)
        "ms_per_step": statistics.mean(walls) * 1e3,
        "value_is": "projection of one oracle solve from the sampled operation times x the GPU "
                    "solve's operation counts; ms_per_step is the wall time actually executed "
                    "per step",
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded N(0,1) Q, c)",
        "config": bench_config(args, world),
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batched_mix():
    """The batch of independent BQP relaxations: 3072 first-order with n uniform on
    [16, 64] and 1024 second-order with n uniform on [6, 14] (Q, c iid N(0, 1),
    instance i seeded 1000 + i; starting factors N_i x 2 Gaussian, same seeds),
    built by the library's host helpers."""
    import paper_2512_04406_gb300 as mds
    from synthetic import batched_bqp_sizes, bqp_instance, gaussian_factor
    s1, s2 = batched_bqp_sizes(3072, 1024, 16, 64, 6, 14)
    spec = [(int(n), 1) for n in s1] + [(int(n), 2) for n in s2]
    maps = {}
    Ns, ms, idxs, bs, ys = [], [], [], [], []
    for i, (q, order) in enumerate(spec):
        if (q, order) not in maps:
            maps[(q, order)] = mds.manidsdp_bqp_index_map(q, order)
        N, m, idx = maps[(q, order)]
        Q, c = bqp_instance(q, 1000 + i)
        Ns.append(N); ms.append(m); idxs.append(idx)
        bs.append(mds.manidsdp_bqp_rhs(q, Q, c, order))
        ys.append(gaussian_factor(N, 2, 1000 + i).ravel())
    return spec, Ns, ms, idxs, bs, np.concatenate(ys)


def run_formulation_curve(mds, torch, qs, engine, stream):
    """Solve time to eta_max <= 1e-8 of the q-variable dense BQP relaxation in the
    projected formulation (DSDP', Algorithm 1) and the direct one (two-block ADMM
    on DSDP, fixed penalty sigma = 0.25), mixed form, one solve each after a
    warm-up solve; CUDA events on the library's stream."""
    from synthetic import gaussian_factor
    for q in qs:
        Q, c, N, m, idx, b, p0 = workload(q, 0)
        Y0 = torch.tensor(gaussian_factor(N, p0, 0), device="cuda")
        row = {"formulation_curve": True, "q": q, "N": N, "m": m}
        for name, dflag in (("projected", 0), ("direct", 1)):
            prm = mds.manidsdp_default_params()
            prm.precision_mode = mds.PREC_MIXED
            prm.tensor_cores = 1 if engine == "tc" else 0
            prm.direct = dflag
            if dflag:
                prm.sigma0, prm.kappa1, prm.kappa2, prm.max_outer = 0.25, -1.0, 1e300, 1000
                prm.sigma_stall = 0.0
            ctx = mds.manidsdp_setup(N, m, idx, b, params=prm, stream=stream.cuda_stream)
            solve_once(mds, torch, ctx, Y0, p0, stream)  # warm-up (graphs, allocations)
            rep, p, ms = solve_once(mds, torch, ctx, Y0, p0, stream)
            mds.manidsdp_destroy(ctx)
            row[name] = {"s": ms / 1e3, "outer": rep.outer, "hessvecs": rep.hessvecs,
                         "eta_max": rep.eta_max, "value": rep.value,
                         "converged": rep.status == mds.OK}
        row["speedup_projected_over_direct"] = row["direct"]["s"] / row["projected"]["s"]
        print(json.dumps(row), flush=True)


def run_batched_uniform(mds, torch, spec, stream):
    """One launch over `count` second-order relaxations at size n (a profiling case)."""
    from synthetic import bqp_instance, gaussian_factor
    n, count = (int(v) for v in spec.split(","))
    N, m, idx = mds.manidsdp_bqp_index_map(n, 2)
    bs, ys = [], []
    for i in range(count):
        Q, c = bqp_instance(n, 5000 + i)
        bs.append(mds.manidsdp_bqp_rhs(n, Q, c, 2))
        ys.append(gaussian_factor(N, 2, 5000 + i).ravel())
    prm = mds.manidsdp_default_params()
    prm.p_max = 32
    prm.precision_mode = mds.PREC_MIXED
    bt = mds.manidsdp_batch_setup([N] * count, [m] * count, [idx] * count, bs, prm,
                                  stream=stream.cuda_stream)
    mds.manidsdp_batch_set_launch(bt, 256, 0)
    res, ms = mds.manidsdp_batch_solve(bt, np.concatenate(ys))
    mds.manidsdp_batch_destroy(bt)
    return {"batched_uniform": True, "n": n, "N": N, "count": count, "ms": ms,
            "all_converged": all(r.status == mds.OK for r in res),
            "hessvecs_mean": float(np.mean([r.hessvecs for r in res])),
            "hessvecs_max": int(max(r.hessvecs for r in res))}


def run_batched(mds, torch, steps, stream):
    """The batched persistent solver on the 4096-instance mix: solves/s at
    KKT <= 1e-8 (device time of the launch), after the launch-shape tuner, with
    an end-to-end figure (host starting factors in, host results out) and the
    per-context FP64 form (manidsdp_solve per instance) on a strided sample."""
    spec, Ns, ms, idxs, bs, Y0 = batched_mix()
    prm = mds.manidsdp_default_params()
    prm.p_max = 32
    prm.precision_mode = mds.PREC_MIXED
    bt = mds.manidsdp_batch_setup(Ns, ms, idxs, bs, prm, stream=stream.cuda_stream)
    Y0d = torch.tensor(Y0, device="cuda")
    shape = mds.manidsdp_batch_tune(bt, Y0d)
    t_dev, res = [], None
    for _ in range(steps):
        res, t = mds.manidsdp_batch_solve(bt, Y0d)
        t_dev.append(t)
    # end to end: host starting factors in, host results and multipliers out
    Y0h = torch.from_numpy(Y0).pin_memory()
    y_h = torch.empty(int(sum(ms)), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mds.manidsdp_batch_solve(bt, Y0h, y_h)
    t_e2e = time.perf_counter() - t0
    mds.manidsdp_batch_destroy(bt)
    n = len(spec)
    ms_dev = statistics.median(t_dev)
    # per-context FP64 form on a strided sample (one context per instance)
    sample = list(range(0, n, 128))
    t_ctx = 0.0
    ok_ctx = True
    for i in sample:
        pc = mds.manidsdp_default_params()
        pc.p_max = 32
        pc.precision_mode = mds.PREC_FP64
        off = sum(Ns[j] * 2 for j in range(i))
        t0 = time.perf_counter()
        cx = mds.manidsdp_setup(Ns[i], ms[i], idxs[i], bs[i], params=pc, stream=stream.cuda_stream)
        rc, _ = mds.manidsdp_solve(cx, Y0[off:off + Ns[i] * 2], 2)
        mds.manidsdp_destroy(cx)
        t_ctx += time.perf_counter() - t0
        ok_ctx &= rc.status == mds.OK
    ctx_rate = len(sample) / t_ctx
    return {
        "workload": "4096 independent BQP relaxations in one persistent launch: 3072 order-1 "
                    "(n uniform in [16, 64]) and 1024 order-2 (n uniform in [6, 14]), Q, c iid "
                    "N(0,1), instance i seeded 1000 + i",
        "metric": "solves/s at KKT<=1e-8", "value": n / (ms_dev * 1e-3), "unit": "solves/s",
        "ms_per_batch": ms_dev, "ms_steps": t_dev, "precision": "mixed (FP32 Hess-vec, FP64 rest)",
        "launch": {"threads": shape[0], "ctas_per_sm": shape[1], "tuned": True},
        "all_converged": all(r.status == mds.OK and r.eta_max <= 1e-8 for r in res),
        "max_eta": max(r.eta_max for r in res),
        "max_outer": max(r.outer for r in res), "hessvecs_total": int(sum(r.hessvecs for r in res)),
        "e2e": {"value": n / t_e2e, "unit": "solves/s",
                "h2d_bytes_per_step": int(Y0.nbytes), "d2h_bytes_per_step": int(n * 96 + y_h.numel() * 8),
                "includes": "H2D of the starting factors, the launch, D2H of the per-instance "
                            "results and the multipliers y (dV/db)"},
        "per_context_fp64": {"value": ctx_rate, "unit": "solves/s", "sample": len(sample),
                             "converged": ok_ctx,
                             "how": "manidsdp_setup + manidsdp_solve (FP64 form) + destroy per "
                                    "instance, every 128th instance, wall clock"},
        "speedup_vs_per_context_fp64": (n / (ms_dev * 1e-3)) / ctx_rate,
    }


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def solve_once(mds, torch, ctx, Y0, p0, stream, Y_out=None):
    """One step: a fresh solve (warm_start = 0) timed with CUDA events on the
    library's stream; the final factor lands in the device buffer Y_out."""
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rep, p = mds.manidsdp_solve(ctx, Y0, p0, Y_out=Y_out)
    e1.record(stream)
    e1.synchronize()
    return rep, p, e0.elapsed_time(e1)


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
    if args.formulation_curve:
        run_formulation_curve(mds, torch, [int(v) for v in args.formulation_curve.split(",")],
                              args.engine, torch.cuda.current_stream())
        return
    if args.batched_only:
        stream = torch.cuda.current_stream()
        out = (run_batched_uniform(mds, torch, args.batched_uniform, stream) if args.batched_uniform
               else run_batched(mds, torch, args.batched_steps, stream))
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = mds.PREC_MIXED if args.precision == "mixed" else mds.PREC_FP64
    Q, c, N, m, idx, b, p0 = workload(args.q, args.seed)
    prm = mds.manidsdp_default_params()
    prm.precision_mode = prec
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
        out = {"hv_only": True, "q": args.q, "N": N, "p": p, "precision": args.precision,
               "engine": args.engine, "ms": ms,
               "gbs": hessvec_bytes(N, p, 4 if prec == mds.PREC_MIXED else 8) / (ms * 1e-3) / 1e9,
               "tflops": hessvec_flops(N, p) / (ms * 1e-3) / 1e12}
        if args.hv_stages:
            out["stages_us"] = {k: round(v / calls * 1e3, 1) for k, v in stages.items()}
        print(json.dumps(out), flush=True)
        mds.manidsdp_destroy(ctx)
        return
    Y0 = torch.tensor(gaussian_factor(N, p0, args.seed + rank), device="cuda")
    for _ in range(args.warmup):
        solve_once(mds, torch, ctx, Y0, p0, stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    Yout = torch.empty(N * prm.p_max, dtype=torch.float64, device="cuda")
    l0 = mds.manidsdp_launch_count()
    reps, ms_steps = [], []
    torch.cuda.nvtx.range_push("timed")  # lets a profiler restrict itself to the timed steps
    for _ in range(args.steps):
        rep, p_fin, ms1 = solve_once(mds, torch, ctx, Y0, p0, stream, Yout)
        reps.append(rep)
        ms_steps.append(ms1)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = mds.manidsdp_launch_count() - l0
    clk = clocks.stop()
    ms = float(sum(ms_steps))
    ms, total_steps = reduce_over_ranks(ms, args.steps, world, "cuda")
    value = job_value(ms, total_steps)
    # tightness of the last timed solve: round its degree-1 moments to x in {-1,1}^q
    rep_t, p_t = reps[-1], p_fin
    tight = None
    if rep_t.status == mds.OK:
        Yf = Yout[: N * p_t].reshape(N, p_t).cpu().numpy()
        S01 = Yf[1:args.q + 1] @ Yf[0]  # S[0, 1..q]: the degree-1 moments
        x = np.where(S01 >= 0, 1.0, -1.0)
        fx = float(x @ Q @ x + c @ x)
        tight = {"f_xhat": fx, "value": rep_t.value, "p_final": p_t,
                 "rel_gap": abs(fx - rep_t.value) / (1.0 + abs(rep_t.value)),
                 "tight": abs(fx - rep_t.value) <= 1e-8 * (1.0 + abs(rep_t.value))}

    # dominant work: the Hessian-vector products, timed live (phase events inside
    # the timed solves)
    hv_ms_total = sum(r.ms_hessvec for r in reps)
    hv_count = sum(r.hessvecs for r in reps)
    p_avg = sum(r.hessvec_p_sum for r in reps) / max(1, hv_count)
    hv_ms = hv_ms_total / max(1, hv_count)
    peaks = load_peaks()
    flops = hessvec_flops(N, p_avg)
    byts = hessvec_bytes(N, p_avg, 4 if prec == mds.PREC_MIXED else 8)
    if prec == mds.PREC_MIXED and args.engine == "tc":
        # kernel timed inside a long step: the sustained bf16 figure, TF32 at half of it
        if "bf16_tflops_sustained" in peaks:
            peak, src = peaks["bf16_tflops_sustained"] * 0.5, "measured (bf16 sustained x 1/2 for TF32)"
        else:
            peak, src = 1700.0 * 0.5, "fallback (bf16 sustained x 1/2 for TF32)"
        roof = {"bound": "tensor", "achieved": flops / (hv_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": src}
    elif prec == mds.PREC_MIXED:
        roof = {"bound": "hbm", "achieved": byts / (hv_ms * 1e-3) / 1e9,
                "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s",
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    else:
        fp64_peak = 1.19  # TFLOP/s: 152 SMs x 2 DFMA/clk x 2 flop x ~1.95 GHz, probe-measured
        roof = {"bound": "alu", "achieved": flops / (hv_ms * 1e-3) / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "peak_source": "FP64 FMA probe on GB300"}
    tr = HV_TRAFFIC.get(args.engine)
    roof.update({"frac": roof["achieved"] / roof["peak"],
                 "traffic": tr["bytes"] if tr and tr.get("current") else None,
                 "kernel": "Hessian-vector product (SDDMM class sums + gather GEMM + epilogue)",
                 "avg_ms": hv_ms, "p_avg": p_avg, "hessvecs_per_solve": hv_count / len(reps),
                 "algorithmic_flops": flops, "algorithmic_bytes": byts,
                 "hbm_gbs": byts / (hv_ms * 1e-3) / 1e9})

    e2e = None
    if not args.no_e2e:
        # the user's call from host memory: setup from the host index map and b, a
        # full solve from a host start, host outputs; pinned host buffers, inputs
        # generated before the timed region
        pe = mds.manidsdp_default_params()
        pe.precision_mode = prec
        pe.tensor_cores = prm.tensor_cores
        idx_h = torch.from_numpy(idx).pin_memory()
        b_h = torch.from_numpy(b).pin_memory()
        Y0h = torch.from_numpy(gaussian_factor(N, p0, args.seed + rank)).pin_memory()
        y_host = torch.empty(m, dtype=torch.float64).pin_memory()
        z_host = torch.empty(N, dtype=torch.float64).pin_memory()
        Yh = torch.empty(N * pe.p_max, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2 = mds.manidsdp_setup(N, m, idx_h, b_h, params=pe, stream=stream.cuda_stream)
        rep2, p2 = mds.manidsdp_solve(ctx2, Y0h, p0, Y_out=Yh, y_out=y_host, z_out=z_host)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        mds.manidsdp_destroy(ctx2)
        e2e = {"value": t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(idx.nbytes + b.nbytes + Y0h.numel() * 8),
               "d2h_bytes_per_step": int(m * 8 + N * 8 + N * p2 * 8),
               "eta_max": rep2.eta_max, "converged": rep2.status == mds.OK,
               "includes": "setup (index-map validation, inverse map, H2D of idx and b) + one "
                           "solve from a pinned host start + D2H of y, z and Y into pinned buffers"}

    compare = None
    if rank == 0 and args.fp64_q > 0:
        # the same instance solved by the mixed form and by the plain FP64 form
        Qc, cc_, Nc, mc, idxc, bc, p0c = workload(args.fp64_q, args.seed)
        Y0c = torch.tensor(gaussian_factor(Nc, p0c, args.seed), device="cuda")
        compare = {"q": args.fp64_q, "N": Nc}
        for name, pm in (("mixed", mds.PREC_MIXED), ("fp64", mds.PREC_FP64)):
            pc = mds.manidsdp_default_params()
            pc.precision_mode = pm
            pc.tensor_cores = prm.tensor_cores
            cx = mds.manidsdp_setup(Nc, mc, idxc, bc, params=pc, stream=stream.cuda_stream)
            rc, _, msc = solve_once(mds, torch, cx, Y0c, p0c, stream)
            compare[name] = {"s": msc / 1e3, "eta_max": rc.eta_max, "value": rc.value,
                             "outer": rc.outer, "hessvecs": rc.hessvecs,
                             "converged": rc.status == mds.OK}
            mds.manidsdp_destroy(cx)
        compare["speedup_mixed_over_fp64"] = compare["fp64"]["s"] / compare["mixed"]["s"]
        compare["value_rel_diff"] = abs(compare["fp64"]["value"] - compare["mixed"]["value"]) / abs(
            compare["fp64"]["value"])

    batched = None
    if rank == 0 and not args.no_batched:
        batched = run_batched(mds, torch, args.batched_steps, stream)

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        counts = dict(hessvecs=hv_count / len(reps), evals=sum(r.evals for r in reps) / len(reps),
                      grads=sum(r.grads for r in reps) / len(reps),
                      lanczos_matvecs=sum(r.lanczos_matvecs for r in reps) / len(reps), p=p_avg)
        cb = cpu_baseline(args.q, args.seed, counts, args.cpu_sample_s)

    mds.manidsdp_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / max(1, total_steps) * world,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32/f64 (TF32-pair tensor-core Hessian-vector products, df64 cost and "
                      "gradient, FP64 multiplier, KKT residuals and Lanczos)"
                      if prec == mds.PREC_MIXED else "f64"),
            "data": "synthetic (seeded N(0,1) Q, c; seeded Gaussian start)",
            "config": bench_config(args, world),
            "solves": [{"s": t / 1e3, "eta_max": r.eta_max, "value": r.value, "outer": r.outer,
                        "hessvecs": r.hessvecs, "converged": r.status == mds.OK}
                       for r, t in zip(reps, ms_steps)],
            "all_converged": all(r.status == mds.OK and r.eta_max <= 1e-8 for r in reps),
            "tightness": tight,
            "phase_ms_per_solve": {
                "hessvec": hv_ms_total / len(reps),
                "eval": sum(r.ms_eval for r in reps) / len(reps),
                "grad": sum(r.ms_grad for r in reps) / len(reps),
                "lanczos": sum(r.ms_lanczos for r in reps) / len(reps),
                "rank_update_host": sum(r.ms_rank for r in reps) / len(reps)},
            "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": int(launches),
            "mixed_vs_fp64": compare,
            "batched": batched,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
