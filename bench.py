#!/usr/bin/env python
"""Benchmark of the explicit RKC EQS solver on GB300.

Metric: RKC DOF-stages/s (free unknowns x stages x steps / second) with
every stage M-solve at ||R - M z|| / ||R|| <= 1e-8, on the 64^3-cell
Kuhn cube (274,625 nodes, 266,175 free, 1.57 M tets, block varistor,
s = 20 stages, dt at the RKC stability bound).  The timed form is the
mixed-precision path; the plain FP64 AMG-PCG form is measured beside it.

A "step" is one RKC step (20 stages: element kernel, right-hand side, AMG-PCG
solve, recurrence) through the C ABI.  L2 is flushed (256 MiB write) between
timed steps, outside the timed intervals.  Multi-GPU runs are independent
replicas (one instance per GPU, no collective on the data path).

--impl reference times the CPU oracle on a bounded sample of the same
workload (first stages of an RKC step) with the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RKC DOF-stages/s and M-solve ms/RHS vs plain FP64 AMG-PCG at 1e-8 residual"
WORKLOADS = {
    1: "cube64_block: 64^3-cell Kuhn cube, 274625 nodes (266175 free), 1572864 P1 tets, "
       "block varistor, s=20, dt=beta_s/rho, rtol=1e-8",
    2: "cube128_jitter_spheres: 128^3-cell Kuhn cube with interior nodes jittered by +-0.2h, "
       "2146689 nodes (2113407 free), 12582912 P1 tets, two varistor spheres, s=20, "
       "dt=beta_s/rho, rtol=1e-8, 4-member ensemble (V0 x 0.5/1/1.5/2), M-solve right-hand "
       "sides blocked 4 at a time (SpMM)",
    3: "learned start vector on cube128_jitter_spheres (2113407 free rows, s=20, rtol=1e-8): "
       "trained on the GPU on 400 stage solutions of 20 FP64 steps, then mixed precision with "
       "the learned guess against the previous-solution guess",
    4: "batch64: 64 independent Kuhn cubes of seeded 16^3..48^3 cells, seeded block varistor "
       "(0.2-0.5 of the edge) and drive 5e3-2e4 V, s=10, dt=beta_s/rho, rtol=1e-8, "
       "mixed precision, one cooperative launch per stage",
}
RTOL = 1e-8
S_STAGES = 20
CONFIG_INDEX = 1
WORKLOAD = WORKLOADS[CONFIG_INDEX]
# AMG/solver options of the timed runs (both precisions): degree-1 Chebyshev
# smoothing and a 2066-row coarsest level (dense inverse: FP64 on the FP64
# path, its FP32 rounding on the mixed path) gave the lowest step time on
# GB300 among degree 1-3 and coarse sizes 88/2066; the SPE Gram pass hands
# its sums to a one-block solve (defer_sums 2; the CG hand-over measured
# slower and stays off).
SOLVER_OPTS = dict(cheb_degree=1, coarse_max=2500, persistent=0, coarse_split=0, defer_sums=2)
SPE_N = 6  # solutions spanning the SPE subspace
# DRAM bytes (read + write) of one k_spmv64 launch per workload from an ncu
# capture (profiles/k_spmv_split_cube64.md); None where not captured.
TRAFFIC_SPMV64 = {1: 33821696, 2: None}
# DRAM bytes (read + write) of one k_spmv_split launch per workload from an
# ncu capture (profiles/k_spmv_split_cube64.md); None where not captured.
TRAFFIC_SPLIT = {1: 32744704, 2: None}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--N", type=int, default=None, help="override mesh size (testing)")
    ap.add_argument("--config", type=int, default=1, choices=[1, 2, 3, 4],
                    help="workload: 1 = 64^3 block cube (default), 2 = 128^3 jittered spheres, "
                         "3 = learned guess on the 128^3 mesh, 4 = batched serving of 64 instances")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the CG loops from the host (same kernels; for ncu launch lists)")
    return ap.parse_args()


# ------------------------------------------------------------ replicas
def max_over_ranks(value, dist=None, device="cuda"):
    """Max of a per-rank scalar over all ranks (the slowest replica's time);
    the value itself without a process group."""
    if dist is None:
        return float(value)
    import torch

    tt = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(units_per_rank, world, total_ms):
    """Whole-job rate of independent replicas (weak scaling): every rank
    processes units_per_rank; the job takes the slowest rank's time."""
    return world * units_per_rank / (total_ms / 1e3)


# ------------------------------------------------------------------ oracle
ORACLE_SNIPPET = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import eqs_inputs as ei
from oracle import run
p = ei.config_problem({cfg}, N={N})
r = run.time_stage_sample(p, {s}, {n_stages}, rtol={rtol})
print(json.dumps(r))
"""


def oracle_sample(n_stages, N=None):
    """Run the oracle in a fresh single-threaded process (spawned, no CUDA)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, cfg=CONFIG_INDEX, N=N, s=S_STAGES, n_stages=n_stages,
                                 rtol=RTOL)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args, rank):
    if rank != 0:
        return
    n_stages = 2
    t_total, dof = 0.0, 0
    for k in range(args.warmup + args.steps):
        r = oracle_sample(n_stages, args.N)
        if k >= args.warmup:
            t_total += r["seconds"]
            dof += r["n_free"] * r["stages"]
    value = dof / t_total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-stages/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"first {n_stages} stages of an RKC step per step"},
        "cpu_baseline": {"value": value, "unit": "DOF-stages/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n_stages} stage evaluations per step, oracle numpy/scipy "
                                   f"FP64 AMG-PCG, single thread"},
        "e2e": {"value": value, "unit": "DOF-stages/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.p = None
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(dev_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm
def time_steps(torch, solver, x, t, dt, steps, flush, stream_sync=True):
    times, launches, iters = [], 0, []
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        solver.step(x, t, dt, S_STAGES, stats=False)
        e1.record()
        st = solver.last_stats()  # synchronises; outside the timed interval
        times.append(e0.elapsed_time(e1))
        launches += st.launches
        iters.append(st.total_iters / S_STAGES)
        t += dt
    return times, launches, iters, t


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import eqs_inputs as ei
    from paper_1612_09447_gb300 import eqs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    eqs.lib()
    p = ei.config_problem(CONFIG_INDEX, N=args.N)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    flushbuf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def flush():
        flushbuf.zero_()

    def make(precision, guess, theta=None):
        solver = eqs.Solver(p, precision=precision, rtol=RTOL, host_loop=int(args.host_loop),
                            spe_n=SPE_N, **SOLVER_OPTS)
        if theta is not None:
            eqs.eqs_guess_set_params(solver.ctx, theta)
        eqs.eqs_set_guess(solver.ctx, guess)
        return solver

    def measure(solver, steps, warmup):
        dt = solver.dt_bound(S_STAGES)
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        t = 0.0
        for _ in range(warmup):
            solver.step(x, t, dt, S_STAGES)
            t += dt
        barrier()
        clk = ClockSampler(local)
        times, launches, iters, t = time_steps(torch, solver, x, t, dt, steps, flush)
        barrier()
        return x, t, dt, times, launches, iters, clk.stop()

    def summary(times, iters):
        return {"value": p.n_free * S_STAGES * len(times) / (sum(times) / 1e3),
                "ms_per_step": sum(times) / len(times),
                "m_solve_ms_per_rhs": sum(times) / len(times) / S_STAGES,
                "cg_iters_per_solve": float(np.mean(iters))}

    # headline: mixed precision with the SPE start vector (Section IV)
    solver = make(eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_SPE)
    x, t, dt, times, launches, iters, clocks = measure(solver, args.steps, args.warmup)
    total_ms = max_over_ranks(sum(times), dist)
    units = world * p.n_free * S_STAGES * args.steps
    value = job_throughput(p.n_free * S_STAGES * args.steps, world, total_ms)

    # end to end through the public API: pinned host x in, step, x back to host
    xh = torch.zeros(p.n_nodes, dtype=torch.float64).pin_memory()
    xh.copy_(x.cpu())
    e2e_ms = 0.0
    for k in range(args.steps):
        flush()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t_host = time.perf_counter()
        e0.record()
        x.copy_(xh, non_blocking=True)
        solver.step(x, t, dt, S_STAGES, stats=False)
        xh.copy_(x, non_blocking=True)
        e1.record()
        e1.synchronize()
        e2e_ms += max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t_host))
        t += dt
    e2e_ms = max_over_ranks(e2e_ms, dist)
    e2e_value = units / (e2e_ms / 1e3)
    roof = dominant_kernel_roofline(torch, eqs, solver, p, flush)
    solver.close()

    variants = {}
    if not args.no_fp64:
        short = max(3, args.steps // 4)
        # fp64_plain is the metric's baseline: plain FP64 AMG-PCG, previous-solution start;
        # mixed_pod / mixed_pod2 are the paper's POD-MOR estimators (fixed / rolling set)
        for name, prec, guess in (("fp64_plain", eqs.EQS_PREC_FP64, eqs.EQS_GUESS_PREV),
                                  ("mixed_prev", eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_PREV),
                                  ("fp64_spe", eqs.EQS_PREC_FP64, eqs.EQS_GUESS_SPE),
                                  ("mixed_pod", eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_POD),
                                  ("mixed_pod2", eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_POD2)):
            S = make(prec, guess)
            r = measure(S, short, 2)
            variants[name] = summary(r[3], r[5])
            S.close()
        # learned start vector: record FP64 stage solutions, train on the GPU
        rec = make(eqs.EQS_PREC_FP64, eqs.EQS_GUESS_PREV, ei.mlp_init())
        eqs.eqs_guess_record(rec.ctx, 5 * S_STAGES)
        xr = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        dtr = rec.dt_bound(S_STAGES)
        for k in range(5):
            rec.step(xr, k * dtr, dtr, S_STAGES)
        t0 = time.perf_counter()
        lf, ll = eqs.eqs_guess_train(rec.ctx, 400, 8192, 2e-3, 1612094470)
        train_s = time.perf_counter() - t0
        theta = eqs.eqs_guess_get_params(rec.ctx)
        rec.close()
        S = make(eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_MLP, theta)
        r = measure(S, short, 2)
        variants["mixed_mlp"] = dict(summary(r[3], r[5]), train_s=train_s, loss_first=lf, loss_last=ll)
        S.close()

    if not args.no_ensemble:
        # 4-member ensemble (drive V0 x {0.5, 1, 1.5, 2}) on the same mesh:
        # every stage's four right-hand sides solved together (blocked CG)
        variants["ensemble4_mixed_prev"] = measure_ensemble(torch, eqs, p, make, flush,
                                                            max(3, args.steps // 4), 2)
        variants["ensemble4_mixed_spe"] = measure_ensemble(torch, eqs, p, make, flush,
                                                           max(3, args.steps // 4), 2, eqs.EQS_GUESS_SPE)
        if "mixed_prev" not in variants:
            S = make(eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_PREV)
            r = measure(S, max(3, args.steps // 4), 2)
            variants["mixed_prev"] = summary(r[3], r[5])
            S.close()

    if not args.no_fp64:
        variants["adaptive_mixed_spe"] = measure_adaptive(torch, eqs, p, make, max(4, args.steps // 2))
        if CONFIG_INDEX == 1 and args.N is None:
            variants["p2_cube32_mixed_spe"] = measure_p2(torch, eqs, flush, max(3, args.steps // 4))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rr = oracle_sample(4, args.N)
        cpu = {"value": rr["dof_stages_per_s"], "unit": "DOF-stages/s", "cores": 1, "kind": "oracle",
               "sample": f"first {rr['stages']} stage evaluations of one RKC step "
                         f"({rr['seconds']:.1f} s, numpy/scipy FP64 AMG-PCG with previous-solution "
                         f"start, single thread)"}
    if rank != 0:
        return
    ms_step = total_ms / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "DOF-stages/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64 mixed", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_free": p.n_free, "stages": S_STAGES, "rtol": RTOL,
                   "solver": dict(SOLVER_OPTS, spe_n=SPE_N),
                   "form": "mixed precision (FP32 element kernel and V-cycle; FP64 CG, recurrence) "
                           "+ SPE start vectors (Section IV)",
                   "m_solve_ms_per_rhs": ms_step / S_STAGES,
                   "cg_iters_per_solve": float(np.mean(iters)),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "forms": variants,
        "e2e": {"value": e2e_value, "unit": "DOF-stages/s", "h2d_bytes_per_step": p.n_nodes * 8,
                "d2h_bytes_per_step": p.n_nodes * 8},
        "gpu_launches": int(launches),
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


ENS_SCALES = (0.5, 1.0, 1.5, 2.0)


def measure_ensemble(torch, eqs, p, make, flush, steps, warmup, guess=None):
    """Timed RKC steps of the 4-trajectory ensemble (mixed precision; start
    vector: previous solution or SPE): DOF-stages count all four
    trajectories."""
    import numpy as np

    S = make(eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_PREV if guess is None else guess)
    dt = S.dt_bound(S_STAGES)
    x = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    t = 0.0
    for _ in range(warmup):
        eqs.eqs_ens_rkc_step(S.ctx, x, ENS_SCALES, t, dt, S_STAGES)
        t += dt
    torch.cuda.synchronize()
    times, iters, passes, launches = [], [], 0, 0
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        eqs.eqs_ens_rkc_step(S.ctx, x, ENS_SCALES, t, dt, S_STAGES, want_stats=False)
        e1.record()
        st = eqs.eqs_ens_get_step_stats(S.ctx)
        times.append(e0.elapsed_time(e1))
        iters.append([v / S_STAGES for v in st.total_iters])
        passes += st.passes
        launches += st.launches
        t += dt
    S.close()
    ms = sum(times) / len(times)
    return {"value": 4 * p.n_free * S_STAGES * len(times) / (sum(times) / 1e3), "ms_per_step": ms,
            "m_solve_ms_per_rhs": ms / (4 * S_STAGES),
            "cg_iters_per_solve_by_column": [float(v) for v in np.mean(iters, axis=0)],
            "cg_passes_per_stage": passes / (steps * S_STAGES), "drive_scales": list(ENS_SCALES),
            "gpu_launches_per_step": launches / steps}


def measure_p2(torch, eqs, flush, steps):
    """Quadratic (P2) elements on the 32^3-cell cube: the same 274,625 nodes
    as the 64^3 P1 cube, about twice the matrix non-zeros per row; mixed
    precision with SPE, s = 20 at the stability bound."""
    import eqs_inputs as ei

    q = ei.make_problem_p2(32)
    S = eqs.Solver(q, precision=eqs.EQS_PREC_MIXED, rtol=RTOL, spe_n=SPE_N, **SOLVER_OPTS)
    eqs.eqs_set_guess(S.ctx, eqs.EQS_GUESS_SPE)
    rows, nnz = S.amg_info()
    dt = S.dt_bound(S_STAGES)
    x = torch.zeros(q.n_nodes, dtype=torch.float64, device="cuda")
    t = 0.0
    for _ in range(2):
        S.step(x, t, dt, S_STAGES)
        t += dt
    times, iters = [], 0
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        S.step(x, t, dt, S_STAGES, stats=False)
        e1.record()
        st = S.last_stats()
        times.append(e0.elapsed_time(e1))
        iters += st.total_iters
        t += dt
    S.close()
    return {"value": q.n_free * S_STAGES * steps / (sum(times) / 1e3), "ms_per_step": sum(times) / steps,
            "n_free": q.n_free, "nnz_per_row": nnz[0] / rows[0], "cg_iters_per_solve": iters / (steps * S_STAGES)}


def measure_adaptive(torch, eqs, p, make, steps):
    """Adaptive RKC (local error 1e-2 relative, 1e-2 V0 absolute, the
    paper's setting; s <= 64) from t = 0, mixed precision with SPE: accepted
    steps, stages and the simulated time per wall-clock second."""
    S = make(eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_SPE)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    t, h = 0.0, S.dt_bound(S_STAGES)
    for _ in range(2):  # graphs of the first stage counts, SPE history
        st = eqs.eqs_rkc_adaptive_step(S.ctx, x, t, h, 1e-2 * p.V0, 1e-2, 64)
        t, h = t + st.h_used, st.h_next
    torch.cuda.synchronize()
    t0_sim, wall0 = t, time.perf_counter()
    stages = tries = iters = 0
    hs, ss = [], []
    for _ in range(steps):
        st = eqs.eqs_rkc_adaptive_step(S.ctx, x, t, h, 1e-2 * p.V0, 1e-2, 64)
        t, h = t + st.h_used, st.h_next
        stages += st.s * st.tries
        tries += st.tries
        iters += st.total_iters
        hs.append(st.h_used)
        ss.append(st.s)
    wall = time.perf_counter() - wall0
    S.close()
    return {"value": p.n_free * stages / wall, "unit": "DOF-stages/s (all tries)", "steps": steps,
            "tries": tries, "mean_h_s": sum(hs) / len(hs), "mean_stages": sum(ss) / len(ss),
            "simulated_s_per_wall_s": (t - t0_sim) / wall, "ms_per_step": 1e3 * wall / steps,
            "cg_iters_per_solve": iters / max(1, stages), "tol": "rtol 1e-2, atol 1e-2 V0"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _time_launches(torch, fn, flush, reps=20):
    ts = []
    for _ in range(reps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts[3:])


def dominant_kernel_roofline(torch, eqs, solver, p, flush):
    """The CG operator product M z of the timed mixed path (k_spmv_split:
    M as two FP32 parts, FP32 z, FP32-pair row sums; the same row product
    as k_pcg_pq_split) timed alone with CUDA events on the launch stream,
    L2 flushed before each launch.  Algorithmic bytes per launch: 8 B per
    non-zero (hi + lo) + 4 B of z and 8 B of y per row.  The FP64 product
    (k_spmv64, the FP64 path's operator) is reported beside it."""
    nf = p.n_free
    rows, nnz = solver.amg_info()
    z = torch.randn(nf, dtype=torch.float32, device="cuda")
    x = z.double()
    y = torch.empty(nf, dtype=torch.float64, device="cuda")
    peak, kind = _peaks()
    ms32 = _time_launches(torch, lambda: eqs.eqs_spmv_M32(solver.ctx, z, y), flush)
    b32 = nnz[0] * 8 + nf * (4 + 8)
    ms64 = _time_launches(torch, lambda: eqs.eqs_spmv_M(solver.ctx, x, y), flush)
    b64 = nnz[0] * 8 + nf * 8 * 2
    ach = b32 / (ms32 / 1e3) / 1e9
    a64 = b64 / (ms64 / 1e3) / 1e9
    return {"kernel": "k_spmv_split (mixed-path CG operator product M z, as in k_pcg_pq_split)",
            "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": TRAFFIC_SPLIT.get(CONFIG_INDEX), "bytes_per_launch": b32, "ms_per_launch": ms32,
            "peak_kind": f"{kind} hbm_gbs (burst: kernel timed alone, L2 flushed before each launch)",
            "fp64_operator": {"kernel": "k_spmv64 (FP64 DIA SpMV of M_ff)", "achieved": a64, "frac": a64 / peak,
                              "bytes_per_launch": b64, "ms_per_launch": ms64,
                              "fp64_tflops": 2.0 * nnz[0] / (ms64 / 1e3) / 1e12,
                              "traffic": TRAFFIC_SPMV64.get(CONFIG_INDEX)}}


def run_batch(args, rank, world):
    """Batched serving: all instances advance together, one cooperative launch
    per stage (rows per CTA autotuned); the same instances stepped one after
    another with the single-instance graphs are measured beside it."""
    import torch

    import eqs_inputs as ei
    from paper_1612_09447_gb300 import autotune, eqs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    eqs.lib()
    dist = None
    if world > 1:  # replicas: every rank serves the whole batch on its own GPU
        import torch.distributed as dist
        dist.init_process_group("nccl")
    s = 10
    probs = [ei.config_problem(4, instance=i) for i in range(64)]
    # instances own a few CTAs each in the batched launch: lanes by row length only
    solvers = [eqs.Solver(p, precision=eqs.EQS_PREC_MIXED, rtol=RTOL, fill_lanes=0, **SOLVER_OPTS)
               for p in probs]
    nfree = sum(S.nf for S in solvers)
    best, tuning = autotune.tune_batch(eqs, solvers, candidates=(256, 512, 1024, 2048), s=s, steps=2)
    b = eqs.eqs_batch_create([S.ctx for S in solvers], best)
    ctas, rows_used = eqs.eqs_batch_info(b)
    dt = solvers[0].dt_bound(s)
    xs = [torch.zeros(S.n, dtype=torch.float64, device="cuda") for S in solvers]
    t = 0.0
    for _ in range(args.warmup):
        eqs.eqs_batch_rkc_step(b, xs, t, dt, s)
        t += dt
    flushbuf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    times, iters = [], 0
    for _ in range(args.steps):
        flushbuf.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        eqs.eqs_batch_rkc_step(b, xs, t, dt, s, want_stats=False)
        e1.record()
        st, _ = eqs.eqs_batch_get_stats(b, len(solvers))
        times.append(e0.elapsed_time(e1))
        iters += st.total_iters
        t += dt
    clocks = clk.stop()
    launches = st.launches * args.steps
    total_ms = max_over_ranks(sum(times), dist)
    value = job_throughput(nfree * s * args.steps, world, total_ms)
    # the same instances one after another (single-instance step graphs)
    xsolo = [torch.zeros(S.n, dtype=torch.float64, device="cuda") for S in solvers]
    ts = 0.0
    for S, x in zip(solvers, xsolo):
        S.step(x, 0.0, dt, s)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(2):
        for S, x in zip(solvers, xsolo):
            S.step(x, dt * (k + 1), dt, s, stats=False)
    e1.record()
    e1.synchronize()
    seq_value = nfree * s * 2 / (e0.elapsed_time(e1) / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "DOF-stages/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64 mixed", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances": len(solvers), "n_free_total": nfree,
                   "stages": s, "rtol": RTOL, "rows_per_block": rows_used, "ctas": ctas,
                   "autotune_ms_per_step": {str(k): v[0] for k, v in tuning.items()},
                   "cg_iters_per_solve": iters / (args.steps * s * len(solvers)),
                   "l2": "flushed between timed steps (256 MiB write)"},
        "sequential_single_instance": {"value": seq_value, "unit": "DOF-stages/s"},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    eqs.eqs_batch_destroy(b)
    for S in solvers:
        S.close()
    if dist is not None:
        dist.destroy_process_group()


def run_learned(args):
    """Record 20 FP64 steps (400 stage solutions) on the 128^3 jittered mesh,
    train the start-vector network on the GPU, then run mixed-precision steps
    with the learned guess and with the previous-solution guess."""
    import numpy as np
    import torch

    import eqs_inputs as ei
    from paper_1612_09447_gb300 import eqs

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    p = ei.config_problem(3, N=args.N)
    rec = eqs.Solver(p, precision=eqs.EQS_PREC_FP64, rtol=RTOL, **SOLVER_OPTS)
    eqs.eqs_guess_set_params(rec.ctx, ei.mlp_init())
    eqs.eqs_guess_record(rec.ctx, 20 * S_STAGES)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    dt = rec.dt_bound(S_STAGES)
    for k in range(20):
        rec.step(x, k * dt, dt, S_STAGES)
    x_start, t_start = x.clone(), 20 * dt
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lf, ll = eqs.eqs_guess_train(rec.ctx, 2000, 16384, 2e-3, 1612094470)
    train_s = time.perf_counter() - t0
    theta = eqs.eqs_guess_get_params(rec.ctx)
    rec.close()
    out = {}
    for name, guess in (("previous_solution", eqs.EQS_GUESS_PREV), ("learned", eqs.EQS_GUESS_MLP)):
        S = eqs.Solver(p, precision=eqs.EQS_PREC_MIXED, rtol=RTOL, **SOLVER_OPTS)
        eqs.eqs_guess_set_params(S.ctx, theta)
        eqs.eqs_set_guess(S.ctx, guess)
        x.copy_(x_start)
        t = t_start
        for _ in range(2):  # the history ring refills
            S.step(x, t, dt, S_STAGES)
            t += dt
        times, iters, kept = [], 0, 0
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            S.step(x, t, dt, S_STAGES, stats=False)
            e1.record()
            st = S.last_stats()
            times.append(e0.elapsed_time(e1))
            iters += st.total_iters
            kept += st.guess_kept
            t += dt
        out[name] = {"ms_per_step": float(np.mean(times)), "cg_iters_per_solve": iters / (args.steps * S_STAGES),
                     "value": p.n_free * S_STAGES * args.steps / (sum(times) / 1e3),
                     "learned_guess_kept": kept / (args.steps * S_STAGES)}
        S.close()
    line = {"metric": METRIC, "value": out["learned"]["value"], "unit": "DOF-stages/s", "n_gpus": 1,
            "steps": args.steps, "warmup": 2, "ms_per_step": out["learned"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64 mixed",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_free": p.n_free, "train_iters": 2000, "batch": 16384,
                       "train_s": train_s, "loss_first": lf, "loss_last": ll},
            "forms": out}
    print(json.dumps(line), flush=True)


def run_ensemble_headline(args, rank, world):
    """Config 2: the 4-member ensemble (drive V0 x {0.5, 1, 1.5, 2}) on the
    128^3 jittered mesh, every stage's four right-hand sides solved together
    (blocked CG, SpMM), mixed precision, per-column SPE start vectors."""
    import numpy as np
    import torch

    import eqs_inputs as ei
    from paper_1612_09447_gb300 import eqs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    eqs.lib()
    p = ei.config_problem(CONFIG_INDEX, N=args.N)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    flushbuf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def flush():
        flushbuf.zero_()

    def make(precision, guess):
        S = eqs.Solver(p, precision=precision, rtol=RTOL, host_loop=int(args.host_loop), spe_n=SPE_N,
                       **SOLVER_OPTS)
        eqs.eqs_set_guess(S.ctx, guess)
        return S

    S = make(eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_SPE)
    dt = S.dt_bound(S_STAGES)
    x = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    t = 0.0
    for _ in range(args.warmup):
        eqs.eqs_ens_rkc_step(S.ctx, x, ENS_SCALES, t, dt, S_STAGES)
        t += dt
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = ClockSampler(local)
    times, iters, launches = [], [], 0
    for _ in range(args.steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        eqs.eqs_ens_rkc_step(S.ctx, x, ENS_SCALES, t, dt, S_STAGES, want_stats=False)
        e1.record()
        st = eqs.eqs_ens_get_step_stats(S.ctx)
        times.append(e0.elapsed_time(e1))
        iters.append([v / S_STAGES for v in st.total_iters])
        launches += st.launches
        t += dt
    torch.cuda.synchronize()
    clocks = clk.stop()
    total_ms = max_over_ranks(sum(times), dist)
    units = world * 4 * p.n_free * S_STAGES * args.steps
    value = job_throughput(4 * p.n_free * S_STAGES * args.steps, world, total_ms)
    # end to end: pinned host x (4 trajectories) in, step, x back to host
    xh = torch.zeros((4, p.n_nodes), dtype=torch.float64).pin_memory()
    xh.copy_(x.cpu())
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t_host = time.perf_counter()
        e0.record()
        x.copy_(xh, non_blocking=True)
        eqs.eqs_ens_rkc_step(S.ctx, x, ENS_SCALES, t, dt, S_STAGES, want_stats=False)
        xh.copy_(x, non_blocking=True)
        e1.record()
        e1.synchronize()
        e2e_ms += max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t_host))
        t += dt
    e2e_ms = max_over_ranks(e2e_ms, dist)
    roof = dominant_kernel_roofline(torch, eqs, S, p, flush)
    S.close()
    forms = {}
    if not args.no_fp64:
        short = max(3, args.steps // 4)
        forms["ensemble4_mixed_prev"] = measure_ensemble(torch, eqs, p, make, flush, short, 2)
        for name, guess in (("single_mixed_spe", eqs.EQS_GUESS_SPE), ("single_mixed_prev", eqs.EQS_GUESS_PREV)):
            T = make(eqs.EQS_PREC_MIXED, guess)
            xs = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
            ts = 0.0
            for _ in range(2):
                T.step(xs, ts, dt, S_STAGES)
                ts += dt
            tm, it = [], []
            for _ in range(short):
                flush()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                T.step(xs, ts, dt, S_STAGES, stats=False)
                e1.record()
                stt = T.last_stats()
                tm.append(e0.elapsed_time(e1))
                it.append(stt.total_iters / S_STAGES)
                ts += dt
            T.close()
            forms[name] = {"value": p.n_free * S_STAGES * len(tm) / (sum(tm) / 1e3),
                           "ms_per_step": sum(tm) / len(tm), "cg_iters_per_solve": float(np.mean(it))}
    if rank != 0:
        return
    ms_step = total_ms / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "DOF-stages/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64 mixed", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_free": p.n_free, "trajectories": 4,
                   "drive_scales": list(ENS_SCALES), "stages": S_STAGES, "rtol": RTOL,
                   "solver": dict(SOLVER_OPTS, spe_n=SPE_N),
                   "form": "4-member ensemble, blocked CG (SpMM over the four right-hand sides of a "
                           "stage), mixed precision, per-column SPE start vectors (Section IV)",
                   "m_solve_ms_per_rhs": ms_step / (4 * S_STAGES),
                   "cg_iters_per_solve_by_column": [float(v) for v in np.mean(iters, axis=0)],
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "forms": forms,
        "e2e": {"value": units / (e2e_ms / 1e3), "unit": "DOF-stages/s",
                "h2d_bytes_per_step": 4 * p.n_nodes * 8, "d2h_bytes_per_step": 4 * p.n_nodes * 8},
        "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": None, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    global CONFIG_INDEX, WORKLOAD
    args = parse()
    CONFIG_INDEX = args.config
    WORKLOAD = WORKLOADS[CONFIG_INDEX]
    if args.config == 3 and args.impl == "ours":
        run_learned(args)
        return
    if args.config == 4 and args.impl == "ours":
        run_batch(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    if args.config == 2 and args.impl == "ours":
        run_ensemble_headline(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world)


if __name__ == "__main__":
    main()
