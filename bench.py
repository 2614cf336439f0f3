#!/usr/bin/env python
"""Benchmark of the explicit RKC EQS solver on GB300.

Metric: RKC DOF-stages/s (free unknowns x stages x steps / second) with
every stage M-solve at ||R - M z|| / ||R|| <= 1e-8.  Default workload: the
128^3-cell jittered Kuhn cube with two varistor spheres (2,146,689 nodes,
2,113,407 free, 12.6 M P1 tets, s = 20 stages, dt at the RKC stability
bound), the paper's P1 problem size, as a 4-member ensemble (drive
V0 x 0.5/1/1.5/2) whose stage right-hand sides are solved 4 at a time, in
mixed precision with SPE start vectors.  The metric's comparison, plain FP64
AMG-PCG with the previous-solution start, and the other single-trajectory
forms are measured beside it on the same mesh (--config 1, 3, 4: the 64^3
cube, the learned start vector, batched serving).

A "step" is one RKC step (20 stages: element kernel, right-hand side, AMG-PCG
solve, recurrence) through the C ABI.  L2 is flushed (256 MiB write) between
timed steps, outside the timed intervals.  Multi-GPU runs are independent
replicas (one instance per GPU, no collective on the data path).

--impl reference times the CPU oracle on a bounded sample of the same
workload (steady-state CG iterations and the element operator of a warm
stage, stage time extrapolated) with the same metric.
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
CONFIG_INDEX = 2
WORKLOAD = WORKLOADS[CONFIG_INDEX]
# AMG/solver options of the timed runs (both precisions): degree-1 Chebyshev
# smoothing and a 2066-row coarsest level (dense inverse: FP64 on the FP64
# path, its FP32 rounding on the mixed path) gave the lowest step time on
# GB300 among degree 1-3 and coarse sizes 88/2066; the SPE Gram pass hands
# its sums to a one-block solve (defer_sums 2; the CG hand-over measured
# slower and stays off).
SOLVER_OPTS = dict(cheb_degree=1, coarse_max=2500, persistent=0, coarse_split=0, defer_sums=2)
SPE_N = 6  # solutions spanning the SPE subspace
# DRAM bytes (read + write) of one launch, per (eqs_launch_kernel id,
# workload), from an ncu capture of the lone launches of the current build on
# the full 128^3 workload (dram__bytes_read.sum + dram__bytes_write.sum, mean
# of 20 launches; the Gram pass is two kernels, summed); a kernel without an
# entry, or a run on another mesh size (--N), reports null.
TRAFFIC = {(16, 2): 943696013, (17, 2): 274488525, (18, 2): 524417740}


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
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4],
                    help="workload: 1 = 64^3 block cube, 2 = 128^3 jittered spheres (default), "
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
run.steady_stage_sample(p, {s}, {warm}, {samples}, rtol={rtol}, with_K={with_K},
                        report=lambda k, r: print(json.dumps(r), flush=True))
"""


def oracle_start(samples, N=None, warm=2, with_K=True):
    """Start the oracle's steady-state sampler in a fresh single-threaded
    process (no CUDA); it prints one JSON line per sample."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, cfg=1 if CONFIG_INDEX == 1 else 2, N=N, s=S_STAGES, warm=warm,
                                 samples=samples, rtol=RTOL, with_K=with_K)
    return subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                            stderr=subprocess.PIPE, text=True)


def oracle_collect(proc, timeout=1800):
    out, err = proc.communicate(timeout=timeout)
    if proc.returncode != 0:
        raise RuntimeError("oracle sample failed: " + err[-2000:])
    return [json.loads(line) for line in out.strip().splitlines() if line.startswith("{")]


def host_cores():
    return os.cpu_count() or 0


def cpu_baseline_entry(rs):
    """cpu_baseline object from the oracle's steady-state samples."""
    stage = sum(r["stage_s"] for r in rs) / len(rs)
    r = rs[-1]
    return {"value": r["n_free"] / stage, "unit": "DOF-stages/s", "cores": 1, "host_cores": host_cores(),
            "kind": "oracle",
            "sample": f"numpy/scipy FP64 oracle, single thread: {len(rs)} timed samples at a warm stage of "
                      f"the first RKC step (after {len(r['warm_iters'])} stages with full M-solves to 1e-8, "
                      f"previous-solution start; CG iterations {r['warm_iters']}): element operator + "
                      f"right-hand side t_K = {r['t_K']:.2f} s, a one-iteration PCG t_1 = {r['t_pcg1']:.2f} s; "
                      f"stage time extrapolated as t_K + (it_ss/2) t_1 with it_ss = {r['cg_iters_ss']}"}


def run_reference(args, rank):
    """The oracle (CPU, single thread) as the reference arm: setup and warm
    stages once, then per step one sample (a one-iteration PCG at the warm
    stage; the element operator time of the warm stages) extrapolated to a
    stage; value = DOF-stages/s over the timed steps."""
    if rank != 0:
        return
    proc = oracle_start(args.warmup + args.steps, args.N, warm=2, with_K=False)
    rs = oracle_collect(proc)[args.warmup:]
    t_total = sum(r["stage_s"] for r in rs) * S_STAGES
    dof = sum(r["n_free"] for r in rs) * S_STAGES
    value = dof / t_total
    cpu = cpu_baseline_entry(rs)
    cpu["sample"] += "; per step one one-iteration PCG sample, t_K from the warm stages"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-stages/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (single trajectory, previous-solution start)",
                   "sample": "per step: one RKC step's 20 stages extrapolated from one steady-state sample"},
        "cpu_baseline": dict(cpu, value=value),
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
    roof = kernel_roofline(torch, eqs, solver, p, flush,
                           {eqs.EQS_KERNEL_SPE_GRAM: S_STAGES, eqs.EQS_KERNEL_ELEM: S_STAGES,
                            eqs.EQS_KERNEL_PCG_PQ: float(np.mean(iters)) * S_STAGES},
                           total_ms / args.steps, CONFIG_INDEX if args.N is None else None)
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
        cpu = cpu_baseline_entry(oracle_collect(oracle_start(2, args.N)))
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


def kernel_bytes(eqs, kid, p, nnz0, nf):
    """Algorithmic bytes of one launch (what the kernel must move once):
    matrix values and per-row vectors read or written once, connectivity and
    materials once per cell (Kuhn cells: 8 corner indices + 6 material
    bytes) or per tet, node data once per node."""
    n = p.n_nodes
    cells = p.N ** 3 if p.tets.shape[1] == 4 else 0
    if kid == eqs.EQS_KERNEL_ENS_SPE_GRAM:  # M (hi, lo FP32), row sums (pair) + newest x, W, b and
        return 8 * nnz0 + (8 + 8 * 32) * nf  # 5 older columns, 4 values of 8 B each
    if kid == eqs.EQS_KERNEL_ENS_ELEM:  # cells + coords (hi, lo) + potentials (4 hi/lo pairs) + y (float4 RMW)
        return 38 * cells + (32 + 32 + 32) * n
    if kid == eqs.EQS_KERNEL_ENS_PCG_PQ:  # M (hi, lo FP32) + z (float4) + p, q (double4, read + write)
        return 8 * nnz0 + (16 + 64 + 64) * nf
    if kid == eqs.EQS_KERNEL_SPE_GRAM:  # M (FP64) + newest x, W, b and 5 older columns
        return 8 * nnz0 + 8 * 8 * nf
    if kid == eqs.EQS_KERNEL_ELEM:  # cells + coords (hi, lo) + potential (hi, lo) + y (float RMW)
        return 38 * cells + (32 + 8 + 8) * n
    if kid == eqs.EQS_KERNEL_PCG_PQ:  # M (hi, lo FP32) + z (float) + p, q (read + write)
        return 8 * nnz0 + (4 + 16 + 16) * nf
    raise ValueError(kid)


KERNEL_NAMES = {16: "k4_spe_w + k4_spe_gram_df<6> (ensemble SPE Gram pass: W = M x_new, then the dot products; double-float)",
                17: "k4_elem32_cell (ensemble element kernel)",
                18: "k4_pcg_pq (ensemble CG operator pass, split M)", 0: "k_spe_gram<6> (SPE Gram pass)",
                1: "k_elem32_cell (element kernel)", 2: "k_pcg_pq_split (CG operator pass, split M)"}


def kernel_roofline(torch, eqs, S, p, flush, kernels, step_ms, workload_key):
    """Each kernel of the last step timed alone (eqs_launch_kernel on the
    context stream, CUDA events, L2 flushed before every launch) with its
    algorithmic bytes; kernels: {id: launches per step}.  The roofline entry
    is the kernel with the largest (time per launch x launches per step);
    the element kernel is reported beside it."""
    rows, nnz = S.amg_info()
    peak, kind = _peaks()
    table = {}
    for kid, per_step in kernels.items():
        ms = _time_launches(torch, lambda: eqs.eqs_launch_kernel(S.ctx, kid), flush)
        b = kernel_bytes(eqs, kid, p, nnz[0], S.nf)
        ach = b / (ms / 1e3) / 1e9
        name = KERNEL_NAMES[kid]
        table[name] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                       "traffic": TRAFFIC.get((kid, workload_key)), "bytes_per_launch": b,
                       "ms_per_launch": ms, "launches_per_step": per_step,
                       "est_share_of_step": ms * per_step / step_ms}
    top = max(table, key=lambda k: table[k]["ms_per_launch"] * table[k]["launches_per_step"])
    elem = [k for k in table if "elem" in k][0]
    roof = dict(kernel=top, **table[top])
    roof["peak_kind"] = f"{kind} hbm_gbs (burst: kernel timed alone, L2 flushed before each launch)"
    roof["element"] = dict(kernel=elem, **table[elem])
    roof["kernels"] = table
    return roof


BATCH_SOLVER_CANDIDATES = (dict(cheb_degree=1, coarse_max=300), dict(cheb_degree=1, coarse_max=2500),
                           dict(cheb_degree=2, coarse_max=300), dict(cheb_degree=2, coarse_max=2500))
BATCH_ROWS_CANDIDATES = (256, 512, 1024, 2048)


def run_batch(args, rank, world):
    """Batched serving: all instances advance together, one cooperative launch
    per stage.  Solver options (smoother degree, coarsest-level size) are
    tuned per size class, rows per CTA for the batched launch; the timed
    batch starts every solve from the instance's SPE vector, the
    previous-solution batch and the same instances stepped one after another
    are measured beside it."""
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
    base = dict(SOLVER_OPTS)
    base.pop("cheb_degree")
    base.pop("coarse_max")
    classes, per_inst = autotune.tune_solver_by_class(
        eqs, probs, [dict(base, fill_lanes=0, spe_n=6, **c) for c in BATCH_SOLVER_CANDIDATES], s=s,
        guess=eqs.EQS_GUESS_SPE)
    # instances own a few CTAs each in the batched launch: lanes by row length only
    solvers = [eqs.Solver(p, precision=eqs.EQS_PREC_MIXED, rtol=RTOL, **o) for p, o in zip(probs, per_inst)]
    for S in solvers:
        eqs.eqs_set_guess(S.ctx, eqs.EQS_GUESS_SPE)
    nfree = sum(S.nf for S in solvers)
    best, tuning, separated = autotune.tune_batch(eqs, solvers, candidates=BATCH_ROWS_CANDIDATES, s=s, steps=2)
    flushbuf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    dt = solvers[0].dt_bound(s)

    def timed_batch(steps, warmup, clk=None):
        b = eqs.eqs_batch_create([S.ctx for S in solvers], best)
        ctas, rows_used = eqs.eqs_batch_info(b)
        xs = [torch.zeros(S.n, dtype=torch.float64, device="cuda") for S in solvers]
        t = 0.0
        for _ in range(warmup):
            eqs.eqs_batch_rkc_step(b, xs, t, dt, s)
            t += dt
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if clk else None
        times, iters = [], 0
        for _ in range(steps):
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
        clocks = sampler.stop() if sampler else None
        eqs.eqs_batch_destroy(b)
        return times, iters, st.launches * steps, ctas, rows_used, clocks

    times, iters, launches, ctas, rows_used, clocks = timed_batch(args.steps, args.warmup, clk=True)
    total_ms = max_over_ranks(sum(times), dist)
    value = job_throughput(nfree * s * args.steps, world, total_ms)
    # the previous-solution batch (same contexts, same tuned options)
    for S in solvers:
        eqs.eqs_set_guess(S.ctx, eqs.EQS_GUESS_PREV)
    short = max(3, args.steps // 4)
    ptimes, piters, _, _, _, _ = timed_batch(short, 2)
    # the same instances one after another (single-instance step graphs, SPE)
    for S in solvers:
        eqs.eqs_set_guess(S.ctx, eqs.EQS_GUESS_SPE)
    xsolo = [torch.zeros(S.n, dtype=torch.float64, device="cuda") for S in solvers]
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
                   "start_vector": "SPE (six solutions per instance, Gram pass inside the instance's CTA group)",
                   "autotune_rows_per_block": {str(k): {"ms_median": v[0], "ms_spread": v[1], "ctas": v[2]}
                                               for k, v in tuning.items()},
                   "autotune_rows_separated": separated,
                   "autotune_solver_by_class": [
                       {"instances": len(c), "N": [probs[i].N for i in c][:3] + ["..."], "best": o,
                        "ms_median": m, "ms_spread": sp} for c, o, m, sp in classes],
                   "cg_iters_per_solve": iters / (args.steps * s * len(solvers)),
                   "l2": "flushed between timed steps (256 MiB write)"},
        "forms": {"batched_previous_solution": {
            "value": nfree * s * len(ptimes) / (sum(ptimes) / 1e3), "ms_per_step": sum(ptimes) / len(ptimes),
            "cg_iters_per_solve": piters / (len(ptimes) * s * len(solvers))}},
        "sequential_single_instance": {"value": seq_value, "unit": "DOF-stages/s"},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
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


def time_single(torch, eqs, p, make, flush, prec, guess, steps, warmup=2, theta=None):
    """Single-trajectory steps on the workload's mesh: ms/step, CG
    iterations per solve, DOF-stages/s."""
    import numpy as np

    T = make(prec, guess, theta)
    dt = T.dt_bound(S_STAGES)
    xs = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    ts = 0.0
    for _ in range(warmup):
        T.step(xs, ts, dt, S_STAGES)
        ts += dt
    tm, it, kept = [], [], 0
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        T.step(xs, ts, dt, S_STAGES, stats=False)
        e1.record()
        stt = T.last_stats()
        tm.append(e0.elapsed_time(e1))
        it.append(stt.total_iters / S_STAGES)
        kept += stt.guess_kept
        ts += dt
    T.close()
    out = {"value": p.n_free * S_STAGES * len(tm) / (sum(tm) / 1e3), "ms_per_step": sum(tm) / len(tm),
           "m_solve_ms_per_rhs": sum(tm) / len(tm) / S_STAGES, "cg_iters_per_solve": float(np.mean(it)),
           "steps": steps}
    if guess == eqs.EQS_GUESS_MLP:
        out["learned_guess_kept"] = kept / (steps * S_STAGES)
    return out


def measure_spe_mlp(torch, eqs, p, make, flush, steps, n_rec=6, iters=1000):
    """The learned correction of the SPE start (EQS_GUESS_SPE_MLP): record
    n_rec mixed-precision SPE steps, train the network on the GPU, then time
    single-trajectory steps with the corrected start (network direction,
    M-norm line search) from the recorded state."""
    import eqs_inputs as ei

    R = make(eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_SPE, ei.mlp_init())
    eqs.eqs_guess_record(R.ctx, n_rec * S_STAGES)
    dt = R.dt_bound(S_STAGES)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    for k in range(n_rec):
        R.step(x, k * dt, dt, S_STAGES)
    eqs.eqs_set_guess(R.ctx, eqs.EQS_GUESS_SPE_MLP)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lf, ll = eqs.eqs_guess_train(R.ctx, iters, 8192, 2e-3, 1612094470)
    train_s = time.perf_counter() - t0
    theta = eqs.eqs_guess_get_params(R.ctx)
    R.close()
    out = time_single(torch, eqs, p, make, flush, eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_SPE_MLP, steps, theta=theta)
    out.update(train_s=train_s, loss_first=lf, loss_last=ll, recorded_steps=n_rec,
               note="starts from phi = 0 after training (the other forms likewise start from 0)")
    return out


def run_ensemble_headline(args, rank, world):
    """Config 2: the 4-member ensemble (drive V0 x {0.5, 1, 1.5, 2}) on the
    128^3 jittered mesh, every stage's four right-hand sides solved together
    (blocked CG, SpMM), mixed precision, per-column SPE start vectors.  The
    metric's comparison (plain FP64 AMG-PCG, previous-solution start) and the
    other single-trajectory forms run on the same mesh beside it."""
    import numpy as np
    import torch

    import eqs_inputs as ei
    from paper_1612_09447_gb300 import eqs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu_proc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_proc = oracle_start(2, args.N)  # runs on a host core while the GPU forms run
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

    def make(precision, guess, theta=None):
        S = eqs.Solver(p, precision=precision, rtol=RTOL, host_loop=int(args.host_loop), spe_n=SPE_N,
                       **SOLVER_OPTS)
        if theta is not None:
            eqs.eqs_guess_set_params(S.ctx, theta)
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
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    times, iters, launches, passes = [], [], 0, 0
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
        passes += st.passes
        t += dt
    torch.cuda.synchronize()
    clocks = clk.stop()
    if dist is not None:
        dist.barrier()
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
    ms_step = total_ms / args.steps
    roof = kernel_roofline(torch, eqs, S, p, flush,
                           {eqs.EQS_KERNEL_ENS_SPE_GRAM: S_STAGES, eqs.EQS_KERNEL_ENS_ELEM: S_STAGES,
                            eqs.EQS_KERNEL_ENS_PCG_PQ: passes / args.steps},
                           ms_step, CONFIG_INDEX if args.N is None else None)
    S.close()
    forms = {}
    if not args.no_fp64:
        short = max(3, args.steps // 4)
        forms["ensemble4_mixed_prev"] = measure_ensemble(torch, eqs, p, make, flush, short, 2)
        # the metric's baseline: plain FP64 AMG-PCG with the previous-solution start
        for name, prec, guess in (("fp64_plain", eqs.EQS_PREC_FP64, eqs.EQS_GUESS_PREV),
                                  ("single_mixed_prev", eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_PREV),
                                  ("single_fp64_spe", eqs.EQS_PREC_FP64, eqs.EQS_GUESS_SPE),
                                  ("single_mixed_spe", eqs.EQS_PREC_MIXED, eqs.EQS_GUESS_SPE)):
            forms[name] = time_single(torch, eqs, p, make, flush, prec, guess, short)
        forms["ensemble_vs_fp64_plain_per_trajectory_step"] = (
            forms["fp64_plain"]["ms_per_step"] / (ms_step / 4))
        forms["single_mixed_spe_mlp"] = measure_spe_mlp(torch, eqs, p, make, flush, short)
    cpu = None
    if cpu_proc is not None:
        cpu = cpu_baseline_entry(oracle_collect(cpu_proc))
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
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
                   "cg_passes_per_stage": passes / (args.steps * S_STAGES),
                   "l2": "flushed between timed steps (256 MiB write); working set > L2",
                   "parallelism": f"replicas x{world}"},
        "forms": forms,
        "e2e": {"value": units / (e2e_ms / 1e3), "unit": "DOF-stages/s",
                "h2d_bytes_per_step": 4 * p.n_nodes * 8, "d2h_bytes_per_step": 4 * p.n_nodes * 8},
        "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
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
