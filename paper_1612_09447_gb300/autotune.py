"""Autotuning of launch parameters by measurement on the actual workload.

``tune_batch`` picks the rows per CTA of the batched stage launch (how many
CTAs each instance's group gets) by timing batched RKC steps for each
candidate; ``tune_solver`` picks single-instance solver options (smoother
degree, coarsest-level size, persistent or graph CG loop) the same way.
Both return the best choice and every timing.
"""
from __future__ import annotations

import statistics


def _time_steps(torch, run, n, warmup):
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    ts = []
    for _ in range(n):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune_batch(eqs, solvers, candidates=(128, 256, 512, 1024, 2048, 4096), s=10, steps=3, warmup=1):
    """solvers: set-up mixed-precision eqs.Solver objects.  Returns
    (best rows_per_block, {rows_per_block: (ms per step, CTAs)})."""
    import torch

    dt = solvers[0].dt_bound(s)
    xs = [torch.zeros(S.n, dtype=torch.float64, device="cuda") for S in solvers]
    results = {}
    for r in candidates:
        b = eqs.eqs_batch_create([S.ctx for S in solvers], r)
        try:
            tb, _ = eqs.eqs_batch_info(b)
            for x in xs:
                x.zero_()
            clock = [0.0]

            def run():
                eqs.eqs_batch_rkc_step(b, xs, clock[0], dt, s, want_stats=False)
                clock[0] += dt

            results[r] = (_time_steps(torch, run, steps, warmup), tb)
        finally:
            eqs.eqs_batch_destroy(b)
    best = min(results, key=lambda k: results[k][0])
    return best, results


def tune_solver(eqs, problem, candidates, s=20, steps=3, warmup=1, rtol=1e-8):
    """candidates: list of option dicts for eqs.Solver (mixed precision).
    Returns (best index, [ms per step])."""
    import torch

    out = []
    for opts in candidates:
        S = eqs.Solver(problem, precision=eqs.EQS_PREC_MIXED, rtol=rtol, **opts)
        x = torch.zeros(S.n, dtype=torch.float64, device="cuda")
        dt = S.dt_bound(s)
        clock = [0.0]

        def run():
            S.step(x, clock[0], dt, s, stats=False)
            clock[0] += dt

        out.append(_time_steps(torch, run, steps, warmup))
        S.close()
    return min(range(len(out)), key=lambda i: out[i]), out
