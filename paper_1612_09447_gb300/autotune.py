"""Autotuning of launch and solver parameters by measurement on the workload.

``tune_solver_by_class`` groups batched instances into size classes and picks,
per class, the solver options (Chebyshev smoother degree, coarsest-level
size) that give the shortest RKC step of the class's largest instance;
``tune_batch`` then picks the rows per CTA of the batched stage launch (how
many CTAs each instance's group gets) by timing batched steps.  Every
candidate is timed ``repeats`` times in interleaved rounds; the result keeps
the median and the spread (max - min) of each, so a winner can be compared
with the noise, and reports whether the winner's margin over the runner-up
exceeds both spreads.  ``tune_solver`` times option sets on one instance.
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


def _summary(samples):
    """{key: [ms, ...]} -> ({key: (median, spread)}, best key, separated)."""
    stats = {k: (statistics.median(v), max(v) - min(v)) for k, v in samples.items()}
    order = sorted(stats, key=lambda k: stats[k][0])
    best = order[0]
    separated = len(order) < 2 or (stats[order[1]][0] - stats[best][0] > max(stats[best][1], stats[order[1]][1]))
    return stats, best, separated


def tune_batch(eqs, solvers, candidates=(128, 256, 512, 1024, 2048, 4096), s=10, steps=3, warmup=1, repeats=3):
    """solvers: set-up mixed-precision eqs.Solver objects.  Returns (best
    rows_per_block, {rows_per_block: (median ms per step, spread, CTAs)},
    separated)."""
    import torch

    dt = solvers[0].dt_bound(s)
    xs = [torch.zeros(S.n, dtype=torch.float64, device="cuda") for S in solvers]
    batches, ctas = {}, {}
    for r in candidates:
        batches[r] = eqs.eqs_batch_create([S.ctx for S in solvers], r)
        ctas[r] = eqs.eqs_batch_info(batches[r])[0]
    samples = {r: [] for r in candidates}
    try:
        for _ in range(repeats):  # interleaved rounds: drift hits every candidate alike
            for r in candidates:
                for x in xs:
                    x.zero_()
                clock = [0.0]

                def run():
                    eqs.eqs_batch_rkc_step(batches[r], xs, clock[0], dt, s, want_stats=False)
                    clock[0] += dt

                samples[r].append(_time_steps(torch, run, steps, warmup))
    finally:
        for b in batches.values():
            eqs.eqs_batch_destroy(b)
    stats, best, separated = _summary(samples)
    return best, {r: (stats[r][0], stats[r][1], ctas[r]) for r in candidates}, separated


def tune_solver(eqs, problem, candidates, s=20, steps=3, warmup=1, rtol=1e-8, repeats=1, guess=None):
    """candidates: list of option dicts for eqs.Solver (mixed precision).
    Returns (best index, [median ms per step], [spread])."""
    import torch

    solvers = []
    for opts in candidates:
        S = eqs.Solver(problem, precision=eqs.EQS_PREC_MIXED, rtol=rtol, **opts)
        if guess is not None:
            eqs.eqs_set_guess(S.ctx, guess)
        solvers.append(S)
    samples = {i: [] for i in range(len(candidates))}
    try:
        for _ in range(repeats):
            for i, S in enumerate(solvers):
                x = torch.zeros(S.n, dtype=torch.float64, device="cuda")
                dt = S.dt_bound(s)
                clock = [0.0]

                def run():
                    S.step(x, clock[0], dt, s, stats=False)
                    clock[0] += dt

                samples[i].append(_time_steps(torch, run, steps, warmup))
    finally:
        for S in solvers:
            S.close()
    stats, best, _ = _summary(samples)
    return best, [stats[i][0] for i in range(len(candidates))], [stats[i][1] for i in range(len(candidates))]


def size_classes(problems, bounds=(26, 38)):
    """Instance indices grouped by mesh size N: N < bounds[0], ..., N >= bounds[-1]."""
    classes = [[] for _ in range(len(bounds) + 1)]
    for i, p in enumerate(problems):
        classes[sum(p.N >= b for b in bounds)].append(i)
    return [c for c in classes if c]


def tune_solver_by_class(eqs, problems, candidates, s=10, steps=3, warmup=2, repeats=3, guess=None,
                         bounds=(26, 38)):
    """Per size class, the option set with the shortest step of the class's
    largest instance.  Returns ([(instance indices, best options, medians,
    spreads)], options per instance)."""
    out, per_inst = [], [None] * len(problems)
    for cls in size_classes(problems, bounds):
        rep = max(cls, key=lambda i: problems[i].n_free)
        best, med, spread = tune_solver(eqs, problems[rep], candidates, s=s, steps=steps, warmup=warmup,
                                        repeats=repeats, guess=guess)
        out.append((cls, candidates[best], med, spread))
        for i in cls:
            per_inst[i] = candidates[best]
    return out, per_inst
