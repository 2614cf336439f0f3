"""Oracle drivers: the RKC step with AMG-PCG stage solves (test infrastructure).

``PCGSolve`` is the M-solve of Section IV as the method runs it: CG with the
constant smoothed-aggregation preconditioner, started from the previous
solve's solution.  ``time_stage_sample`` runs the first ``n_stages`` stage
evaluations of one RKC step and reports DOF-stages per second;
``steady_stage_sample`` times the element operator and CG iterations at a
warm (previous-solution) stage and extrapolates the stage time.  They are
the CPU baselines the benchmark prints next to the GPU numbers.
"""
from __future__ import annotations

import time

import numpy as np

from . import amg, pcg, rkc, system


class PCGSolve:
    def __init__(self, S: system.EQSSystem, rtol=1e-8, hierarchy=None, **amg_opts):
        self.S = S
        self.H = hierarchy or amg.SAHierarchy(S.Mff, **amg_opts)
        self.rtol = rtol
        self.prev = np.zeros(S.Mff.shape[0])
        self.iters = []

    def __call__(self, R):
        z, it, ok = pcg.pcg(self.S.Mff, R, x0=self.prev, precond=self.H, rtol=self.rtol)
        if not ok:
            raise RuntimeError("oracle PCG did not converge")
        self.iters.append(it)
        self.prev = z
        return z


class _Enough(Exception):
    pass


def time_stage_sample(problem, s, n_stages, rtol=1e-8, dt=None):
    """Time the first n_stages stage evaluations (element operator + M-solve +
    recurrence) of an RKC step from phi = 0 at t = 0.  Setup (assembly, AMG
    hierarchy) is outside the timed region, as on the GPU."""
    from . import dtbound

    S = system.EQSSystem(problem)
    solve = PCGSolve(S, rtol=rtol)
    coef = rkc.RKCCoefficients(s)
    dt = dt or dtbound.dt_bound(problem.materials, s)
    count = [0]

    def F(t, y):
        if count[0] >= n_stages:
            raise _Enough
        count[0] += 1
        return S.F(t, y, solve)

    t0 = time.perf_counter()
    try:
        rkc.rkc_step(F, 0.0, np.zeros(problem.n_free), dt, coef)
    except _Enough:
        pass
    el = time.perf_counter() - t0
    return {"seconds": el, "stages": count[0], "n_free": problem.n_free,
            "dof_stages_per_s": problem.n_free * count[0] / el, "cg_iters": solve.iters}


def steady_stage_sample(problem, s, warm_stages, samples, rtol=1e-8, dt=None, with_K=True, report=None):
    """CPU baseline at steady state (the previous-solution start of the
    method).  Runs ``warm_stages`` stage evaluations of the first RKC step
    from phi = 0 (untimed as a whole; full M-solves to rtol, each started
    from the previous solve's solution; the element operator with the
    right-hand side, R of Eq. 2, is timed in each: t_K); the last one gives
    the steady-state CG iteration count it_ss.  Then ``samples`` times, on
    that last stage's state: a PCG solve cut after its first iteration from
    the previous solution (timed: t_1; it applies M and the V-cycle twice,
    i.e. costs about two CG iterations) and, with ``with_K``, the element
    operator again (timed: t_K; otherwise the warm stages' mean t_K is
    used).  Stage time is extrapolated as t_K + (it_ss / 2) t_1 and
    reported as DOF-stages/s = n_free / stage time.  ``report(k, dict)`` is
    called after every sample."""
    from . import dtbound

    S = system.EQSSystem(problem)
    S.geometry()
    solve = PCGSolve(S, rtol=rtol)
    coef = rkc.RKCCoefficients(s)
    dt = dt or dtbound.dt_bound(problem.materials, s)
    state, tKs = {}, []
    count = [0]

    def F(t, y):
        if count[0] >= warm_stages:
            state["t"], state["y"] = t, y
            raise _Enough
        count[0] += 1
        t0 = time.perf_counter()
        R = S.rhs(t, y)
        tKs.append(time.perf_counter() - t0)
        return solve(R)

    try:
        rkc.rkc_step(F, 0.0, np.zeros(problem.n_free), dt, coef)
    except _Enough:
        pass
    it_ss = solve.iters[-1]
    R = S.rhs(state["t"], state["y"])
    out = []
    for k in range(samples):
        t0 = time.perf_counter()
        if with_K:
            R = S.rhs(state["t"], state["y"])
        t1 = time.perf_counter()
        pcg.pcg(S.Mff, R, x0=solve.prev, precond=solve.H, rtol=0.0, maxit=1)
        t2 = time.perf_counter()
        tK = t1 - t0 if with_K else float(np.mean(tKs))
        t_1 = t2 - t1
        stage = tK + 0.5 * it_ss * t_1
        r = {"t_K": tK, "t_pcg1": t_1, "cg_iters_ss": it_ss, "stage_s": stage,
             "sample_s": t2 - t0, "n_free": problem.n_free,
             "dof_stages_per_s": problem.n_free / stage, "warm_iters": list(solve.iters),
             "warm_t_K": tKs}
        out.append(r)
        if report:
            report(k, r)
    return out
