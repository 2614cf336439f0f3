"""Oracle drivers: the RKC step with AMG-PCG stage solves (test infrastructure).

``PCGSolve`` is the M-solve of Section IV as the method runs it: CG with the
constant smoothed-aggregation preconditioner, started from the previous
solve's solution.  ``time_stage_sample`` runs the first ``n_stages`` stage
evaluations of one RKC step and reports DOF-stages per second; it is the
CPU baseline the benchmark prints next to the GPU numbers.
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
