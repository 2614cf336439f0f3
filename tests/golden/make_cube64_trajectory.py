"""Writes cube64_block_trajectory.txt: the oracle's FP64 RKC trajectory of the
64^3-cell block cube (274,625 nodes, 1,572,864 P1 tets; the P1 problem class
of Section V, built by the seeded recipe in eqs_inputs.mesh), used by
tests/test_gpu_fullsize.py to measure the GPU path's error on phi after N
steps at the benchmark's full size.

Run: phi(0) = 0, 100 steps of the RKC scheme (Section II; the coefficients
of the cited Sommeijer-Shampine-Verwer scheme) with s = 20 stages at the
stability-bound step dt = beta_20 / rho, t accumulated as t += dt.  Every
stage's M-solve is the oracle's AMG-preconditioned CG to relative residual
1e-13 (started from the previous stage's solution, which changes only the
iteration count).  phi is stored at 8192 seeded sample nodes after steps 50
and 100, next to the step size and the sample seed.

This script calls only oracle/ and the seeded input generator.  It runs for
about two hours:

    python tests/golden/make_cube64_trajectory.py [--steps 100]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import eqs_inputs as ei  # noqa: E402
from oracle import amg, dtbound, pcg, rkc, system  # noqa: E402

S_STAGES = 20
SAMPLE_SEED = 1612094475
N_SAMPLE = 8192
RTOL = 1e-13


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--out", default=os.path.join(HERE, "cube64_block_trajectory.txt"))
    args = ap.parse_args()
    p = ei.config_problem(1)
    Sy = system.EQSSystem(p)
    H = amg.SAHierarchy(Sy.Mff)
    coef = rkc.RKCCoefficients(S_STAGES)
    dt = dtbound.dt_bound(p.materials, S_STAGES, coef)
    last = [np.zeros(p.n_free)]

    def solve(R):
        z, _, ok = pcg.pcg(Sy.Mff, R, x0=last[0], precond=H, rtol=RTOL)
        if not ok:
            raise RuntimeError("oracle PCG did not converge")
        last[0] = z
        return z

    def F(t, xf):
        return Sy.F(t, xf, solve=solve)

    sample = np.sort(np.random.default_rng(SAMPLE_SEED).choice(p.n_nodes, N_SAMPLE, replace=False))
    keep = sorted({min(50, args.steps), args.steps})
    xf, t, saved = np.zeros(p.n_free), 0.0, {}
    t0 = time.time()
    for k in range(1, args.steps + 1):
        xf, _ = rkc.rkc_step(F, t, xf, dt, coef)
        t += dt
        if k in keep:
            saved[k] = Sy.full(t, xf)[sample]
        print(f"step {k}/{args.steps}  {time.time() - t0:.0f} s", flush=True)
    with open(args.out, "w") as f:
        f.write("# oracle FP64 RKC trajectory, 64^3-cell block cube (eqs_inputs.config_problem(1))\n")
        f.write(f"# written by tests/golden/make_cube64_trajectory.py; M-solves: oracle AMG-PCG, rtol {RTOL:g}\n")
        f.write(f"# s {S_STAGES}\n# dt {float(dt)!r}\n# steps {' '.join(str(k) for k in keep)}\n")
        f.write(f"# sample_seed {SAMPLE_SEED}\n# n_sample {N_SAMPLE}\n")
        f.write("# columns: node, then phi after each listed step\n")
        for i, node in enumerate(sample):
            f.write(f"{int(node)} " + " ".join(repr(float(saved[k][i])) for k in keep) + "\n")


if __name__ == "__main__":
    main()
