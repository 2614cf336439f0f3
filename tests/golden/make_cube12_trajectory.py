"""Writes cube12_block_trajectory.txt: the oracle's FP64 RKC trajectory of the
12^3-cell block cube (2,197 nodes, 1,859 free, 10,368 P1 tets; the small
P1 case of the seeded recipe in eqs_inputs.mesh), used by
tests/test_gpu_config0.py to compare the GPU path with the oracle over the
whole 200-step run of this case.

Run: phi(0) = 0, 200 steps of the RKC scheme (Section II; the coefficients
of the cited Sommeijer-Shampine-Verwer scheme) with s = 10 stages at the
stability-bound step dt = beta_10 / rho, t accumulated as t += dt.  Every
stage's M-solve is the oracle's AMG-preconditioned CG to relative residual
1e-13 (started from the previous stage's solution, which changes only the
iteration count).  phi is stored at every node after steps 1, 50, 100 and
200, next to the step size.

This script calls only oracle/ and the seeded input generator.  It runs for
about a minute:

    python tests/golden/make_cube12_trajectory.py
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import eqs_inputs as ei  # noqa: E402
from oracle import amg, dtbound, pcg, rkc, system  # noqa: E402

S_STAGES = 10
STEPS = 200
KEEP = (1, 50, 100, 200)
RTOL = 1e-13


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "cube12_block_trajectory.txt"))
    args = ap.parse_args()
    p = ei.config_problem(0)
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

    xf, t, saved = np.zeros(p.n_free), 0.0, {}
    for k in range(1, STEPS + 1):
        xf, _ = rkc.rkc_step(F, t, xf, dt, coef)
        t += dt
        if k in KEEP:
            saved[k] = Sy.full(t, xf)
    with open(args.out, "w") as f:
        f.write("# oracle FP64 RKC trajectory, 12^3-cell block cube (eqs_inputs.config_problem(0))\n")
        f.write(f"# written by tests/golden/make_cube12_trajectory.py; M-solves: oracle AMG-PCG, rtol {RTOL:g}\n")
        f.write(f"# s {S_STAGES}\n# dt {float(dt)!r}\n# steps {' '.join(str(k) for k in KEEP)}\n")
        f.write("# columns: node, then phi after each listed step\n")
        for node in range(p.n_nodes):
            f.write(f"{node} " + " ".join(repr(float(saved[k][node])) for k in KEEP) + "\n")


if __name__ == "__main__":
    main()
