"""Writes cube128_ensemble_trajectory.txt: the oracle's FP64 RKC trajectories
of the 128^3-cell jittered two-sphere mesh (2,146,689 nodes, 12,582,912 P1
tets; the P1 size of the paper's Section V model, built by the seeded recipe
in eqs_inputs.mesh), one per drive amplitude V0 x {0.5, 1, 1.5, 2} of the
four-member ensemble, used by tests/test_gpu_fullsize_c24.py to measure the
GPU path's error on phi at the benchmark's full size.

Run per member: phi(0) = 0, the first 5 steps of the RKC scheme (Section II;
coefficients of the cited Sommeijer-Shampine-Verwer scheme) with s = 20
stages at the stability-bound step dt = beta_20 / rho, t accumulated as
t += dt.  Every stage's M-solve is the oracle's AMG-preconditioned CG to
relative residual 1e-13, started from the previous stage's solution (the
start changes only the iteration count).  phi is stored at 8192 seeded
sample nodes after steps 1, 3 and 5.

The mesh, M and the AMG hierarchy do not depend on V0, so they are built
once and the four members run in forked worker processes.  This script
calls only oracle/ and the seeded input generator.  Several hours of CPU:

    python tests/golden/make_cube128_ensemble.py [--workers 4] [--N 128]
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import copy  # noqa: E402
import dataclasses  # noqa: E402
import multiprocessing as mp  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import eqs_inputs as ei  # noqa: E402
from oracle import amg, dtbound, pcg, rkc, system  # noqa: E402

S_STAGES = 20
STEPS = (1, 3, 5)
SCALES = (0.5, 1.0, 1.5, 2.0)
SAMPLE_SEED = 1612094476
N_SAMPLE = 8192
RTOL = 1e-13

_BASE = {}


def _member(scale):
    Sy0, H, dt, sample = _BASE["Sy"], _BASE["H"], _BASE["dt"], _BASE["sample"]
    Sy = copy.copy(Sy0)  # same mesh, M and geometry; only the drive changes
    Sy.p = dataclasses.replace(Sy0.p, V0=Sy0.p.V0 * scale)
    coef = rkc.RKCCoefficients(S_STAGES)
    last = [np.zeros(Sy.p.n_free)]
    iters = []

    def solve(R):
        z, it, ok = pcg.pcg(Sy.Mff, R, x0=last[0], precond=H, rtol=RTOL)
        if not ok:
            raise RuntimeError("oracle PCG did not converge")
        iters.append(it)
        last[0] = z
        return z

    xf, t, saved = np.zeros(Sy.p.n_free), 0.0, {}
    t0 = time.time()
    for k in range(1, max(STEPS) + 1):
        xf, _ = rkc.rkc_step(lambda tt, y: Sy.F(tt, y, solve=solve), t, xf, dt, coef)
        t += dt
        if k in STEPS:
            saved[k] = Sy.full(t, xf)[sample]
        print(f"scale {scale}: step {k}  {time.time() - t0:.0f} s  "
              f"mean CG iterations {np.mean(iters):.1f}", flush=True)
    return scale, saved


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    out = args.out or os.path.join(HERE, "cube128_ensemble_trajectory.txt")
    t0 = time.time()
    p = ei.config_problem(2, N=args.N)
    Sy = system.EQSSystem(p)
    Sy.geometry()
    H = amg.SAHierarchy(Sy.Mff)
    coef = rkc.RKCCoefficients(S_STAGES)
    dt = dtbound.dt_bound(p.materials, S_STAGES, coef)
    n_sample = min(N_SAMPLE, p.n_nodes)
    sample = np.sort(np.random.default_rng(SAMPLE_SEED).choice(p.n_nodes, n_sample, replace=False))
    _BASE.update(Sy=Sy, H=H, dt=dt, sample=sample)
    print(f"setup {time.time() - t0:.0f} s: {p.n_nodes} nodes, {len(H.levels)} AMG levels", flush=True)
    with mp.get_context("fork").Pool(min(args.workers, len(SCALES))) as pool:
        res = dict(pool.map(_member, SCALES))
    with open(out, "w") as f:
        f.write(f"# oracle FP64 RKC trajectories, {args.N}^3-cell jittered two-sphere mesh "
                f"(eqs_inputs.config_problem(2, N={args.N})), drive V0 x scale\n")
        f.write(f"# written by tests/golden/make_cube128_ensemble.py; M-solves: oracle AMG-PCG, rtol {RTOL:g}\n")
        f.write(f"# N {args.N}\n# s {S_STAGES}\n# dt {float(dt)!r}\n")
        f.write(f"# steps {' '.join(str(k) for k in STEPS)}\n")
        f.write(f"# scales {' '.join(repr(s) for s in SCALES)}\n")
        f.write(f"# sample_seed {SAMPLE_SEED}\n# n_sample {n_sample}\n")
        f.write("# columns: node, then phi for each scale (outer) after each listed step (inner)\n")
        for i, node in enumerate(sample):
            vals = [repr(float(res[sc][k][i])) for sc in SCALES for k in STEPS]
            f.write(f"{int(node)} " + " ".join(vals) + "\n")
    print(f"wrote {out} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
