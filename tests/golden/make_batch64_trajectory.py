"""Writes batch64_trajectory.txt: the oracle's FP64 RKC trajectories of all
64 instances of the batched-serving workload at full size (Kuhn cubes of
seeded size 16^3..48^3 cells, seeded varistor block fraction and drive
amplitude, eqs_inputs.config_problem(4, instance=i)), used by
tests/test_gpu_fullsize_c24.py to check every instance of a batched step.

Run per instance: phi(0) = 0, the first 5 steps of the RKC scheme (Section
II; coefficients of the cited Sommeijer-Shampine-Verwer scheme) with s = 10
stages at the stability-bound step dt = beta_10 / rho (all instances share
materials, so they share dt and step in lockstep), t accumulated as
t += dt.  Every stage's M-solve is the oracle's AMG-preconditioned CG to
relative residual 1e-13, started from the previous stage's solution.  phi
is stored at 256 seeded sample nodes of each instance after steps 1 and 5.

This script calls only oracle/ and the seeded input generator.  About an
hour of CPU with 6 workers:

    python tests/golden/make_batch64_trajectory.py [--workers 6]
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import multiprocessing as mp  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import eqs_inputs as ei  # noqa: E402
from oracle import amg, dtbound, pcg, rkc, system  # noqa: E402

S_STAGES = 10
STEPS = (1, 5)
N_INSTANCES = 64
SAMPLE_SEED = 1612094477
N_SAMPLE = 256
RTOL = 1e-13


def _instance(i):
    t0 = time.time()
    p = ei.config_problem(4, instance=i)
    Sy = system.EQSSystem(p)
    H = amg.SAHierarchy(Sy.Mff)
    coef = rkc.RKCCoefficients(S_STAGES)
    dt = dtbound.dt_bound(p.materials, S_STAGES, coef)
    sample = np.sort(np.random.default_rng(SAMPLE_SEED + i).choice(p.n_nodes, N_SAMPLE, replace=False))
    last = [np.zeros(p.n_free)]

    def solve(R):
        z, _, ok = pcg.pcg(Sy.Mff, R, x0=last[0], precond=H, rtol=RTOL)
        if not ok:
            raise RuntimeError("oracle PCG did not converge")
        last[0] = z
        return z

    xf, t, saved = np.zeros(p.n_free), 0.0, {}
    for k in range(1, max(STEPS) + 1):
        xf, _ = rkc.rkc_step(lambda tt, y: Sy.F(tt, y, solve=solve), t, xf, dt, coef)
        t += dt
        if k in STEPS:
            saved[k] = Sy.full(t, xf)[sample]
    print(f"instance {i}: N {p.N}, {p.n_nodes} nodes, {time.time() - t0:.0f} s", flush=True)
    return i, p.N, float(dt), sample, saved


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=6)
    ap.add_argument("--count", type=int, default=N_INSTANCES)
    ap.add_argument("--out", default=os.path.join(HERE, "batch64_trajectory.txt"))
    args = ap.parse_args()
    t0 = time.time()
    # largest instances first so the pool's tail is short
    order = sorted(range(args.count), key=lambda i: -ei.batch_instance_params(i)[0])
    with mp.get_context("fork").Pool(args.workers) as pool:
        res = {r[0]: r for r in pool.imap_unordered(_instance, order)}
    dts = {r[2] for r in res.values()}
    assert len(dts) == 1
    with open(args.out, "w") as f:
        f.write(f"# oracle FP64 RKC trajectories of the batched-serving instances "
                f"(eqs_inputs.config_problem(4, instance=i), i < {args.count})\n")
        f.write(f"# written by tests/golden/make_batch64_trajectory.py; M-solves: oracle AMG-PCG, rtol {RTOL:g}\n")
        f.write(f"# s {S_STAGES}\n# dt {dts.pop()!r}\n# steps {' '.join(str(k) for k in STEPS)}\n")
        f.write(f"# sample_seed {SAMPLE_SEED} + instance\n# n_sample {N_SAMPLE}\n")
        f.write("# columns: instance, N, node, then phi after each listed step\n")
        for i in range(args.count):
            _, N, _, sample, saved = res[i]
            for j, node in enumerate(sample):
                f.write(f"{i} {N} {int(node)} " + " ".join(repr(float(saved[k][j])) for k in STEPS) + "\n")
    print(f"wrote {args.out} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
