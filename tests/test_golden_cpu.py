"""The stored oracle trajectories are what the oracle computes now: the
first step of the 12^3 block cube's 200-step run, recomputed by the oracle
on the CPU, equals the stored step-1 column (a golden file that the oracle
no longer reproduces would make a GPU comparison against it meaningless)."""
import os

import numpy as np

import eqs_inputs as ei
from oracle import amg, dtbound, pcg, rkc, system

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cube12_block_trajectory.txt")


def _golden():
    meta, rows = {}, []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#"):
                parts = line[1:].split()
                if len(parts) >= 2 and parts[0] in ("s", "dt", "steps"):
                    meta[parts[0]] = parts[1:]
                continue
            rows.append([float(v) for v in line.split()])
    return meta, np.array(rows)


def test_cube12_golden_first_step_is_the_oracles():
    meta, a = _golden()
    p = ei.config_problem(0)
    s, dt = int(meta["s"][0]), float(meta["dt"][0])
    assert meta["steps"][0] == "1"
    coef = rkc.RKCCoefficients(s)
    assert dt == dtbound.dt_bound(p.materials, s, coef)
    Sy = system.EQSSystem(p)
    H = amg.SAHierarchy(Sy.Mff)
    last = [np.zeros(p.n_free)]

    def solve(R):
        z, _, ok = pcg.pcg(Sy.Mff, R, x0=last[0], precond=H, rtol=1e-13)
        assert ok
        last[0] = z
        return z

    xf, _ = rkc.rkc_step(lambda t, x: Sy.F(t, x, solve=solve), 0.0, np.zeros(p.n_free), dt, coef)
    got = Sy.full(dt, xf)
    assert np.array_equal(a[:, 0].astype(np.int64), np.arange(p.n_nodes))
    ref = a[:, 1]
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_batch_golden_first_step_of_the_smallest_instance_is_the_oracles():
    path = os.path.join(os.path.dirname(__file__), "golden", "batch64_trajectory.txt")
    dt = None
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("# dt "):
                dt = float(line.split()[2])
            if not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    a = np.array(rows)
    inst = int(a[np.argmin(a[:, 1]), 0])  # an instance of the smallest mesh
    sel = a[:, 0] == inst
    nodes, ref = a[sel, 2].astype(np.int64), a[sel, 3]
    p = ei.config_problem(4, instance=inst)
    assert p.N == int(a[sel, 1][0])
    s = 10
    coef = rkc.RKCCoefficients(s)
    assert dt == dtbound.dt_bound(p.materials, s, coef)
    Sy = system.EQSSystem(p)
    H = amg.SAHierarchy(Sy.Mff)
    last = [np.zeros(p.n_free)]

    def solve(R):
        z, _, ok = pcg.pcg(Sy.Mff, R, x0=last[0], precond=H, rtol=1e-13)
        assert ok
        last[0] = z
        return z

    xf, _ = rkc.rkc_step(lambda t, x: Sy.F(t, x, solve=solve), 0.0, np.zeros(p.n_free), dt, coef)
    got = Sy.full(dt, xf)[nodes]
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
