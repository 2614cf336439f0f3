"""Full-size trajectory parity of the ensemble and batched-serving workloads,
in the launch configuration the benchmark times (bench.py's solver options,
CUDA-graph steps, M-solves to 1e-8, mixed precision).

* The 128^3-cell jittered two-sphere mesh (2,146,689 nodes, 12,582,912
  tets), four-member ensemble with drive V0 x {0.5, 1, 1.5, 2} whose four
  stage right-hand sides are solved together (Section IV's multiple
  right-hand sides, blocked), SPE start vectors (Eq. 4-5): phi of every
  column after steps 1, 3 and 5 of the RKC scheme (Section II, s = 20,
  stability-bound dt) against the oracle's FP64 runs at 8192 sample nodes
  (tests/golden/cube128_ensemble_trajectory.txt, written by
  tests/golden/make_cube128_ensemble.py).  The single-trajectory form with
  SPE is checked against the V0 x 1 column.
* All 64 instances of the batched-serving workload at full size (16^3 to
  48^3 cells), one cooperative launch per stage, for every rows-per-CTA
  candidate of the benchmark's autotuner: phi of every instance after steps
  1 and 5 (s = 10) against the oracle at 256 sample nodes per instance
  (tests/golden/batch64_trajectory.txt, written by
  tests/golden/make_batch64_trajectory.py).

Bar: the mixed path's 1e-6 relative L2 error on phi (max over the stored
steps of ||phi - phi_oracle|| over max of ||phi_oracle||), per column and
per instance.
"""
import os

import numpy as np
import pytest

import eqs_inputs as ei

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ENS_GOLDEN = os.path.join(HERE, "golden", "cube128_ensemble_trajectory.txt")
BATCH_GOLDEN = os.path.join(HERE, "golden", "batch64_trajectory.txt")
# bench.py's solver options and batched-serving candidates
BENCH_OPTS = dict(cheb_degree=1, coarse_max=2500, persistent=0, coarse_split=0, defer_sums=2)
BATCH_CANDIDATES = (256, 512, 1024, 2048)
RTOL = 1e-8
TOL = 1e-6


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_09447_gb300 import build, eqs
    if not os.path.exists(build.LIB):
        build.build()
    return eqs


def _header(path):
    h = {}
    with open(path) as f:
        for line in f:
            if not line.startswith("#"):
                break
            parts = line[1:].split()
            if len(parts) >= 2:
                h[parts[0]] = parts[1:]
    return h


def _rel(got, ref):
    """max over steps of ||got - ref|| / max over steps of ||ref|| (rows: steps)."""
    return np.linalg.norm(got - ref, axis=1).max() / np.linalg.norm(ref, axis=1).max()


@pytest.fixture(scope="module")
def ens_golden():
    if not os.path.exists(ENS_GOLDEN):
        pytest.skip("tests/golden/cube128_ensemble_trajectory.txt not written yet")
    h = _header(ENS_GOLDEN)
    steps = [int(v) for v in h["steps"]]
    scales = [float(v) for v in h["scales"]]
    data = np.loadtxt(ENS_GOLDEN, comments="#")
    nodes = data[:, 0].astype(np.int64)
    phi = data[:, 1:].reshape(len(nodes), len(scales), len(steps))
    return {"N": int(h["N"][0]), "s": int(h["s"][0]), "dt": float(h["dt"][0]), "steps": steps,
            "scales": scales, "nodes": nodes, "phi": phi}


def test_ensemble_full_size_vs_oracle(E, ens_golden):
    g = ens_golden
    p = ei.config_problem(2, N=g["N"])
    S = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=RTOL, spe_n=6, **BENCH_OPTS)
    E.eqs_set_guess(S.ctx, E.EQS_GUESS_SPE)
    assert abs(S.dt_bound(g["s"]) - g["dt"]) <= 1e-12 * g["dt"]
    x = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    got = {}
    t = 0.0
    for k in range(1, max(g["steps"]) + 1):
        st = E.eqs_ens_rkc_step(S.ctx, x, g["scales"], t, g["dt"], g["s"])
        assert st.status == 0 and st.max_relres <= RTOL
        t += g["dt"]
        if k in g["steps"]:
            got[k] = x[:, torch.as_tensor(g["nodes"], device="cuda")].cpu().numpy()
    S.close()
    for c, sc in enumerate(g["scales"]):
        mine = np.stack([got[k][c] for k in g["steps"]])
        ref = g["phi"][:, c, :].T
        err = _rel(mine, ref)
        assert err <= TOL, (sc, err)


def test_single_trajectory_full_size_vs_oracle(E, ens_golden):
    g = ens_golden
    c = g["scales"].index(1.0)
    p = ei.config_problem(2, N=g["N"])
    S = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=RTOL, spe_n=6, **BENCH_OPTS)
    E.eqs_set_guess(S.ctx, E.EQS_GUESS_SPE)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    idx = torch.as_tensor(g["nodes"], device="cuda")
    got = []
    t = 0.0
    for k in range(1, max(g["steps"]) + 1):
        st = S.step(x, t, g["dt"], g["s"])
        assert st.status == 0
        t += g["dt"]
        if k in g["steps"]:
            got.append(x[idx].cpu().numpy())
    S.close()
    err = _rel(np.stack(got), g["phi"][:, c, :].T)
    assert err <= TOL, err


@pytest.fixture(scope="module")
def batch_golden():
    h = _header(BATCH_GOLDEN)
    data = np.loadtxt(BATCH_GOLDEN, comments="#")
    steps = [int(v) for v in h["steps"]]
    inst = data[:, 0].astype(np.int64)
    out = {}
    for i in np.unique(inst):
        rows = data[inst == i]
        out[int(i)] = {"N": int(rows[0, 1]), "nodes": rows[:, 2].astype(np.int64), "phi": rows[:, 3:]}
    return {"s": int(h["s"][0]), "dt": float(h["dt"][0]), "steps": steps, "inst": out}


@pytest.fixture(scope="module")
def batch_solvers(E, batch_golden):
    probs = [ei.config_problem(4, instance=i) for i in sorted(batch_golden["inst"])]
    for i, p in enumerate(probs):
        assert p.N == batch_golden["inst"][i]["N"]
    solvers = [E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=RTOL, fill_lanes=0, **BENCH_OPTS) for p in probs]
    yield probs, solvers
    for S in solvers:
        S.close()


@pytest.mark.parametrize("rows_per_block", BATCH_CANDIDATES)
def test_batch_full_size_vs_oracle(E, batch_golden, batch_solvers, rows_per_block):
    g = batch_golden
    probs, solvers = batch_solvers
    b = E.eqs_batch_create([S.ctx for S in solvers], rows_per_block)
    xs = [torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda") for p in probs]
    idx = [torch.as_tensor(g["inst"][i]["nodes"], device="cuda") for i in range(len(probs))]
    got = {i: [] for i in range(len(probs))}
    t = 0.0
    for k in range(1, max(g["steps"]) + 1):
        st = E.eqs_batch_rkc_step(b, xs, t, g["dt"], g["s"])
        assert st.status == 0 and st.max_relres <= RTOL
        t += g["dt"]
        if k in g["steps"]:
            for i in range(len(probs)):
                got[i].append(xs[i][idx[i]].cpu().numpy())
    E.eqs_batch_destroy(b)
    errs = [_rel(np.stack(got[i]), g["inst"][i]["phi"].T) for i in range(len(probs))]
    worst = int(np.argmax(errs))
    assert max(errs) <= TOL, (worst, probs[worst].N, errs[worst])
