"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (solver options of bench.py, CUDA-graph CG loop).

Workloads: the 64^3-cell block cube (274,625 nodes, 1,572,864 tets) and the
128^3-cell jittered cube with two varistor spheres (2,146,689 nodes,
12,582,912 tets).  The oracle cannot redo whole passes at these sizes in a
test, so it checks

* K(x)x (Section III) on 4096 seeded sample nodes, computed one by one from
  every tet that touches a sampled node (that is all of the node's terms);
* the M-solve (Section II) through a property that holds at any size: the
  residual R - M z of a sampled row, with M's row built by the oracle from
  the tets around the node, is bounded by the solver's stopping test
  ||R - M z||_2 <= rtol ||R||_2;
* phi after 50 and 100 RKC steps of s = 20 (Section II) on the 64^3 cube
  against the oracle's FP64 trajectory at 8192 sample nodes
  (tests/golden/cube64_block_trajectory.txt, written by
  tests/golden/make_cube64_trajectory.py).
"""
import os

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1
# bench.py's solver options
BENCH_OPTS = dict(cheb_degree=1, coarse_max=2500, persistent=0, coarse_split=0, defer_sums=2)
CASES = {"cube64": 1, "jitter128": 2}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cube64_block_trajectory.txt")
_PROBLEMS = {}


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_09447_gb300 import build, eqs
    if not os.path.exists(build.LIB):
        build.build()
    return eqs


def _problem(name):
    if name not in _PROBLEMS:
        _PROBLEMS[name] = ei.config_problem(CASES[name])
    return _PROBLEMS[name]


def _cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _sample(n, count, seed):
    return np.sort(np.random.default_rng(seed).choice(n, count, replace=False))


def _around(p, nodes):
    """The tets that touch any of the given nodes."""
    return np.isin(p.tets, nodes).any(axis=1)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (MIXED, 2e-5)])
def test_apply_K_full_size_sampled(E, name, prec, tol):
    p = _problem(name)
    rng = np.random.default_rng(21)
    Emag = 5.2e5  # a field in the varistor's switching range, plus noise
    x = -Emag * p.xyz[:, 2] + 0.3 * Emag * (0.1 / p.N) * rng.standard_normal(p.n_nodes)
    S = E.Solver(p, precision=prec, **BENCH_OPTS)
    got = S.apply_K(_cuda(x)).cpu().numpy()
    S.close()
    nodes = _sample(p.n_nodes, 4096, seed=22)
    sub = _around(p, nodes)
    ref = fem.apply_K(p.xyz, p.tets[sub], p.tet_mat[sub], p.materials, x)[nodes]
    assert np.abs(got[nodes] - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("name,prec", [("cube64", FP64), ("cube64", MIXED), ("jitter128", MIXED)])
def test_solve_M_full_size_sampled_residual(E, name, prec):
    p = _problem(name)
    free = np.nonzero(p.node_tag == 0)[0]  # internal order of the solver's vectors
    R = np.random.default_rng(23).standard_normal(p.n_free)
    rtol = 1e-8
    S = E.Solver(p, precision=prec, rtol=rtol, **BENCH_OPTS)
    z, iters = S.solve_M(_cuda(R), rtol=rtol)
    S.close()
    assert 0 < iters[0] < 500
    rows = _sample(p.n_free, 4096, seed=24)
    nodes = free[rows]
    sub = _around(p, nodes)
    Msub = fem.assemble_M(p.xyz, p.tets[sub], p.tet_mat[sub], p.materials)
    zfull = np.zeros(p.n_nodes)
    zfull[free] = z.cpu().numpy()  # Dirichlet columns are not part of M_ff
    res = R[rows] - (Msub @ zfull)[nodes]
    # every row of the residual is bounded by its 2-norm, which the stopping
    # test holds below rtol ||R|| (slack for the recursively updated residual)
    assert np.abs(res).max() <= 1.5 * rtol * np.linalg.norm(R)


def _golden():
    meta, rows = {}, []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#"):
                parts = line[1:].split()
                if len(parts) >= 2 and parts[0] in ("s", "dt", "steps", "sample_seed", "n_sample"):
                    meta[parts[0]] = parts[1:]
                continue
            rows.append([float(v) for v in line.split()])
    a = np.array(rows)
    return meta, a[:, 0].astype(np.int64), a[:, 1:]


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="oracle trajectory not generated")
@pytest.mark.parametrize("prec,guess,rtol,tol", [(MIXED, "spe", 1e-8, 1e-6), (FP64, "spe", 1e-13, 1e-10)])
def test_trajectory_full_size_vs_oracle(E, prec, guess, rtol, tol):
    """phi after 50 and 100 steps (s = 20, dt at the stability bound) of the
    64^3 block cube against the oracle's FP64 run, relative L2 over the 8192
    sample nodes.  The mixed form runs exactly as the benchmark times it
    (SPE start vectors, M-solves to 1e-8)."""
    meta, nodes, ref = _golden()
    p = _problem("cube64")
    s, dt = int(meta["s"][0]), float(meta["dt"][0])
    keep = [int(k) for k in meta["steps"]]
    S = E.Solver(p, precision=prec, rtol=rtol, spe_n=6, **BENCH_OPTS)
    E.eqs_set_guess(S.ctx, E.EQS_GUESS_SPE if guess == "spe" else E.EQS_GUESS_PREV)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    t, errs = 0.0, []
    for k in range(1, max(keep) + 1):
        S.step(x, t, dt, s, stats=False)
        t += dt
        if k in keep:
            got = x.cpu().numpy()[nodes]
            col = ref[:, keep.index(k)]
            errs.append(float(np.linalg.norm(got - col) / np.linalg.norm(col)))
    S.close()
    print(f"relative L2 error on phi (sample of {len(nodes)} nodes) after steps {keep}: {errs}")
    assert max(errs) <= tol
