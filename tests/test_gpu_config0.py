"""The whole 200-step run of the 12^3-cell block cube (2,197 nodes, 1,859
free, s = 10, dt at the stability bound) through the C ABI against the
oracle's FP64 trajectory (tests/golden/cube12_block_trajectory.txt, written
by tests/golden/make_cube12_trajectory.py): phi at every node after steps
1, 50, 100 and 200 of the RKC scheme (Section II) with each stage's M-solve
(Section II, start vectors of Section IV)."""
import os

import numpy as np
import pytest

import eqs_inputs as ei

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cube12_block_trajectory.txt")


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_09447_gb300 import build, eqs
    if not os.path.exists(build.LIB):
        build.build()
    return eqs


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
    a = np.array(rows)
    return meta, a[:, 0].astype(np.int64), a[:, 1:]


# (precision, start vector, M-solve tolerance, bound on the relative L2
# error of phi): the FP64 forms solve to 1e-13 like the oracle; the mixed
# form runs as it is timed (degree-1 smoother, SPE, M-solves to 1e-8)
FORMS = [
    (FP64, "prev", 1e-13, 1e-10, {}),
    (FP64, "spe", 1e-13, 1e-10, {}),
    (MIXED, "spe", 1e-8, 1e-6, dict(cheb_degree=1, coarse_max=60, defer_sums=2)),
    (MIXED, "prev", 1e-13, 1e-6, {}),
]


@pytest.mark.parametrize("prec,guess,rtol,tol,opts", FORMS)
def test_config0_200_steps_vs_oracle(E, prec, guess, rtol, tol, opts):
    meta, nodes, ref = _golden()
    p = ei.config_problem(0)
    assert len(nodes) == p.n_nodes
    s, dt = int(meta["s"][0]), float(meta["dt"][0])
    keep = [int(k) for k in meta["steps"]]
    S = E.Solver(p, precision=prec, rtol=rtol, spe_n=6, **opts)
    assert abs(S.dt_bound(s) - dt) <= 1e-14 * dt
    E.eqs_set_guess(S.ctx, E.EQS_GUESS_SPE if guess == "spe" else E.EQS_GUESS_PREV)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    t, errs = 0.0, []
    for k in range(1, max(keep) + 1):
        st = S.step(x, t, dt, s)
        assert st.status == 0
        assert st.max_relres <= rtol
        t += dt
        if k in keep:
            got = x.cpu().numpy()
            col = ref[:, keep.index(k)]
            errs.append(float(np.linalg.norm(got - col) / np.linalg.norm(col)))
    S.close()
    print(f"relative L2 error on phi after steps {keep}: {errs}")
    assert max(errs) <= tol
