"""SPE start vector (Section IV, Eq. 4-5) on the GPU against the oracle."""
import os

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import rkc, spe, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_09447_gb300 import build, eqs
    if not os.path.exists(build.LIB):
        build.build()
    return eqs


def _cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n", [1, 4, 6])
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-7)])
def test_spe_projection_matches_oracle(E, n, prec, tol):
    """The device projection (incremental Gram matrix, Cholesky with
    dropping) in both precision modes against the oracle's Gram-Schmidt."""
    p = ei.config_problem(2, N=10)
    Sy = system.EQSSystem(p)
    S = E.Solver(p, spe_n=n, precision=prec)
    rng = np.random.default_rng(n)
    base = np.sin(np.linspace(0, 5, p.n_free))
    H = [base * (1 + 0.3 * k) + 0.2 * rng.standard_normal(p.n_free) for k in range(n)]
    b = Sy.Mff @ (0.7 * H[0] + 0.2 * rng.standard_normal(p.n_free))
    x0 = torch.empty(p.n_free, dtype=torch.float64, device="cuda")
    E.eqs_spe_eval(S.ctx, _cuda(np.concatenate(H)), _cuda(b), n, x0)
    ref = spe.spe_start(Sy.Mff, H, b)
    got = x0.cpu().numpy()
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    S.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6)])
@pytest.mark.parametrize("defer", [0, 3])
def test_spe_trajectory_and_iterations(E, prec, tol, defer):
    """The start vector changes iteration counts, never the converged
    trajectory; SPE needs far fewer CG iterations than the previous solution.
    defer 3: the Gram pass leaves its sums as per-block partials for the
    one-block small solve (and the CG sums are deferred where they apply)."""
    p = ei.config_problem(0)
    s, steps = 10, 8
    res = {}
    for mode in (E.EQS_GUESS_PREV, E.EQS_GUESS_SPE):
        S = E.Solver(p, precision=prec, rtol=1e-13, defer_sums=defer)
        E.eqs_set_guess(S.ctx, mode)
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        dt, t, its, traj = S.dt_bound(s), 0.0, 0, []
        for k in range(steps):
            st = S.step(x, t, dt, s)
            if k >= 2:
                its += st.total_iters
            t += dt
            traj.append(x.cpu().numpy())
        res[mode] = (np.array(traj), its)
        S.close()
    Sy = system.EQSSystem(p)
    coef = rkc.RKCCoefficients(s)
    xf, t, ref = np.zeros(p.n_free), 0.0, []
    for _ in range(steps):
        xf, _ = rkc.rkc_step(Sy.F, t, xf, dt, coef)
        t += dt
        ref.append(Sy.full(t, xf))
    ref = np.array(ref)
    for mode in res:
        err = np.linalg.norm(res[mode][0] - ref, axis=1).max() / np.linalg.norm(ref, axis=1).max()
        assert err <= tol, (mode, err)
    print(f"CG iterations (steps 3-{steps}): previous solution {res[0][1]}, SPE {res[3][1]}")
    assert res[3][1] * 1.5 < res[0][1]
