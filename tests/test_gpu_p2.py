"""Quadratic (P2) elements (Section V's 2nd order ansatz functions) on the
GPU against the oracle."""
import os

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import fem, rkc, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


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


PROBLEMS = {
    "p2_cube4": lambda: ei.make_problem_p2(4),
    "p2_jitter3": lambda: ei.make_problem_p2(3, jitter=0.2, seed=7),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (MIXED, 2e-5)])
def test_apply_K_p2(E, name, prec, tol):
    p = PROBLEMS[name]()
    S = E.Solver(p, precision=prec)
    rng = np.random.default_rng(0)
    for Emag in (5e4, 5.2e5):  # below and in the varistor switching range
        x = -Emag * p.xyz[:, 2] + 0.3 * Emag * (0.1 / p.N) * rng.standard_normal(p.n_nodes)
        got = S.apply_K(_cuda(x)).cpu().numpy()
        ref = fem.apply_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    S.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_spmv_M_p2(E, name):
    p = PROBLEMS[name]()
    S = E.Solver(p)
    Sy = system.EQSSystem(p)
    x = np.random.default_rng(3).standard_normal(p.n_free)
    got = S.spmv_M(_cuda(x)).cpu().numpy()
    ref = Sy.Mff @ x
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    S.close()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6)])
@pytest.mark.parametrize("guess", [0, 3])
def test_rkc_trajectory_p2(E, prec, tol, guess):
    p = ei.make_problem_p2(4)
    s, steps = 10, 5
    S = E.Solver(p, precision=prec, rtol=1e-13)
    E.eqs_set_guess(S.ctx, guess)
    dt = S.dt_bound(s)
    Sy = system.EQSSystem(p)
    coef = rkc.RKCCoefficients(s)
    xf, t, ref = np.zeros(p.n_free), 0.0, []
    for _ in range(steps):
        xf, _ = rkc.rkc_step(Sy.F, t, xf, dt, coef)
        t += dt
        ref.append(Sy.full(t, xf))
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    got, t = [], 0.0
    for _ in range(steps):
        st = S.step(x, t, dt, s)
        assert st.status == 0
        t += dt
        got.append(x.cpu().numpy())
    ref, got = np.array(ref), np.array(got)
    err = np.linalg.norm(got - ref, axis=1).max() / np.linalg.norm(ref, axis=1).max()
    assert err <= tol, err
    S.close()


def test_p2_rejected_by_ensemble(E):
    p = ei.make_problem_p2(2)
    S = E.Solver(p, precision=MIXED)
    x = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    with pytest.raises(E.EqsError) as ex:
        E.eqs_ens_rkc_step(S.ctx, x, (1.0, 1.0, 1.0, 1.0), 0.0, 1e-3, 10)
    assert ex.value.status == E.EQS_ERR_STATE
    S.close()
