"""POD-MOR start vectors (Section IV) on the GPU against the oracle."""
import os

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import pcg, pod, rkc, system

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


@pytest.mark.parametrize("K,m", [(8, 3), (8, 8), (12, 5), (1, 1)])
def test_pod_projection_matches_oracle(E, K, m):
    """Gram matrices + device Jacobi eigendecomposition give the oracle's
    SVD-based basis: same eigenvalues (squared singular values), same x0."""
    p = ei.config_problem(2, N=10)
    Sy = system.EQSSystem(p)
    S = E.Solver(p, pod_k=12, pod_m=m)
    rng = np.random.default_rng(K + 10 * m)
    base = np.sin(np.linspace(0, 7, p.n_free))
    # snapshots with well separated singular values
    X = np.stack([base * (1 + 0.2 * k) + (0.5 ** k) * rng.standard_normal(p.n_free) for k in range(K)], axis=1)
    b = Sy.Mff @ (0.6 * X[:, -1] + 0.1 * rng.standard_normal(p.n_free))
    x0 = torch.empty(p.n_free, dtype=torch.float64, device="cuda")
    E.eqs_pod_eval(S.ctx, _cuda(X.T), K, _cuda(b), x0)
    V, sig = pod.pod_basis(X, m, drop=1e-7)
    ref = pod.pod_start(Sy.Mff, V, b)
    got = x0.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    S.close()


def test_pod_eigenvalues_match_singular_values(E):
    """The device Jacobi eigenvalues of X^T X are the squared singular values
    of the snapshot matrix (oracle: LAPACK SVD)."""
    p = ei.config_problem(2, N=10)
    S = E.Solver(p, pod_k=10, pod_m=10)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((p.n_free, 10)) * (2.0 ** -np.arange(10))
    x0 = torch.empty(p.n_free, dtype=torch.float64, device="cuda")
    E.eqs_pod_eval(S.ctx, _cuda(X.T), 10, _cuda(np.ones(p.n_free)), x0)
    info = E.eqs_pod_info(S.ctx)
    S.close()
    assert info["count"] == 10 and info["modes"] == 10 and info["rebuilds"] == 1
    _, sig = pod.pod_basis(X, 10)
    np.testing.assert_allclose(info["lam"][:10], sig ** 2, rtol=1e-9)


def _run(E, p, prec, guess, s, steps, rtol, **opt):
    S = E.Solver(p, precision=prec, rtol=rtol, **opt)
    E.eqs_set_guess(S.ctx, guess)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    dt, t, its, traj = S.dt_bound(s), 0.0, [], []
    for _ in range(steps):
        st = S.step(x, t, dt, s)
        its.append(st.total_iters)
        t += dt
        traj.append(x.cpu().numpy())
    info = E.eqs_pod_info(S.ctx)
    S.close()
    return np.array(traj), its, info, dt


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6)])
def test_pod_trajectories_and_iterations(E, prec, tol):
    """The start vector changes iteration counts, never the converged
    trajectory; both POD rules beat the previous-solution start."""
    p = ei.config_problem(0)
    s, steps = 10, 8
    ref = None
    runs = {}
    for guess in (E.EQS_GUESS_PREV, E.EQS_GUESS_POD, E.EQS_GUESS_POD2):
        traj, its, info, dt = _run(E, p, prec, guess, s, steps, 1e-13, pod_k=12, pod_m=6, pod_min_iters=3)
        runs[guess] = (traj, its, info)
    Sy = system.EQSSystem(p)
    coef = rkc.RKCCoefficients(s)
    xf, t, ref = np.zeros(p.n_free), 0.0, []
    for _ in range(steps):
        xf, _ = rkc.rkc_step(Sy.F, t, xf, dt, coef)
        t += dt
        ref.append(Sy.full(t, xf))
    ref = np.array(ref)
    for guess, (traj, its, info) in runs.items():
        err = np.linalg.norm(traj - ref, axis=1).max() / np.linalg.norm(ref, axis=1).max()
        assert err <= tol, (guess, err)
    prev = sum(runs[E.EQS_GUESS_PREV][1][3:])
    for guess in (E.EQS_GUESS_POD, E.EQS_GUESS_POD2):
        print(guess, sum(runs[guess][1][3:]), "vs", prev)
        assert sum(runs[guess][1][3:]) * 1.3 < prev
    mor = runs[E.EQS_GUESS_POD][2]
    assert mor["count"] == 12 and mor["rebuilds"] == 1 and mor["adds"] == 12
    mor2 = runs[E.EQS_GUESS_POD2][2]
    assert mor2["rebuilds"] == mor2["adds"] >= 1 and mor2["count"] == min(12, mor2["adds"])


def test_mor2_adds_only_above_threshold(E):
    """With a threshold above every iteration count nothing is added and the
    start vector stays the previous solution (same counts as PREV)."""
    p = ei.config_problem(0)
    a = _run(E, p, 0, E.EQS_GUESS_PREV, 10, 3, 1e-10)
    b = _run(E, p, 0, E.EQS_GUESS_POD2, 10, 3, 1e-10, pod_min_iters=10000)
    assert b[2]["adds"] == 0 and b[2]["rebuilds"] == 0
    assert a[1] == b[1]
