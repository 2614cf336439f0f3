"""Learned start vector on the GPU against the oracle, and its effect."""
import os

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import mlp, rkc, system

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


def _theta(seed=5):
    th = ei.mlp_init(seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    th[256:288] = 0.1 * rng.standard_normal(32)
    th[1312:1344] = 0.1 * rng.standard_normal(32)
    th[1344:1376] = 0.3 * rng.standard_normal(32)
    th[1376] = 0.05
    return th.astype(np.float32)


def test_guess_eval_matches_oracle(E):
    p = ei.config_problem(2, N=10)
    S = E.Solver(p)
    Sy = system.EQSSystem(p)
    A = mlp.free_adjacency(p.tets, Sy.free, p.n_nodes)
    th = _theta()
    E.eqs_guess_set_params(S.ctx, th)
    rng = np.random.default_rng(3)
    base = np.sin(np.linspace(0, 6, p.n_free))
    H = [base * (1 + 0.1 * k) + 0.05 * rng.standard_normal(p.n_free) for k in range(4)]
    Hd = torch.tensor(np.concatenate(H), dtype=torch.float64, device="cuda")
    z0 = torch.empty(p.n_free, dtype=torch.float64, device="cuda")
    E.eqs_guess_eval(S.ctx, Hd, z0)
    got = z0.cpu().numpy() - H[0]
    ref = mlp.guess(th, A, H) - H[0]
    assert np.abs(ref).max() > 1e-3
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    S.close()


def test_guess_gradient_matches_oracle(E):
    p = ei.make_problem(3)
    S = E.Solver(p)
    th = _theta(7)
    E.eqs_guess_set_params(S.ctx, th)
    rng = np.random.default_rng(4)
    B = 1000  # spans several training blocks and a ragged tail
    X = rng.standard_normal((B, 8)).astype(np.float32)
    T = (0.5 * rng.standard_normal(B)).astype(np.float32)
    g, loss = E.eqs_guess_grad(S.ctx, X, T)
    lref, gref = mlp.loss_and_grad(th, X.astype(np.float64), T.astype(np.float64))
    assert loss == pytest.approx(lref, rel=1e-4)
    assert np.abs(g - gref).max() <= 2e-4 * np.abs(gref).max()
    S.close()


def test_untrained_guess_equals_previous_solution(E):
    """Zero output layer: the MLP mode reproduces the previous-solution mode."""
    p = ei.config_problem(0)
    runs = {}
    for mode in (E.EQS_GUESS_PREV, E.EQS_GUESS_MLP):
        S = E.Solver(p, rtol=1e-10)
        E.eqs_guess_set_params(S.ctx, ei.mlp_init())
        E.eqs_set_guess(S.ctx, mode)
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        dt, t, its = S.dt_bound(10), 0.0, []
        for _ in range(6):
            st = S.step(x, t, dt, 10)
            its.append(st.total_iters)
            t += dt
        runs[mode] = (x.cpu().numpy(), its)
        S.close()
    assert runs[0][1] == runs[1][1]
    np.testing.assert_allclose(runs[1][0], runs[0][0], rtol=0, atol=1e-12 * np.abs(runs[0][0]).max())


def test_trained_guess_gain_and_unchanged_solution(E):
    """Record FP64 stage solutions, train on the GPU, then compare CG
    iterations of the learned guess with the previous-solution guess over the
    same steps; the trajectory must stay on the oracle's."""
    p = ei.config_problem(2, N=16)
    s, n_rec, n_cmp = 10, 12, 6
    S = E.Solver(p, rtol=1e-8)
    dt = S.dt_bound(s)
    E.eqs_guess_set_params(S.ctx, ei.mlp_init())
    E.eqs_guess_record(S.ctx, n_rec * s)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    t = 0.0
    for _ in range(n_rec):
        S.step(x, t, dt, s)
        t += dt
    lf, ll = E.eqs_guess_train(S.ctx, 600, 4096, 2e-3, 12345)
    assert ll < lf
    x_start, t_start = x.clone(), t
    iters = {}
    for mode in (E.EQS_GUESS_PREV, E.EQS_GUESS_MLP):
        E.eqs_guess_record(S.ctx, 0)
        E.eqs_set_guess(S.ctx, mode)
        x.copy_(x_start)
        t = t_start
        tot = 0
        for k in range(n_cmp):
            st = S.step(x, t, dt, s)
            if k > 0:  # the first step starts from the other run's history
                tot += st.total_iters
            t += dt
        iters[mode] = tot
    print(f"CG iterations over {n_cmp - 1} steps: previous-solution guess {iters[0]}, learned guess {iters[1]};"
          f" loss {lf:.3e} -> {ll:.3e}")
    assert iters[1] <= iters[0] * 1.1
    S.close()
