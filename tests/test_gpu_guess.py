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


def test_adam_training_steps_match_oracle(E):
    """Four Adam steps of the GPU training loop (training kernel: forward,
    backward and gradient with BF16 weights, FP32 accumulation; update kernel
    on FP32 master weights) on fixed host mini-batches against the oracle's
    loss_and_grad + adam_step at t = 1..4 in FP64.  Adam normalises each
    component by its own gradient history, so a component whose gradient is
    tiny can move by up to lr either way on FP32-level differences; those
    (below 1e-3 of the step's largest gradient) are left out of the bound."""
    p = ei.make_problem(3)
    S = E.Solver(p)
    th0 = _theta(9)
    E.eqs_guess_set_params(S.ctx, th0)
    rng = np.random.default_rng(8)
    nb, B, lr = 4, 777, 2e-3
    X = rng.standard_normal((nb, B, 8)).astype(np.float32)
    T = (0.5 * rng.standard_normal((nb, B))).astype(np.float32)
    losses = E.eqs_guess_train_batches(S.ctx, X, T, lr)
    got = E.eqs_guess_get_params(S.ctx).astype(np.float64)
    th = th0.astype(np.float32).astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    small = np.zeros(th.shape, dtype=bool)
    for k in range(nb):
        lk, g = mlp.loss_and_grad(th, X[k].astype(np.float64), T[k].astype(np.float64))
        assert losses[k] == pytest.approx(lk, rel=2e-4), k
        small |= np.abs(g) < 1e-3 * np.abs(g).max()
        th, m, v = mlp.adam_step(th, g, m, v, k + 1, lr=lr)
    moved = np.abs(th - th0)
    assert np.median(moved[~small]) > 0.5 * lr  # the checked components took real steps
    assert np.abs(got - th)[~small].max() <= 0.02 * lr
    assert np.abs(got - th).max() <= 2.0 * nb * lr
    assert (~small).mean() > 0.8
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
    same steps: the learned guess must take strictly fewer, and both runs
    must stay on the oracle's trajectory (the start vector changes only the
    iteration count; M-solves to 1e-8)."""
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
    # oracle: the same n_rec + n_cmp steps with direct M-solves
    Sy = system.EQSSystem(p)
    coef = rkc.RKCCoefficients(s)
    xf, tt = np.zeros(p.n_free), 0.0
    for _ in range(n_rec + n_cmp):
        xf, _ = rkc.rkc_step(Sy.F, tt, xf, dt, coef)
        tt += dt
    ref = Sy.full(tt, xf)
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
        err = np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-6, (mode, err)
    print(f"CG iterations over {n_cmp - 1} steps: previous-solution guess {iters[0]}, learned guess {iters[1]};"
          f" loss {lf:.3e} -> {ll:.3e}")
    assert iters[1] < iters[0]
    S.close()


def test_spe_correction_eval_matches_oracle(E):
    """The SPE-correction mode's start (network direction from increment
    inputs, 1-ring means, BF16 weights; M-norm line search from x0) against
    the oracle's spe_corrected_start."""
    p = ei.config_problem(2, N=10)
    S = E.Solver(p)
    Sy = system.EQSSystem(p)
    A = mlp.free_adjacency(p.tets, Sy.free, p.n_nodes)
    th = _theta(11)
    E.eqs_guess_set_params(S.ctx, th)
    rng = np.random.default_rng(12)
    base = 1e3 * np.sin(np.linspace(0, 6, p.n_free))
    H = [base * (1 + 0.01 * k) + rng.standard_normal(p.n_free) for k in range(4)]
    x0 = H[0] + 0.5 * (H[0] - H[1]) + 0.1 * rng.standard_normal(p.n_free)
    R = Sy.Mff @ (x0 + 0.3 * (H[0] - H[1]) + 0.05 * rng.standard_normal(p.n_free))
    Hd = torch.tensor(np.concatenate(H), dtype=torch.float64, device="cuda")
    x0d = torch.tensor(x0, dtype=torch.float64, device="cuda")
    Rd = torch.tensor(R, dtype=torch.float64, device="cuda")
    z0 = torch.empty_like(x0d)
    E.eqs_guess_eval_spe(S.ctx, x0d, Hd, Rd, z0)
    got = z0.cpu().numpy() - x0
    zref, alpha = mlp.spe_corrected_start(Sy.Mff, th, A, x0, H, R)
    ref = zref - x0
    assert alpha != 0.0 and np.abs(ref).max() > 1e-6
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    S.close()


def test_spe_correction_never_worse_and_on_trajectory(E):
    """Record mixed-precision SPE steps (each solution's distance from its
    SPE start), train the correction on the GPU, then run SPE alone and SPE
    with the learned direction from the same state with fresh histories.
    The M-norm line search keeps the corrected start at least as close to
    the solution as x0, so the corrected run takes no more CG iterations
    than SPE (to within one iteration per step of count noise), and both
    runs stay on the oracle's trajectory (M-solves to 1e-8)."""
    p = ei.config_problem(2, N=24)
    s, n_rec, n_cmp = 20, 8, 5
    opts = dict(cheb_degree=1, coarse_max=2500, spe_n=6)
    A = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-8, **opts)
    E.eqs_set_guess(A.ctx, E.EQS_GUESS_SPE)
    E.eqs_guess_set_params(A.ctx, ei.mlp_init())
    E.eqs_guess_record(A.ctx, n_rec * s)
    dt = A.dt_bound(s)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    t = 0.0
    for _ in range(n_rec):
        A.step(x, t, dt, s)
        t += dt
    E.eqs_set_guess(A.ctx, E.EQS_GUESS_SPE_MLP)
    lf, ll = E.eqs_guess_train(A.ctx, 1000, 8192, 2e-3, 12345)
    theta = E.eqs_guess_get_params(A.ctx)
    A.close()
    Sy = system.EQSSystem(p)
    coef = rkc.RKCCoefficients(s)
    xf, tt = np.zeros(p.n_free), 0.0
    for _ in range(n_rec + 1 + n_cmp):
        xf, _ = rkc.rkc_step(Sy.F, tt, xf, dt, coef)
        tt += dt
    ref = Sy.full(tt, xf)
    iters, kept = {}, {}
    for mode in (E.EQS_GUESS_SPE, E.EQS_GUESS_SPE_MLP):
        B = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-8, **opts)
        E.eqs_guess_set_params(B.ctx, theta)
        E.eqs_set_guess(B.ctx, mode)
        xb, tb = x.clone(), t
        B.step(xb, tb, dt, s)  # fills the history
        tb += dt
        its = kp = 0
        for _ in range(n_cmp):
            st = B.step(xb, tb, dt, s)
            its += st.total_iters
            kp += st.guess_kept
            tb += dt
        iters[mode], kept[mode] = its, kp
        err = np.linalg.norm(xb.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-6, (mode, err)
        B.close()
    print(f"CG iterations over {n_cmp} steps: SPE {iters[E.EQS_GUESS_SPE]}, SPE + learned direction "
          f"{iters[E.EQS_GUESS_SPE_MLP]} (direction taken in {kept[E.EQS_GUESS_SPE_MLP]} solves); "
          f"loss {lf:.3f} -> {ll:.3f}")
    assert kept[E.EQS_GUESS_SPE_MLP] > 0
    assert iters[E.EQS_GUESS_SPE_MLP] <= iters[E.EQS_GUESS_SPE] + n_cmp
