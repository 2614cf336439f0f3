"""Four-trajectory ensemble (blocked multiple right-hand-side solves,
Section IV) on the GPU: each column against its own solo run and the oracle."""
import dataclasses
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import eqs_inputs as ei
from oracle import rkc, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1
SCALES = (0.5, 1.0, 1.5, 2.0)


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_09447_gb300 import build, eqs
    if not os.path.exists(build.LIB):
        build.build()
    return eqs


def _oracle_run(p, s, steps, dt):
    Sy = system.EQSSystem(p)
    coef = rkc.RKCCoefficients(s)
    xf, t, out = np.zeros(p.n_free), 0.0, []
    for _ in range(steps):
        xf, _ = rkc.rkc_step(Sy.F, t, xf, dt, coef)
        t += dt
        out.append(Sy.full(t, xf))
    return np.array(out)


def _ens_run(E, p, scales, s, steps, rtol, host_loop=0, guess=0):
    S = E.Solver(p, precision=MIXED, rtol=rtol, persistent=0, host_loop=host_loop)
    E.eqs_set_guess(S.ctx, guess)
    dt = S.dt_bound(s)
    x = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    traj, stats, t = [], [], 0.0
    for _ in range(steps):
        st = E.eqs_ens_rkc_step(S.ctx, x, scales, t, dt, s)
        stats.append(st)
        t += dt
        traj.append(x.cpu().numpy().copy())
    S.close()
    return np.array(traj), stats, dt


def _err(a, b):
    return np.linalg.norm(a - b, axis=-1).max() / np.linalg.norm(b, axis=-1).max()


@pytest.mark.parametrize("name,V0,steps", [("cube12", 1e4, 8), ("jitter10", 2e5, 4)])
def test_ensemble_matches_solo_and_oracle(E, name, V0, steps):
    """Every column equals its own single-trajectory run (drive V0 * scale)
    and the FP64 oracle; V0 = 2e5 drives the varistor into switching, so
    the columns see different conductivities."""
    p0 = ei.config_problem(0) if name == "cube12" else ei.config_problem(2, N=10)
    p = dataclasses.replace(p0, V0=V0)
    s = 10
    traj, stats, dt = _ens_run(E, p, SCALES, s, steps, rtol=1e-12)
    for st in stats:
        assert st.status == 0 and st.max_relres <= 1e-12
        assert st.passes >= max(st.total_iters) // s
    for c, sc in enumerate(SCALES):
        pc = dataclasses.replace(p, V0=V0 * sc)
        solo = E.Solver(pc, precision=MIXED, rtol=1e-12, persistent=0)
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        got, t = [], 0.0
        for _ in range(steps):
            solo.step(x, t, dt, s)
            t += dt
            got.append(x.cpu().numpy())
        solo.close()
        assert _err(traj[:, c], np.array(got)) <= 1e-7, c
        ref = _oracle_run(pc, s, steps, dt)
        assert _err(traj[:, c], ref) <= 1e-6, c


def test_ensemble_zero_column_and_counts(E):
    """A column with zero drive stays exactly zero (its right-hand sides are
    zero: no iterations) while the others iterate; per-column counts add up."""
    p = ei.config_problem(0)
    traj, stats, _ = _ens_run(E, p, (0.0, 1.0, 2.0, 0.0), 10, 3, rtol=1e-10)
    assert not traj[:, 0].any() and not traj[:, 3].any()
    assert np.abs(traj[:, 1]).max() > 0
    for st in stats:
        assert st.total_iters[0] == 0 and st.total_iters[3] == 0
        assert st.total_iters[1] > 0 and st.total_iters[2] > 0
        assert st.passes >= max(st.total_iters) // st.s
        assert st.launches > 0


def test_ensemble_host_loop_matches_graph(E):
    p = ei.config_problem(2, N=10)
    a, sa, _ = _ens_run(E, p, SCALES, 10, 3, rtol=1e-10, host_loop=0)
    b, sb, _ = _ens_run(E, p, SCALES, 10, 3, rtol=1e-10, host_loop=1)
    assert [list(x.total_iters) for x in sa] == [list(x.total_iters) for x in sb]
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-7 * np.abs(a).max())


def test_ensemble_solve_blocked(E):
    """eqs_ens_solve_M: four right-hand sides at once, each column as the
    direct solve; the per-column iteration counts match single solves."""
    p = ei.config_problem(2, N=10)
    S = E.Solver(p, precision=MIXED, rtol=1e-10, persistent=0)
    Sy = system.EQSSystem(p)
    rng = np.random.default_rng(7)
    R = rng.standard_normal((4, p.n_free))
    R[2] *= 1e-3  # columns of very different size converge independently
    rhs = torch.tensor(R, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(rhs)
    its = E.eqs_ens_solve_M(S.ctx, rhs, z)
    zs = z.cpu().numpy()
    for c in range(4):
        zd = spla.spsolve(Sy.Mff.tocsc(), R[c])
        assert np.linalg.norm(zs[c] - zd) / np.linalg.norm(zd) <= 1e-7
        assert np.linalg.norm(R[c] - Sy.Mff @ zs[c]) / np.linalg.norm(R[c]) <= 2e-10
        _, it1 = S.solve_M(torch.tensor(R[c], device="cuda"), rtol=1e-10)
        assert abs(its[c] - it1[0]) <= 1, (c, its, it1)
    S.close()


def test_ensemble_requires_mixed(E):
    p = ei.make_problem(3)
    S = E.Solver(p, precision=FP64)
    x = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    with pytest.raises(E.EqsError) as ex:
        E.eqs_ens_rkc_step(S.ctx, x, SCALES, 0.0, 1e-3, 10)
    assert ex.value.status == E.EQS_ERR_STATE
    S.close()


def test_ensemble_spe_start(E):
    """Per-column SPE start vectors (Section IV, Eq. 4-5) in the ensemble:
    same trajectories as the oracle, far fewer CG iterations than starting
    from the previous solutions."""
    p = ei.config_problem(0)
    s, steps = 10, 6
    a, sa, dt = _ens_run(E, p, SCALES, s, steps, rtol=1e-12, guess=E.EQS_GUESS_PREV)
    b, sb, _ = _ens_run(E, p, SCALES, s, steps, rtol=1e-12, guess=E.EQS_GUESS_SPE)
    for c, sc in enumerate(SCALES):
        ref = _oracle_run(dataclasses.replace(p, V0=p.V0 * sc), s, steps, dt)
        assert _err(b[:, c], ref) <= 1e-6, c
    it_prev = [sum(st.total_iters[c] for st in sa[2:]) for c in range(4)]
    it_spe = [sum(st.total_iters[c] for st in sb[2:]) for c in range(4)]
    print("ensemble iterations per column, previous solution", it_prev, "SPE", it_spe)
    for c in range(4):
        assert it_spe[c] * 1.5 < it_prev[c]
    for st in sb:
        assert st.status == 0 and st.max_relres <= 1e-12


def test_ensemble_rejects_other_guess_modes(E):
    p = ei.make_problem(3)
    S = E.Solver(p, precision=MIXED)
    E.eqs_set_guess(S.ctx, E.EQS_GUESS_POD)
    x = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    with pytest.raises(E.EqsError) as ex:
        E.eqs_ens_rkc_step(S.ctx, x, SCALES, 0.0, 1e-3, 10)
    assert ex.value.status == E.EQS_ERR_STATE
    S.close()


def test_ensemble_cell_and_tet_element_paths_agree(E):
    """Kuhn-ordered tets take the four-column cell kernel; shuffled tets the
    per-tet kernel: the trajectories agree."""
    p = ei.config_problem(2, N=6)
    perm = np.random.default_rng(2).permutation(p.n_tets)
    q = ei.Problem(p.N, p.xyz, p.tets[perm], p.tet_mat[perm], p.node_tag, p.materials, p.V0)
    a, _, _ = _ens_run(E, p, SCALES, 10, 2, rtol=1e-12)
    b, _, _ = _ens_run(E, q, SCALES, 10, 2, rtol=1e-12)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-7 * np.abs(a).max())


def test_ensemble_spe_start_matches_oracle_and_true_residual(E):
    """The ensemble's SPE start (Eq. 4-5) from a given six-solution history:
    x0 of every column against the oracle's projection, and the start
    residual b - W y that the CG begins from against the true b - M x0
    (W = M X comes from the Gram pass's FP32-pair products).  The history
    carries a large constant offset: M is Laplace-type, so M x cancels to a
    tiny fraction of sum |m_ij x_j|; the start residual must still agree
    with the FP64 product to about FP64 rounding."""
    from oracle import spe

    p = ei.config_problem(2, N=12)
    S = E.Solver(p, precision=MIXED, rtol=1e-10)
    Sy = system.EQSSystem(p)
    xyz = p.xyz[Sy.free]
    nf = p.n_free
    hist = np.empty((6, 4, nf))
    for k in range(6):
        for c in range(4):
            w = 2 * np.pi / 0.1 * (1 + 0.3 * c)
            hist[k, c] = (1e3 * (1 + c) + 40 * np.sin(w * xyz[:, 0] + 0.2 * k) * np.cos(w * xyz[:, 1])
                          + 25 * (1 + 0.1 * k) * np.sin(w * xyz[:, 2] * 0.5 + c))
    coef = np.array([1.9, -1.2, 0.5, -0.2, 0.05, -0.01])
    rng = np.random.default_rng(4)
    b = np.stack([Sy.Mff @ (np.tensordot(coef, hist[:, c], 1) + 5 * np.sin(9 * xyz[:, 0] / 0.1)
                            + 0.5 * rng.standard_normal(nf)) for c in range(4)])
    X = torch.tensor(hist, dtype=torch.float64, device="cuda")
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    x0 = torch.empty((4, nf), dtype=torch.float64, device="cuda")
    r0 = torch.empty_like(x0)
    E.eqs_ens_spe_eval(S.ctx, X, bd, x0, r0)
    x0, r0 = x0.cpu().numpy(), r0.cpu().numpy()
    for c in range(4):
        ref = spe.spe_start(Sy.Mff, [hist[k, c] for k in range(6)], b[c])
        assert np.linalg.norm(x0[c] - ref) <= 1e-7 * np.linalg.norm(ref), c
        true_r = b[c] - Sy.Mff @ x0[c]
        assert np.linalg.norm(r0[c] - true_r) <= 1e-11 * np.linalg.norm(b[c]), c
    S.close()


def _field_state(p, seed):
    """A potential whose field reaches the varistor switching range."""
    rng = np.random.default_rng(seed)
    Emag = 5.2e5
    return -Emag * p.xyz[:, 2] + 0.3 * Emag * (0.1 / p.N) * rng.standard_normal(p.n_nodes)


def _shuffled(p, seed=1):
    perm = np.random.default_rng(seed).permutation(p.n_tets)
    return ei.Problem(p.N, p.xyz, p.tets[perm], p.tet_mat[perm], p.node_tag, p.materials, p.V0)


@pytest.mark.parametrize("name", ["cube12", "jitter10", "batch7", "jitter6_shuffled"])
def test_ens_apply_K_matches_oracle(E, name):
    """The ensemble's four-column element kernel (Section III) through
    eqs_ens_apply_K: every column equals the oracle's K(x)x to the mixed
    tolerance of the single-column kernel, on Kuhn-cell meshes (cell kernel)
    and on a mesh with its tets shuffled (per-tet kernel), with fields that
    span the varistor's switching range (drive scales 0.5 to 2), on two
    calls in a row."""
    from oracle import fem

    p = {"cube12": lambda: ei.config_problem(0), "jitter10": lambda: ei.config_problem(2, N=10),
         "batch7": lambda: ei.config_problem(4, N=7, instance=3),
         "jitter6_shuffled": lambda: _shuffled(ei.config_problem(2, N=6))}[name]()
    S = E.Solver(p, precision=MIXED)
    cols = [sc * _field_state(p, seed=k) for k, sc in enumerate(SCALES)]
    X = torch.tensor(np.stack(cols), dtype=torch.float64, device="cuda")
    for _ in range(2):
        Y = torch.full_like(X, np.nan)
        E.eqs_ens_apply_K(S.ctx, X, Y)
        got = Y.cpu().numpy()
        for k, x in enumerate(cols):
            ref = fem.apply_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
            assert np.abs(got[k] - ref).max() <= 2e-5 * np.abs(ref).max(), (name, k)
    S.close()


def test_ens_apply_K_needs_mixed_linear(E):
    p = ei.config_problem(0)
    S = E.Solver(p, precision=FP64)
    X = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    with pytest.raises(E.EqsError) as ei_:
        E.eqs_ens_apply_K(S.ctx, X, torch.empty_like(X))
    assert ei_.value.status == E.EQS_ERR_STATE
    S.close()
