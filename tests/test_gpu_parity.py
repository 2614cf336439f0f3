"""CUDA path against the CPU oracle, through the C ABI (needs a GPU)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import eqs_inputs as ei
from oracle import amg, fem, pcg, rkc, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_09447_gb300 import build, eqs
    import os
    if not os.path.exists(build.LIB):
        build.build()
    return eqs


PROBLEMS = {
    "cube12": lambda: ei.config_problem(0),                 # 2197 nodes, block varistor
    "jitter10": lambda: ei.config_problem(2, N=10),         # jittered, two spheres, ragged
    "cube2": lambda: ei.make_problem(2),                    # 27 nodes: single-level AMG
    "batch7": lambda: ei.config_problem(4, N=7, instance=3),
}


def _state(p, Emag=5.2e5, seed=0):
    """A potential whose field reaches the varistor switching range."""
    rng = np.random.default_rng(seed)
    return -Emag * p.xyz[:, 2] + 0.3 * Emag * (0.1 / p.N) * rng.standard_normal(p.n_nodes)


def _cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (MIXED, 2e-5)])
def test_apply_K(E, name, prec, tol):
    p = PROBLEMS[name]()
    S = E.Solver(p, precision=prec)
    for seed in (0, 1):
        x = _state(p, seed=seed)
        got = S.apply_K(_cuda(x)).cpu().numpy()
        ref = fem.apply_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
        assert _relmax(got, ref) <= tol
    S.close()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (MIXED, 2e-5)])
def test_apply_K_cell_and_tet_paths_agree(E, prec, tol):
    """Kuhn-ordered tets take the per-cell element kernel; the same mesh with
    its tets shuffled takes the per-tet kernel: both equal the oracle."""
    p = ei.config_problem(2, N=6)
    perm = np.random.default_rng(1).permutation(p.n_tets)
    x = _state(p, seed=4)
    ref = fem.apply_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
    for order in (np.arange(p.n_tets), perm):
        q = ei.Problem(p.N, p.xyz, p.tets[order], p.tet_mat[order], p.node_tag, p.materials, p.V0)
        S = E.Solver(q, precision=prec)
        got = S.apply_K(_cuda(x)).cpu().numpy()
        assert _relmax(got, ref) <= tol
        S.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_spmv_M(E, name):
    p = PROBLEMS[name]()
    S = E.Solver(p)
    Sy = system.EQSSystem(p)
    x = np.random.default_rng(3).standard_normal(p.n_free)
    got = S.spmv_M(_cuda(x)).cpu().numpy()
    assert _relmax(got, Sy.Mff @ x) <= 1e-14
    S.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_spmv_M_split(E, name):
    """The mixed CG operator product (FP32 parts of M, FP32-pair row sums)
    against FP64 M x for FP32 x: every row within 1e-13 of sum |m_ij x_j|,
    far below what an FP32 product would give (about 6e-8)."""
    p = PROBLEMS[name]()
    S = E.Solver(p, precision=MIXED)
    Sy = system.EQSSystem(p)
    rng = np.random.default_rng(5)
    # a smooth field plus noise: strong cancellation in the Laplace rows
    x = (np.sin(np.arange(p.n_free) / 50.0) + 1e-3 * rng.standard_normal(p.n_free)).astype(np.float32)
    y = torch.empty(p.n_free, dtype=torch.float64, device="cuda")
    E.eqs_spmv_M32(S.ctx, torch.tensor(x, device="cuda"), y)
    xd = x.astype(np.float64)
    ref = Sy.Mff @ xd
    scale = abs(Sy.Mff) @ np.abs(xd)
    err = np.abs(y.cpu().numpy() - ref) / np.maximum(scale, 1e-300)
    assert err.max() <= 1e-13, err.max()
    S.close()


def test_spmv_M_split_requires_mixed(E):
    p = PROBLEMS["cube2"]()
    S = E.Solver(p, precision=FP64)
    x = torch.zeros(p.n_free, dtype=torch.float32, device="cuda")
    y = torch.empty(p.n_free, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EqsError) as ex:
        E.eqs_spmv_M32(S.ctx, x, y)
    assert ex.value.status == E.EQS_ERR_STATE
    S.close()


@pytest.mark.parametrize("name", ["cube12", "jitter10", "cube2"])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-4)])
def test_vcycle(E, name, prec, tol):
    p = PROBLEMS[name]()
    S = E.Solver(p, precision=prec)
    H = amg.SAHierarchy(system.EQSSystem(p).Mff)
    r = np.random.default_rng(4).standard_normal(p.n_free)
    got = S.vcycle(_cuda(r)).cpu().numpy()
    assert _relmax(got, H(r)) <= tol
    S.close()


@pytest.mark.parametrize("name", ["cube12", "jitter10"])
@pytest.mark.parametrize("coarse_split", [0, 1])
def test_vcycle_mixed_coarse_forms(E, name, coarse_split):
    """Both mixed coarsest-level forms (FP32 inverse, FP32-pair inverse) give
    the oracle's V-cycle to FP32 accuracy, on a three-level hierarchy."""
    p = PROBLEMS[name]()
    S = E.Solver(p, precision=MIXED, coarse_max=60, coarse_split=coarse_split)
    H = amg.SAHierarchy(system.EQSSystem(p).Mff, coarse_max=60)
    assert len(H.levels) >= 3
    r = np.random.default_rng(14).standard_normal(p.n_free)
    got = S.vcycle(_cuda(r)).cpu().numpy()
    assert _relmax(got, H(r)) <= 1e-4
    S.close()


@pytest.mark.parametrize("name", ["cube12", "jitter10", "cube2"])
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_solve_M(E, name, prec):
    p = PROBLEMS[name]()
    S = E.Solver(p, precision=prec)
    Sy = system.EQSSystem(p)
    R = np.random.default_rng(5).standard_normal(p.n_free)
    zd = spla.spsolve(Sy.Mff.tocsc(), R)
    z, iters = S.solve_M(_cuda(R), rtol=1e-12)
    z = z.cpu().numpy()
    assert np.linalg.norm(z - zd) / np.linalg.norm(zd) <= 1e-9
    res = np.linalg.norm(R - Sy.Mff @ z) / np.linalg.norm(R)
    assert res <= 1e-11
    H = amg.SAHierarchy(Sy.Mff)
    _, it_or, _ = pcg.pcg(Sy.Mff, R, precond=H, rtol=1e-12)
    if prec == FP64:
        assert abs(iters[0] - it_or) <= 1
    else:
        assert iters[0] <= it_or + 3
    # zero right-hand side and a perfect start vector
    z0, it0 = S.solve_M(_cuda(np.zeros(p.n_free)), z0=_cuda(R))
    assert it0[0] == 0 and not z0.cpu().numpy().any()
    z1, it1 = S.solve_M(_cuda(R), z0=_cuda(zd), rtol=1e-8)
    assert it1[0] == 0
    S.close()


def _oracle_run(p, s, steps, dt):
    Sy = system.EQSSystem(p)
    coef = rkc.RKCCoefficients(s)
    xf, t, out = np.zeros(p.n_free), 0.0, []
    for _ in range(steps):
        xf, _ = rkc.rkc_step(Sy.F, t, xf, dt, coef)
        t += dt
        out.append(Sy.full(t, xf))
    return np.array(out)


@pytest.mark.parametrize("name,s,steps", [("cube12", 10, 12), ("jitter10", 20, 4), ("batch7", 10, 6)])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6)])
@pytest.mark.parametrize("persistent", [0, 1])
def test_rkc_trajectory(E, name, s, steps, prec, tol, persistent):
    p = PROBLEMS[name]()
    S = E.Solver(p, precision=prec, rtol=1e-13, persistent=persistent)
    dt = S.dt_bound(s)
    ref = _oracle_run(p, s, steps, dt)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    got, t = [], 0.0
    for _ in range(steps):
        st = S.step(x, t, dt, s)
        assert st.status == 0 and st.max_relres <= 1e-13
        t += dt
        got.append(x.cpu().numpy())
    got = np.array(got)
    err = np.linalg.norm(got - ref, axis=1).max() / np.linalg.norm(ref, axis=1).max()
    assert err <= tol, err
    S.close()


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_host_loop_matches_graph(E, prec):
    """The host-driven CG loop runs the same kernels as the graph's device loop."""
    p = PROBLEMS["jitter10"]()
    out = []
    for host_loop in (0, 1):
        S = E.Solver(p, precision=prec, rtol=1e-10, host_loop=host_loop, persistent=0)
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        dt, t, its = S.dt_bound(10), 0.0, []
        for _ in range(3):
            st = S.step(x, t, dt, 10)
            its.append(list(st.iters[:10]))
            t += dt
        out.append((x.cpu().numpy(), its, st.launches))
        S.close()
    assert out[0][1] == out[1][1]
    assert out[0][2] == out[1][2]  # launch counts agree
    # FP32 atomics in the mixed element kernel sum in a different order per run
    tol = 1e-11 if prec == FP64 else 1e-7
    np.testing.assert_allclose(out[1][0], out[0][0], rtol=0, atol=tol * np.abs(out[0][0]).max())


@pytest.mark.parametrize("name", ["cube12", "jitter10"])
@pytest.mark.parametrize("defer", [0, 1])
def test_mixed_degree1_trajectory_deferred_sums(E, name, defer):
    """The mixed path in the benchmark's smoother setting (degree-1
    Chebyshev, CG dots fused into the last smoothing pass), with the CG sums
    formed in the producer's last block (defer_sums 0) or added by every
    block of the consuming kernel (1): the oracle's trajectory to the mixed
    tolerance, graph and host loop with identical iteration counts, and the
    M-solve against a direct solve."""
    p = PROBLEMS[name]()
    s, steps = 10, 4
    opts = dict(cheb_degree=1, coarse_max=60, defer_sums=defer)
    out = []
    for host_loop in (0, 1):
        S = E.Solver(p, precision=MIXED, rtol=1e-13, host_loop=host_loop, **opts)
        dt = S.dt_bound(s)
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        t, its = 0.0, []
        for _ in range(steps):
            st = S.step(x, t, dt, s)
            assert st.status == 0 and st.max_relres <= 1e-13
            its.append(list(st.iters[:s]))
            t += dt
        out.append((x.cpu().numpy(), its))
        S.close()
    assert out[0][1] == out[1][1]
    ref = _oracle_run(p, s, steps, dt)[-1]
    assert np.linalg.norm(out[0][0] - ref) / np.linalg.norm(ref) <= 1e-6
    S = E.Solver(p, precision=MIXED, **opts)
    Sy = system.EQSSystem(p)
    R = np.random.default_rng(15).standard_normal(p.n_free)
    zd = spla.spsolve(Sy.Mff.tocsc(), R)
    z, iters = S.solve_M(_cuda(R), rtol=1e-12)
    S.close()
    assert 0 < iters[0] < 100
    assert np.linalg.norm(z.cpu().numpy() - zd) / np.linalg.norm(zd) <= 1e-9
