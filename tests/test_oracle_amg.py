"""Pins of the oracle's smoothed-aggregation AMG and PCG."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.sparse.csgraph import connected_components

import eqs_inputs as ei
from oracle import amg, pcg, rkc, system


@pytest.fixture(scope="module")
def sys4():
    return system.EQSSystem(ei.make_problem(6, jitter=0.2, seed=3))


def test_aggregation_partition_connected(sys4):
    A = sys4.Mff
    S = amg.strong_neighbours(A, 0.08)
    assert abs(S - S.T).max() == 0
    agg, na = amg.aggregate(S)
    assert agg.min() == 0 and agg.max() == na - 1
    assert np.all(np.bincount(agg) > 0)
    for a in range(na):
        nodes = np.nonzero(agg == a)[0]
        sub = S[nodes][:, nodes]
        ncomp, _ = connected_components(sub, directed=False)
        assert ncomp == 1


def test_tentative_prolongator_orthonormal(sys4):
    agg, na = amg.aggregate(amg.strong_neighbours(sys4.Mff, 0.08))
    P0 = amg.tentative_prolongator(agg, na)
    np.testing.assert_allclose((P0.T @ P0).toarray(), np.eye(na), atol=1e-15)


def test_chebyshev_error_factor_closed_form(sys4):
    H = amg.SAHierarchy(sys4.Mff, degree=3)
    lev = H.levels[0]
    A = lev.A.toarray()
    d = np.diag(A)
    B = A / np.sqrt(np.outer(d, d))
    lam, Q = np.linalg.eigh(B)
    lmax, lmin = lev.lam_max, lev.lam_max / H.alpha
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    for k in (0, len(lam) // 2, len(lam) - 1):
        v = Q[:, k] / np.sqrt(d)  # eigenvector of D^-1 A
        e = H.chebyshev(lev, np.zeros_like(v), v.copy())
        T = rkc.chebyshev_T((theta - lam[k]) / delta, 3)[0][3]
        T0 = rkc.chebyshev_T(theta / delta, 3)[0][3]
        np.testing.assert_allclose(e, (T / T0) * v, rtol=1e-9, atol=1e-12 * np.abs(v).max())


def test_vcycle_spd_projection_and_contraction():
    S = system.EQSSystem(ei.make_problem(5, jitter=0.2, seed=4))
    H = amg.SAHierarchy(S.Mff, coarse_max=40)
    assert len(H.levels) >= 2
    lev = H.levels[0]
    A = lev.A.toarray()
    P = lev.P.toarray()
    Ac = H.levels[1].A.toarray()
    np.testing.assert_allclose(Ac, P.T @ A @ P, rtol=1e-12, atol=1e-12 * abs(Ac).max())
    C = P @ np.linalg.solve(Ac, P.T @ A)
    np.testing.assert_allclose(C @ C, C, atol=1e-10)
    np.testing.assert_allclose(A @ C, (A @ C).T, atol=1e-10 * abs(A).max())
    n = A.shape[0]
    Bm = np.column_stack([H(np.eye(n)[:, i]) for i in range(n)])
    np.testing.assert_allclose(Bm, Bm.T, atol=1e-10 * abs(Bm).max())
    assert np.linalg.eigvalsh(0.5 * (Bm + Bm.T)).min() > 0
    ev = np.linalg.eigvals(np.eye(n) - Bm @ A)
    assert np.abs(ev.imag).max() < 1e-8 and ev.real.min() > -1e-8  # I - BA ~ [0, 1)
    assert np.abs(ev).max() < 0.95  # V-cycle error operator contracts


def test_pcg_reaches_direct_solution(sys4):
    H = amg.SAHierarchy(sys4.Mff)
    rng = np.random.default_rng(2)
    R = rng.standard_normal(sys4.Mff.shape[0])
    z_direct = spla.spsolve(sys4.Mff.tocsc(), R)
    for flex in (True, False):
        z, it, ok = pcg.pcg(sys4.Mff, R, precond=H, rtol=1e-13, flexible=flex)
        assert ok and 0 < it < 40
        np.testing.assert_allclose(z, z_direct, rtol=1e-9, atol=1e-9 * np.abs(z_direct).max())
    z, it, ok = pcg.pcg(sys4.Mff, R, x0=z_direct, precond=H, rtol=1e-8)
    assert ok and it == 0
    z, it, ok = pcg.pcg(sys4.Mff, np.zeros_like(R), precond=H)
    assert ok and it == 0 and not z.any()


def test_hierarchy_config0_shape():
    S = system.EQSSystem(ei.config_problem(0))
    H = amg.SAHierarchy(S.Mff)
    assert [l.n for l in H.levels][0] == 1859
    assert H.levels[-1].n <= 500
    assert 1.0 < H.operator_complexity() < 2.0
