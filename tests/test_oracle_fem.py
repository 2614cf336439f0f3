"""Pins of the oracle's P1 element operator (Eq. 2, Section III)."""
import os

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import fem

CONST1 = ei.Material(1.0 / fem.EPS0, 1.0, 1.0)  # eps = 1, kappa = 1


def test_reference_tet_local_matrix(golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "ref_tet_stiffness.txt"))
            if l.strip() and not l.startswith("#")]
    want = np.array(rows, dtype=float) / 6.0
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    mat = np.zeros(1, dtype=np.uint8)
    K = fem.assemble_K(xyz, tets, mat, [CONST1], np.zeros(4)).toarray()
    M = fem.assemble_M(xyz, tets, mat, [CONST1]).toarray()
    np.testing.assert_allclose(K, want, rtol=0, atol=1e-15)
    np.testing.assert_allclose(M, want, rtol=0, atol=1e-15)


def _jittered(N=5):
    return ei.make_problem(N, jitter=0.2, seed=7, varistor="spheres",
                           spheres=[[0.05, 0.05, 0.05]], radius=0.03)


def test_volumes_sum_to_cube():
    p = _jittered()
    _, V = fem.tet_geometry(p.xyz, p.tets)
    assert np.all(V > 0)
    assert abs(V.sum() - ei.L_CUBE ** 3) < 1e-14 * ei.L_CUBE ** 3


def test_patch_test_linear_field():
    p = _jittered(6)
    a = np.array([3.0e4, -1.5e4, 2.0e4])
    phi = p.xyz @ a + 7.0
    G, V = fem.tet_geometry(p.xyz, p.tets)
    grad = np.einsum("tkd,tk->td", G, phi[p.tets])
    np.testing.assert_allclose(grad, np.broadcast_to(a, grad.shape), rtol=1e-11)
    # uniform kappa: interior residual vanishes
    mat = np.zeros(p.n_tets, dtype=np.uint8)
    y = fem.apply_K(p.xyz, p.tets, mat, [ei.Material(3.0, 2e-9, 2e-9)], phi)
    N = p.N
    n1 = N + 1
    idx = np.arange(p.n_nodes)
    i, j, k = idx % n1, (idx // n1) % n1, idx // (n1 * n1)
    inner = (i > 0) & (i < N) & (j > 0) & (j < N) & (k > 0) & (k < N)
    scale = np.abs(y).max()
    assert scale > 0
    assert np.abs(y[inner]).max() <= 1e-11 * scale


def _field_state(p, Emag=5.2e5):
    rng = np.random.default_rng(3)
    base = -Emag * p.xyz[:, 2]
    return base + 0.3 * Emag * 0.1 / p.N * rng.standard_normal(p.n_nodes)


def test_zero_row_sums_symmetry_psd():
    p = _jittered()
    x = _field_state(p)
    K = fem.assemble_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
    M = fem.assemble_M(p.xyz, p.tets, p.tet_mat, p.materials)
    for A in (K, M):
        rs = np.abs(A @ np.ones(p.n_nodes)).max()
        assert rs <= 1e-12 * abs(A).max()
        assert abs(A - A.T).max() <= 1e-15 * abs(A).max()
    ev = np.linalg.eigvalsh(M.toarray())
    assert ev.min() >= -1e-12 * ev.max()
    rng = np.random.default_rng(0)
    for _ in range(5):
        v = rng.standard_normal(p.n_nodes)
        assert v @ (K @ v) >= -1e-12 * abs(K).max() * (v @ v)


def test_matrix_free_equals_assembled():
    p = _jittered()
    x = _field_state(p)
    K = fem.assemble_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
    y = fem.apply_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
    kap, E = fem.tet_kappa(p.xyz, p.tets, p.tet_mat, p.materials, x)
    assert kap[p.tet_mat == 1].max() > 10 * ei.VARISTOR.kappa_lo  # nonlinearity active
    np.testing.assert_allclose(y, K @ x, rtol=0, atol=1e-13 * np.abs(y).max())


def test_kappa_law():
    m = ei.VARISTOR.as_tuple()
    assert fem.kappa_of_E(np.array([5e5]), m)[0] == pytest.approx((1e-12 + 1e-6) / 2, rel=1e-15)
    big = fem.kappa_of_E(np.array([0.0, 1e9]), m)
    assert np.all(np.isfinite(big))
    import math
    assert big[0] == pytest.approx(1e-12 + (1e-6 - 1e-12) / (1 + math.exp(10.0)), rel=1e-14)
    assert big[1] == pytest.approx(1e-6, rel=1e-15)
    const = fem.kappa_of_E(np.array([1.0, 1e7]), ei.BACKGROUND.as_tuple())
    assert np.all(const == 1e-14)


def test_sampled_rows_from_the_tets_around_a_node():
    """The full-size GPU tests let the oracle compute sampled rows only, from
    the tets that touch the sampled nodes: those rows of K(x)x and of M z
    equal the oracle's full products exactly (every term of a row comes from
    a tet around its node)."""
    p = ei.config_problem(2, N=14)  # jittered, two spheres
    rng = np.random.default_rng(5)
    x = -5.2e5 * p.xyz[:, 2] + 2e3 * rng.standard_normal(p.n_nodes)
    nodes = np.sort(rng.choice(p.n_nodes, 300, replace=False))
    sub = np.isin(p.tets, nodes).any(axis=1)
    assert 0 < sub.sum() < len(p.tets)
    y_sub = fem.apply_K(p.xyz, p.tets[sub], p.tet_mat[sub], p.materials, x)[nodes]
    y = fem.apply_K(p.xyz, p.tets, p.tet_mat, p.materials, x)[nodes]
    assert np.array_equal(y_sub, y)
    z = rng.standard_normal(p.n_nodes)
    Mz_sub = (fem.assemble_M(p.xyz, p.tets[sub], p.tet_mat[sub], p.materials) @ z)[nodes]
    Mz = (fem.assemble_M(p.xyz, p.tets, p.tet_mat, p.materials) @ z)[nodes]
    np.testing.assert_allclose(Mz_sub, Mz, rtol=0, atol=1e-15 * np.abs(Mz).max())
