"""Pins of the oracle's quadratic (P2) element (the paper's 2nd order
ansatz functions, Section V)."""
import numpy as np
import pytest

import eqs_inputs as ei
from oracle import fem, fem_p2, system

sympy = pytest.importorskip("sympy")


def test_reference_tet_matrix_against_symbolic_integration():
    """M_e of the unit reference tet (eps = 1) equals the exact integral of
    grad N_i . grad N_j, computed symbolically from the shape functions."""
    x, y, z = sympy.symbols("x y z")
    l = [1 - x - y - z, x, y, z]
    N = [l[k] * (2 * l[k] - 1) for k in range(4)] + [4 * l[a] * l[b] for a, b in fem_p2.EDGES]
    grads = [[sympy.diff(n, v) for v in (x, y, z)] for n in N]
    exact = np.zeros((10, 10))
    for i in range(10):
        for j in range(i, 10):
            f = sum(grads[i][d] * grads[j][d] for d in range(3))
            val = sympy.integrate(f, (z, 0, 1 - x - y), (y, 0, 1 - x), (x, 0, 1))
            exact[i, j] = exact[j, i] = float(val)
    xyz = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    mids = np.array([(xyz[a] + xyz[b]) / 2 for a, b in fem_p2.EDGES])
    xyz10 = np.vstack([xyz, mids])
    tets = np.arange(10, dtype=np.int32)[None, :]
    mat = (ei.Material(1.0 / fem.EPS0, 0.0, 0.0),)
    M = fem_p2.assemble_M(xyz10, tets, np.zeros(1, np.uint8), mat).toarray()
    np.testing.assert_allclose(M, exact, rtol=1e-12, atol=1e-14)


def _mesh(N=3):
    return ei.make_problem_p2(N, jitter=0.2, seed=7)


def test_mesh_counts_and_volume():
    p = _mesh(3)
    assert p.xyz.shape == (7 ** 3, 3) and p.tets.shape == (6 * 27, 10)
    G, V = fem_p2.geometry(p.xyz, p.tets)
    assert V.sum() == pytest.approx(ei.L_CUBE ** 3, rel=1e-13)
    for e, (a, b) in enumerate(fem_p2.EDGES):
        np.testing.assert_allclose(p.xyz[p.tets[:, 4 + e]], 0.5 * (p.xyz[p.tets[:, a]] + p.xyz[p.tets[:, b]]),
                                   rtol=0, atol=1e-15)


def test_quadratic_fields_are_exact():
    """phi quadratic: its nodal values reproduce grad phi at every
    quadrature point of every tet."""
    p = _mesh(2)
    X, Y, Z = p.xyz.T
    phi = 3 * X * X - 2 * Y * Z + X + 0.5 * Z
    G, _ = fem_p2.geometry(p.xyz, p.tets)
    for q in range(4):
        B = fem_p2.shape_gradients(G, fem_p2.QUAD_LAMBDA[q])
        g = np.einsum("tkd,tk->td", B, phi[p.tets])
        pts = np.einsum("k,tkd->td", fem_p2.QUAD_LAMBDA[q], p.xyz[p.tets[:, :4]])
        ref = np.stack([6 * pts[:, 0] + 1, -2 * pts[:, 2], -2 * pts[:, 1] + 0.5], axis=1)
        np.testing.assert_allclose(g, ref, rtol=1e-10, atol=1e-10)


def test_row_sums_symmetry_and_linear_patch():
    p = _mesh(3)
    x = np.random.default_rng(1).standard_normal(p.n_nodes) * 1e4
    K = fem.assemble_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
    np.testing.assert_allclose(K @ np.ones(p.n_nodes), 0, atol=1e-14 * abs(K).max())
    assert abs(K - K.T).max() <= 1e-14 * abs(K).max()
    M = fem.assemble_M(p.xyz, p.tets, p.tet_mat, p.materials)
    ev = np.linalg.eigvalsh(M.toarray())
    assert ev.min() >= -1e-12 * ev.max()
    # uniform conductivity, linear field: zero residual at interior nodes
    q = ei.make_problem_p2(3, jitter=0.2, seed=7)
    q.materials = (ei.Material(3.0, 1e-9, 1e-9),)
    q.tet_mat = np.zeros_like(q.tet_mat)
    lin = 2.0 * q.xyz[:, 0] - q.xyz[:, 1] + 4.0 * q.xyz[:, 2]
    r = fem.apply_K(q.xyz, q.tets, q.tet_mat, q.materials, lin)
    R = 7
    I, J, Kk = np.arange(R ** 3) % R, (np.arange(R ** 3) // R) % R, np.arange(R ** 3) // (R * R)
    interior = (I > 0) & (I < R - 1) & (J > 0) & (J < R - 1) & (Kk > 0) & (Kk < R - 1)
    assert np.abs(r[interior]).max() <= 1e-12 * np.abs(r).max()


def test_matrix_free_equals_assembled():
    p = _mesh(3)
    x = np.random.default_rng(2).standard_normal(p.n_nodes) * 5e3 + 4e5 * p.xyz[:, 2]
    y = fem.apply_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
    K = fem.assemble_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
    np.testing.assert_allclose(y, K @ x, rtol=1e-12, atol=1e-12 * np.abs(y).max())


def test_system_lift_linear_in_z():
    """Homogeneous P2 slab: the static lift M_ff^-1 (-M_fd 1_top) is z/L."""
    p = ei.make_problem_p2(3, jitter=0.2, seed=7)
    p.materials = (ei.Material(3.0, 1e-9, 1e-9),)
    p.tet_mat = np.zeros_like(p.tet_mat)
    S = system.EQSSystem(p)
    H = S.solve_direct(-S.m_top)
    np.testing.assert_allclose(H, p.xyz[S.free, 2] / ei.L_CUBE, rtol=1e-11, atol=1e-12)
