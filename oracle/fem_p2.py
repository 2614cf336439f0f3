"""Quadratic (P2, 10-node) tetrahedral elements for the EQS problem (oracle).

The paper's second workload uses 2nd order ansatz functions (Section V,
Figs. 4-5; 17.4 M DoF, 494 M non-zeros); the method is unchanged: every
stage forms K(x)x tet by tet (Section III) and solves with the constant M.

For one tet with vertices p0..p3 (straight edges) the barycentric
coordinates lambda_k have the constant gradients of the P1 element (rows
of J^-1, grad lambda_0 = -sum).  The ten shape functions are

    vertex k:      N_k  = lambda_k (2 lambda_k - 1),
                   grad = (4 lambda_k - 1) grad lambda_k
    edge (k, l):   N_kl = 4 lambda_k lambda_l,
                   grad = 4 (lambda_k grad lambda_l + lambda_l grad lambda_k)

in the node order p0..p3, then the edges (0,1), (0,2), (0,3), (1,2), (1,3),
(2,3).  grad phi is linear in the tet, so kappa(|E|) varies inside it;
both local matrices are integrated with the symmetric 4-point rule of
degree 2 (barycentric points (a, b, b, b) and permutations,
a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20, weights V/4):

    r_e = sum_q (V/4) kappa(|grad phi(q)|) B_q (B_q^T phi_e)
    M_e = eps (V/4) sum_q B_q B_q^T     (exact: the integrand is quadratic)

with B_q the 10 x 3 matrix of shape-function gradients at point q.
Readings: the degree-2 rule for the nonlinear conductivity (the paper does
not say how it integrates K(x) for P2); straight edges (midpoint nodes at
edge midpoints).

Pins (tests/test_oracle_fem_p2.py): the reference tet's M_e against exact
symbolic integration; quadratic fields interpolated exactly (gradient at the
quadrature points); zero row sums; zero interior residual of a linear field
for uniform kappa; symmetry and semi-definiteness; matrix-free equals
assembled; volumes sum to L^3.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fem import kappa_of_E, material_arrays, tet_geometry

EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
_A = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
_B = (5.0 - np.sqrt(5.0)) / 20.0
QUAD_LAMBDA = np.array([[_A, _B, _B, _B], [_B, _A, _B, _B], [_B, _B, _A, _B], [_B, _B, _B, _A]])
QUAD_WEIGHT = np.full(4, 0.25)  # times the volume


def shape_gradients(G, lam):
    """B[t, 10, 3]: shape-function gradients at barycentric point lam (4,)
    for tets with barycentric gradients G[t, 4, 3]."""
    B = np.empty((G.shape[0], 10, 3))
    for k in range(4):
        B[:, k] = (4.0 * lam[k] - 1.0) * G[:, k]
    for e, (k, l) in enumerate(EDGES):
        B[:, 4 + e] = 4.0 * (lam[k] * G[:, l] + lam[l] * G[:, k])
    return B


def geometry(xyz, tets10):
    """(G[t,4,3], V[t]) from the four vertices."""
    return tet_geometry(xyz, np.ascontiguousarray(tets10[:, :4]))


def apply_K(xyz, tets10, tet_mat, materials, x):
    """y = K(x) x (quadrature-point conductivities), formed tet by tet."""
    G, V = geometry(xyz, tets10)
    mats, mid = material_arrays(tet_mat, materials)
    xe = x[tets10]  # (T, 10)
    r = np.zeros((len(tets10), 10))
    for q in range(4):
        B = shape_gradients(G, QUAD_LAMBDA[q])
        g = np.einsum("tkd,tk->td", B, xe)
        E = np.sqrt(np.einsum("td,td->t", g, g))
        kap = np.empty(len(tets10))
        for m, mat in enumerate(mats):
            sel = mid == m
            kap[sel] = kappa_of_E(E[sel], mat)
        r += (QUAD_WEIGHT[q] * V * kap)[:, None] * np.einsum("tkd,td->tk", B, g)
    y = np.zeros(len(xyz))
    np.add.at(y, tets10.reshape(-1), r.reshape(-1))
    return y


def _assemble(xyz, tets10, coef_q):
    """sum over tets and quadrature points of coef_q[q][t] (V/4) B_q B_q^T."""
    G, V = geometry(xyz, tets10)
    Ke = np.zeros((len(tets10), 10, 10))
    for q in range(4):
        B = shape_gradients(G, QUAD_LAMBDA[q])
        Ke += (QUAD_WEIGHT[q] * V * coef_q[q])[:, None, None] * np.einsum("tid,tjd->tij", B, B)
    rows = np.repeat(tets10, 10, axis=1).reshape(-1)
    cols = np.tile(tets10, (1, 10)).reshape(-1)
    n = len(xyz)
    A = sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def assemble_M(xyz, tets10, tet_mat, materials):
    from .fem import EPS0
    mats, mid = material_arrays(tet_mat, materials)
    eps = np.array([EPS0 * mats[m][0] for m in mid])
    return _assemble(xyz, tets10, [eps] * 4)


def assemble_K(xyz, tets10, tet_mat, materials, x):
    G, _ = geometry(xyz, tets10)
    mats, mid = material_arrays(tet_mat, materials)
    xe = x[tets10]
    kq = []
    for q in range(4):
        B = shape_gradients(G, QUAD_LAMBDA[q])
        g = np.einsum("tkd,tk->td", B, xe)
        E = np.sqrt(np.einsum("td,td->t", g, g))
        kap = np.empty(len(tets10))
        for m, mat in enumerate(mats):
            sel = mid == m
            kap[sel] = kappa_of_E(E[sel], mat)
        kq.append(kap)
    return _assemble(xyz, tets10, kq)
