"""P1 tetrahedral finite elements for the EQS problem (oracle).

The EQS equation (Eq. 1) div(kappa grad phi) + div(eps grad dphi/dt) = 0 is
discretised with linear (P1) tetrahedra into M dx/dt + K(x) x = b (Eq. 2).
For one tet with vertices p0..p3:

* J = [p1-p0 | p2-p0 | p3-p0], volume V = det(J)/6;
* the rows of J^-1 are grad(lambda_1..3), grad(lambda_0) = -sum of them;
  G is the 4x3 matrix of these gradients;
* the field is constant per tet: grad phi = G^T phi_e, E = |grad phi|, so
  kappa(E) is constant per tet (one-point quadrature is exact on P1);
* local matrices K_e = kappa(E) V G G^T and M_e = eps V G G^T.

Section III: the explicit scheme never needs the global K(x), only the
vector K(x)x; every tet forms its local matrix, multiplies it with its own
four potentials and adds the four results into the global vector.
``apply_K`` does exactly that.  ``assemble_K``/``assemble_M`` build the
global CSR matrices (the classical assembly the paper contrasts with) and
serve as a check of ``apply_K``.

Pins (tests/test_oracle_fem.py): the reference tet's hand-computed local
matrix (tests/golden/ref_tet_stiffness.txt); volumes sum to L^3; the P1
patch test (linear phi has an exact constant gradient and zero interior
residual for uniform kappa); zero row sums; symmetry and positive
semi-definiteness; matrix-free equals assembled.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

EPS0 = 8.8541878128e-12  # vacuum permittivity [F/m], CODATA 2018


def tet_geometry(xyz, tets):
    """Return (G[n_tet,4,3], V[n_tet]) of every tet; raises on det J <= 0."""
    p = xyz[tets]  # (T, 4, 3)
    J = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], axis=2)
    det = np.linalg.det(J)
    if np.any(det <= 0.0):
        raise ValueError("inverted or degenerate tetrahedron")
    Jinv = np.linalg.inv(J)  # rows are grad(lambda_1..3)
    G = np.empty((len(tets), 4, 3))
    G[:, 1:, :] = Jinv
    G[:, 0, :] = -Jinv.sum(axis=1)
    return G, det / 6.0


def logistic(u):
    """Numerically stable logistic function 1/(1+exp(-u))."""
    e = np.exp(-np.abs(u))
    return np.where(u >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def kappa_of_E(E, mat):
    """Nonlinear conductivity kappa(E) = lo + (hi - lo) * logistic((E-E0)/w)
    of one material tuple (eps_r, kappa_lo, kappa_hi, E0, w)."""
    _, lo, hi, E0, w = mat
    if hi == lo:
        return np.full_like(np.asarray(E, dtype=np.float64), lo)
    return lo + (hi - lo) * logistic((np.asarray(E) - E0) / w)


def material_arrays(tet_mat, materials):
    mats = [m.as_tuple() if hasattr(m, "as_tuple") else tuple(m) for m in materials]
    return mats, np.asarray(tet_mat, dtype=np.int64)


def tet_kappa(xyz, tets, tet_mat, materials, x, G=None):
    """kappa of every tet at the potential x (E = |G^T x_e|)."""
    if G is None:
        G, _ = tet_geometry(xyz, tets)
    mats, mid = material_arrays(tet_mat, materials)
    grad = np.einsum("tkd,tk->td", G, x[tets])
    E = np.sqrt(np.einsum("td,td->t", grad, grad))
    kap = np.empty(len(tets))
    for m, mat in enumerate(mats):
        sel = mid == m
        kap[sel] = kappa_of_E(E[sel], mat)
    return kap, E


def local_matrices(G, V, coef):
    """coef_e * V_e * G_e G_e^T for every tet: (T, 4, 4)."""
    return (coef * V)[:, None, None] * np.einsum("tkd,tld->tkl", G, G)


def apply_K(xyz, tets, tet_mat, materials, x, geometry=None):
    """y = K(x) x, formed tet by tet and scattered into y (Section III).
    10-node tets go to the P2 element (oracle.fem_p2).  ``geometry`` is an
    optional (G, V) pair from tet_geometry of the same mesh (the geometry
    does not depend on x; passing it only saves recomputing it)."""
    if tets.shape[1] == 10:
        from . import fem_p2
        return fem_p2.apply_K(xyz, tets, tet_mat, materials, x)
    G, V = tet_geometry(xyz, tets) if geometry is None else geometry
    kap, _ = tet_kappa(xyz, tets, tet_mat, materials, x, G)
    Ke = local_matrices(G, V, kap)
    re = np.einsum("tkl,tl->tk", Ke, x[tets])
    y = np.zeros(len(xyz))
    np.add.at(y, tets, re)
    return y


def _assemble(n, tets, Ke):
    rows = np.repeat(tets, 4, axis=1).reshape(-1)
    cols = np.tile(tets, (1, 4)).reshape(-1)
    A = sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def assemble_K(xyz, tets, tet_mat, materials, x):
    """Global CSR K(x) (classical assembly), all nodes, before Dirichlet BCs."""
    if tets.shape[1] == 10:
        from . import fem_p2
        return fem_p2.assemble_K(xyz, tets, tet_mat, materials, x)
    G, V = tet_geometry(xyz, tets)
    kap, _ = tet_kappa(xyz, tets, tet_mat, materials, x, G)
    return _assemble(len(xyz), tets, local_matrices(G, V, kap))


def tet_eps(tet_mat, materials):
    mats, mid = material_arrays(tet_mat, materials)
    eps = np.array([EPS0 * m[0] for m in mats])
    return eps[mid]


def assemble_M(xyz, tets, tet_mat, materials):
    """Global CSR M (eps-weighted Laplace-type "mass" matrix of Eq. 2)."""
    if tets.shape[1] == 10:
        from . import fem_p2
        return fem_p2.assemble_M(xyz, tets, tet_mat, materials)
    G, V = tet_geometry(xyz, tets)
    return _assemble(len(xyz), tets, local_matrices(G, V, tet_eps(tet_mat, materials)))


def assemble_dKx(xyz, tets, tet_mat, materials, x):
    """Jacobian d(K(x)x)/dx: per tet V G [kappa I + kappa'(E) g g^T / E] G^T
    with g = grad phi (used to check the stability bound)."""
    G, V = tet_geometry(xyz, tets)
    mats, mid = material_arrays(tet_mat, materials)
    g = np.einsum("tkd,tk->td", G, x[tets])
    E = np.sqrt(np.einsum("td,td->t", g, g))
    kap = np.empty(len(tets))
    dk = np.zeros(len(tets))
    for m, (eps_r, lo, hi, E0, w) in enumerate(mats):
        sel = mid == m
        kap[sel] = kappa_of_E(E[sel], (eps_r, lo, hi, E0, w))
        if hi != lo:
            s = logistic((E[sel] - E0) / w)
            dk[sel] = (hi - lo) * s * (1 - s) / w
    with np.errstate(invalid="ignore", divide="ignore"):
        fac = np.where(E > 0, dk / np.where(E > 0, E, 1.0), 0.0)
    D = kap[:, None, None] * np.eye(3)[None] + fac[:, None, None] * np.einsum("td,te->tde", g, g)
    Ke = V[:, None, None] * np.einsum("tkd,tde,tle->tkl", G, D, G)
    return _assemble(len(xyz), tets, Ke)
