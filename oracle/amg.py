"""Smoothed-aggregation AMG preconditioner for the constant M (oracle).

Section II / IV: M is constant, so the AMG preconditioner of the CG solver
is set up once and reused for every stage solve (the multiple right-hand
side problem).  The paper uses the AMG-CG solvers of refs. [7,8] (CUSP-based
smoothed aggregation) and names ref. [6] for AMG; it prints no setup
details, so this module follows the textbook smoothed-aggregation
construction (Vanek, Mandel, Brezina 1996) with choices fixed as below;
the CUDA library implements the same definition independently.

Setup of level l with matrix A (SPD, CSR with sorted columns):

1. strength: j != i is a strong neighbour of i iff a_ij != 0 and
   a_ij^2 >= theta_l^2 |a_ii a_jj|, theta_l = 0.08 * 0.5^l on level l
   (the level-scaled threshold of Vanek et al.; symmetric relation);
2. aggregation, nodes visited in index order:
   pass 1: an unaggregated node whose strong neighbours are all
           unaggregated starts a new aggregate = itself + those neighbours;
   pass 2: every node still unaggregated joins the pass-1 aggregate of its
           strong neighbour with the smallest index (a node with no
           aggregated strong neighbour becomes a singleton aggregate);
3. tentative prolongator: P^_{i, agg(i)} = 1/sqrt(|agg(i)|)
   (the constant near-null-space vector, column-normalised);
4. smoothed prolongator: P = (I - omega D^-1 A) P^,
   omega = (4/3)/lambda^, lambda^ = max_i sum_j |a_ij| / a_ii
   (Gershgorin bound of rho(D^-1 A));
5. Galerkin coarse matrix A_c = P^T A P.
Coarsening stops when a level has <= coarse_max rows, when max_levels is
reached or when aggregation no longer reduces the size; the coarsest level
is solved exactly (dense Cholesky).

V-cycle (symmetric, V(nu, nu) with the same polynomial pre- and
post-smoother): Chebyshev iteration (Saad, Iterative Methods, Alg. 12.1)
of degree ``degree`` on D^-1 A over [lambda^/alpha, lambda^]; residual
restriction with P^T; coarse correction prolongated with P.

Pins (tests/test_oracle_amg.py): aggregation covers every node exactly
once with connected aggregates; P^ has orthonormal columns; the Chebyshev
smoother's error factor on each eigenvector of D^-1 A equals the
closed-form T_k((theta - lambda)/delta)/T_k(theta/delta); the coarse-grid
correction is an A-orthogonal projector; the V-cycle is symmetric positive
definite and its two-grid error operator contracts in the A-norm; PCG with
it reaches the direct solution.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def strong_neighbours(A, theta):
    """CSR boolean pattern S of strong connections (no diagonal)."""
    A = A.tocsr()
    n = A.shape[0]
    diag = A.diagonal()
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    cols = A.indices
    vals = A.data
    keep = (cols != rows) & (vals != 0.0) & (vals * vals >= theta * theta * np.abs(diag[rows] * diag[cols]))
    S = sp.csr_matrix((np.ones(np.count_nonzero(keep)), (rows[keep], cols[keep])), shape=(n, n))
    S.sort_indices()
    return S


def aggregate(S):
    """Greedy two-pass aggregation; returns (agg[n] int64, n_agg)."""
    n = S.shape[0]
    ptr, idx = S.indptr, S.indices
    agg = np.full(n, -1, dtype=np.int64)
    n_agg = 0
    for i in range(n):  # pass 1
        if agg[i] >= 0:
            continue
        nb = idx[ptr[i]:ptr[i + 1]]
        if np.all(agg[nb] < 0):
            agg[i] = n_agg
            agg[nb] = n_agg
            n_agg += 1
    agg1 = agg.copy()
    for i in range(n):  # pass 2
        if agg[i] >= 0:
            continue
        nb = idx[ptr[i]:ptr[i + 1]]
        joined = nb[agg1[nb] >= 0]
        if len(joined):
            agg[i] = agg1[joined[0]]
        else:
            agg[i] = n_agg
            n_agg += 1
    return agg, n_agg


def tentative_prolongator(agg, n_agg):
    n = len(agg)
    counts = np.bincount(agg, minlength=n_agg).astype(np.float64)
    vals = 1.0 / np.sqrt(counts[agg])
    P = sp.csr_matrix((vals, (np.arange(n), agg)), shape=(n, n_agg))
    P.sort_indices()
    return P


def gershgorin_DinvA(A):
    """lambda^ = max_i sum_j |a_ij| / a_ii  >=  rho(D^-1 A)."""
    A = A.tocsr()
    absA = abs(A)
    return float(np.max(np.asarray(absA.sum(axis=1)).ravel() / A.diagonal()))


class Level:
    def __init__(self, A):
        self.A = A.tocsr()
        self.A.sort_indices()
        self.n = A.shape[0]
        self.Dinv = 1.0 / self.A.diagonal()
        self.lam_max = gershgorin_DinvA(self.A)
        self.P = None
        self.agg = None


class SAHierarchy:
    def __init__(self, A, theta=0.08, coarse_max=500, max_levels=10, degree=2, alpha=30.0):
        self.theta, self.degree, self.alpha = theta, degree, alpha
        self.levels = [Level(A)]
        while len(self.levels) < max_levels and self.levels[-1].n > coarse_max:
            lev = self.levels[-1]
            S = strong_neighbours(lev.A, theta * 0.5 ** (len(self.levels) - 1))
            agg, n_agg = aggregate(S)
            if n_agg >= lev.n:
                break
            P0 = tentative_prolongator(agg, n_agg)
            omega = (4.0 / 3.0) / lev.lam_max
            P = (P0 - omega * (sp.diags(lev.Dinv) @ (lev.A @ P0))).tocsr()
            P.sort_indices()
            Ac = (P.T @ lev.A @ P).tocsr()
            Ac.sort_indices()
            lev.P, lev.agg, lev.n_agg, lev.omega = P, agg, n_agg, omega
            self.levels.append(Level(Ac))
        self.coarse_chol = sla.cho_factor(self.levels[-1].A.toarray(), lower=True)

    def operator_complexity(self):
        return sum(l.A.nnz for l in self.levels) / self.levels[0].A.nnz

    def chebyshev(self, lev, b, x=None):
        """Chebyshev iteration of degree self.degree for A x = b, Jacobi-scaled,
        on the interval [lam_max/alpha, lam_max]; x is the initial guess."""
        lmax = lev.lam_max
        lmin = lmax / self.alpha
        theta = 0.5 * (lmax + lmin)
        delta = 0.5 * (lmax - lmin)
        sigma = theta / delta
        rho_old = 1.0 / sigma
        if x is None:
            x = np.zeros_like(b)
            r = b.copy()
        else:
            r = b - lev.A @ x
        d = lev.Dinv * r / theta
        x = x + d
        for _ in range(1, self.degree):
            r = r - lev.A @ d
            rho_new = 1.0 / (2.0 * sigma - rho_old)
            d = rho_new * rho_old * d + (2.0 * rho_new / delta) * (lev.Dinv * r)
            x = x + d
            rho_old = rho_new
        return x

    def vcycle(self, r, l=0):
        lev = self.levels[l]
        if l == len(self.levels) - 1:
            return sla.cho_solve(self.coarse_chol, r)
        z = self.chebyshev(lev, r)
        rc = lev.P.T @ (r - lev.A @ z)
        z = z + lev.P @ self.vcycle(rc, l + 1)
        return self.chebyshev(lev, r, z)

    def __call__(self, r):
        return self.vcycle(r)
