"""Subspace projection extrapolation start vector (oracle).

Section IV, Eq. 4-5 (the SPE scheme of its ref. [12]): the last n solutions
x_1..x_n of the multiple right-hand-side sequence are orthonormalised by the
modified Gram-Schmidt process into V = [v_1 .. v_m], m <= n (a vector whose
remaining norm falls below ``drop`` times its own norm is linearly dependent
on the earlier ones and is skipped); the start vector of the next solve with
right-hand side b is

    x0 = V (V^T M V)^-1 V^T b,

the M-orthogonal projection of the solution onto span(V).  The most recent
solution is orthogonalised first.

Pins (tests/test_oracle_spe.py): V^T V = I; span preserved; a dependent
history vector is dropped; b = M x with x in the span is reproduced
exactly; the error of x0 is M-orthogonal to span(V); the result does not
depend on the order of the history.
"""
from __future__ import annotations

import numpy as np


def mgs(X, drop=1e-6):
    """Columns of X (most recent first) -> orthonormal V (n x m)."""
    V = []
    for k in range(X.shape[1]):
        v = np.array(X[:, k], dtype=np.float64, copy=True)
        n0 = np.linalg.norm(v)
        if n0 == 0.0:
            continue
        for u in V:
            v -= (u @ v) * u
        nv = np.linalg.norm(v)
        if nv > drop * n0:
            V.append(v / nv)
    return np.stack(V, axis=1) if V else np.zeros((X.shape[0], 0))


def spe_start(M, history, b, drop=1e-6):
    """x0 of Eq. 5 from the history [x_1 (most recent), x_2, ...]."""
    if len(history) == 0:
        return np.zeros_like(b)
    V = mgs(np.stack(history, axis=1), drop)
    if V.shape[1] == 0:
        return np.zeros_like(b)
    A = V.T @ (M @ V)
    return V @ np.linalg.solve(A, V.T @ b)
