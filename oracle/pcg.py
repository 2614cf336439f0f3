"""Preconditioned conjugate gradients for the M-solve (oracle).

Section IV: every RKC stage solves M z = R with the constant M by PCG (ref.
[3], Saad Alg. 9.1), started from an estimated solution.  Stopping test:
||r_k||_2 <= rtol ||R||_2 with the recursively updated residual r_k, i.e.
relative to the right-hand side (not to the initial residual), so that a
better start vector really saves iterations.  ``flexible=True`` uses the
Polak-Ribiere beta = z_{k+1}.(r_{k+1} - r_k) / (z_k.r_k), which equals the
Fletcher-Reeves value for a fixed linear preconditioner and keeps CG robust
when the preconditioner is applied in reduced precision.

Pins: tests/test_oracle_amg.py (converges to the direct solution; the
iteration count with a perfect start vector is 0; the zero right-hand side
returns zero).
"""

from __future__ import annotations

import numpy as np


def pcg(A, b, x0=None, precond=None, rtol=1e-8, maxit=1000, flexible=True):
    """Returns (x, iterations, converged)."""
    nb = float(np.linalg.norm(b))
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    if nb == 0.0:
        return np.zeros_like(b), 0, True
    r = b - A @ x
    if np.linalg.norm(r) <= rtol * nb:
        return x, 0, True
    M = precond if precond is not None else (lambda v: v.copy())
    z = M(r)
    p = z.copy()
    rz = float(r @ z)
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r_new = r - alpha * q
        if np.linalg.norm(r_new) <= rtol * nb:
            return x, it, True
        z = M(r_new)
        rz_new = float(r_new @ z)
        beta = float(z @ (r_new - r)) / rz if flexible else rz_new / rz
        rz = rz_new
        p = z + beta * p
        r = r_new
    return x, maxit, False
