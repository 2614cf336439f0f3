"""A-priori bound of the stiffness of the EQS ODE and the RKC step (oracle).

Section II: the RKC step size is limited by the stability interval
[-beta_s, 0] of the scheme.  The paper does not say how the spectral radius
is estimated; the reading used here is a mesh-independent a-priori bound.
The Jacobian of the element residual kappa(|g|) V G g (g = G^T phi_e) is
V G [kappa I + kappa'(E) g g^T / E] G^T whose 3x3 core has eigenvalues
kappa and sigma_d = d(kappa E)/dE = kappa + E kappa'.  Since each local
Jacobian is bounded by max(kappa, sigma_d)/eps_e times the local M_e, the
Rayleigh quotient gives

    rho(M_ff^-1 J_ff) <= max over materials, E of max(kappa, sigma_d) / eps.

For the logistic law sigma_d(E) = lo + (hi-lo)[s + (E/w) s (1-s)],
s = logistic((E - E0)/w); its maximum is found by golden-section search on
the unimodal bump.  dt = beta_s / rho (no safety factor: rho is an upper
bound already).

Pin: tests/test_oracle_dtbound.py compares rho with the largest
generalised eigenvalue of (J_ff, M_ff) on small meshes.
"""

from __future__ import annotations

import math

from .fem import EPS0


def _logistic(u):
    if u >= 0:
        return 1.0 / (1.0 + math.exp(-u))
    e = math.exp(u)
    return e / (1.0 + e)


def sigma_d(E, mat):
    _, lo, hi, E0, w = mat
    if hi == lo:
        return lo
    s = _logistic((E - E0) / w)
    return lo + (hi - lo) * (s + (E / w) * s * (1.0 - s))


def max_sigma_d(mat):
    """max over E >= 0 of sigma_d(E) (and kappa(E) <= sigma_d for kappa' >= 0)."""
    _, lo, hi, E0, w = mat
    if hi == lo:
        return lo
    # coarse scan in u = (E-E0)/w, then golden-section refinement
    best_u, best = None, -1.0
    u = -E0 / w
    while u <= 60.0:
        v = sigma_d(E0 + u * w, mat)
        if v > best:
            best, best_u = v, u
        u += 0.01
    lo_u, hi_u = best_u - 0.02, best_u + 0.02
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    for _ in range(200):
        a = hi_u - gr * (hi_u - lo_u)
        b = lo_u + gr * (hi_u - lo_u)
        if sigma_d(E0 + a * w, mat) > sigma_d(E0 + b * w, mat):
            hi_u = b
        else:
            lo_u = a
    um = 0.5 * (lo_u + hi_u)
    return max(best, sigma_d(E0 + um * w, mat), hi)


def rho_bound(materials):
    rho = 0.0
    for m in materials:
        mat = m.as_tuple() if hasattr(m, "as_tuple") else tuple(m)
        rho = max(rho, max_sigma_d(mat) / (EPS0 * mat[0]))
    return rho


def dt_bound(materials, s, coef=None):
    from .rkc import RKCCoefficients
    coef = coef or RKCCoefficients(s)
    return coef.beta / rho_bound(materials)
