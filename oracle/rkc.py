"""Runge-Kutta-Chebyshev scheme (oracle).

Section II proposes the explicit RKC scheme of ref. [9] (Sommeijer,
Shampine, Verwer 1998), extended to a non-diagonal mass matrix: every stage
evaluates F(t, y) = M^-1 (b(t) - K(y) y), i.e. one M-solve per stage.  The
paper prints no coefficients; they are those of the cited damped
second-order scheme:

    damping eps = 2/13, w0 = 1 + eps/s^2, w1 = T_s'(w0) / T_s''(w0)
    b_j = T_j''(w0) / T_j'(w0)^2   (j >= 2),   b_0 = b_1 = b_2
    a_j = 1 - b_j T_j(w0)
    mu~_1 = b_1 w1
    mu_j = 2 b_j w0 / b_{j-1},  nu_j = -b_j / b_{j-2},
    mu~_j = 2 b_j w1 / b_{j-1},  gamma~_j = -a_{j-1} mu~_j          (j >= 2)
    c_0 = 0, c_j = w1 T_j''(w0) / T_j'(w0) (j >= 2), c_1 = c_2 / T_2'(w0)

and the stages

    Y_0 = y_n,  Y_1 = Y_0 + mu~_1 tau F_0,
    Y_j = (1-mu_j-nu_j) Y_0 + mu_j Y_{j-1} + nu_j Y_{j-2}
          + mu~_j tau F_{j-1} + gamma~_j tau F_0,     F_k = F(t_n + c_k tau, Y_k)
    y_{n+1} = Y_s.

The stability polynomial after j stages is P_j(z) = a_j + b_j T_j(w0 + w1 z);
its real stability interval is [-beta_s, 0] with beta_s = (1 + w0)/w1
(about 0.653 s^2 for eps = 2/13).

Pins (tests/test_oracle_rkc.py): the Chebyshev recurrences against the
closed forms cosh(j acosh x), j sinh(j t)/sinh(t); the stage recurrence on
y' = lambda y against the closed-form P_j; P_s(z) = 1 + z + z^2/2 + O(z^3);
|P_s| <= 1 on [-beta_s, 0]; beta_s against (2/3)(s^2-1)(1-2 eps/15);
second-order convergence under step refinement.

Adaptive stepping (the paper runs with a local time-integration error below
1e-2; ref. [9] controls it): per step the number of stages is the smallest
s with beta_s >= h rho, the local error estimate is
Est = (12 (y_n - y_{n+1}) + 6 h (F_n + F_{n+1})) / 15 in a weighted RMS
norm, a step is accepted when that norm is <= 1 and the next step is
h 0.8 err^(-1/3) within [0.1 h, 10 h].  Readings: rho is the a-priori bound
of dtbound (the paper does not say how it is estimated); the simple
(non-PI) step controller.  Pins (tests/test_oracle_rkc_adaptive.py): the
estimate vanishes where the scheme is exact and equals h^3 y3/15 - 12/15
of the local error to leading order (y3 the third derivative); the stage
choice against brute force; global error and step counts scale with the
tolerance like a second-order method; a rejected step shrinks.
"""

from __future__ import annotations

import numpy as np

DAMPING = 2.0 / 13.0


def chebyshev_T(x: float, s: int):
    """T_j(x), T_j'(x), T_j''(x) for j = 0..s by the three-term recurrences."""
    T = np.zeros(s + 1)
    dT = np.zeros(s + 1)
    d2T = np.zeros(s + 1)
    T[0] = 1.0
    if s >= 1:
        T[1] = x
        dT[1] = 1.0
    for j in range(2, s + 1):
        T[j] = 2.0 * x * T[j - 1] - T[j - 2]
        dT[j] = 2.0 * T[j - 1] + 2.0 * x * dT[j - 1] - dT[j - 2]
        d2T[j] = 4.0 * dT[j - 1] + 2.0 * x * d2T[j - 1] - d2T[j - 2]
    return T, dT, d2T


class RKCCoefficients:
    """All scalar coefficients of the s-stage RKC scheme (s >= 2)."""

    def __init__(self, s: int, damping: float = DAMPING):
        if s < 2:
            raise ValueError("RKC needs s >= 2 stages")
        self.s = s
        self.w0 = w0 = 1.0 + damping / (s * s)
        T, dT, d2T = chebyshev_T(w0, s)
        self.w1 = w1 = dT[s] / d2T[s]
        b = np.zeros(s + 1)
        for j in range(2, s + 1):
            b[j] = d2T[j] / dT[j] ** 2
        b[0] = b[1] = b[2]
        a = 1.0 - b * T
        self.a, self.b, self.T = a, b, T
        self.mu = np.zeros(s + 1)
        self.nu = np.zeros(s + 1)
        self.mut = np.zeros(s + 1)
        self.gt = np.zeros(s + 1)
        self.mut[1] = b[1] * w1
        for j in range(2, s + 1):
            self.mu[j] = 2.0 * b[j] * w0 / b[j - 1]
            self.nu[j] = -b[j] / b[j - 2]
            self.mut[j] = 2.0 * b[j] * w1 / b[j - 1]
            self.gt[j] = -a[j - 1] * self.mut[j]
        c = np.zeros(s + 1)
        for j in range(2, s + 1):
            c[j] = w1 * d2T[j] / dT[j]
        c[1] = c[2] / dT[2]
        self.c = c
        self.beta = (1.0 + w0) / w1

    def stability_poly(self, z, j=None):
        """P_j(z) = a_j + b_j T_j(w0 + w1 z) (closed form, any j <= s)."""
        j = self.s if j is None else j
        x = self.w0 + self.w1 * np.asarray(z, dtype=np.float64)
        if j == 0:
            return np.ones_like(x)
        Tj = np.where(np.abs(x) <= 1.0, np.cos(j * np.arccos(np.clip(x, -1, 1))),
                      np.sign(x) ** j * np.cosh(j * np.arccosh(np.maximum(np.abs(x), 1.0))))
        return self.a[j] + self.b[j] * Tj


def rkc_step(F, t: float, y: np.ndarray, dt: float, coef: RKCCoefficients):
    """One RKC step y_n -> y_{n+1}; F(t, y) is called s times (F_0..F_{s-1}).

    Returns (y_{n+1}, stages) where stages is the list of (t_k, F_k)."""
    s = coef.s
    Y0 = y
    F0 = F(t, Y0)
    calls = [(t, F0)]
    Yjm2 = Y0
    Yjm1 = Y0 + coef.mut[1] * dt * F0
    for j in range(2, s + 1):
        tk = t + coef.c[j - 1] * dt
        Fjm1 = F(tk, Yjm1)
        calls.append((tk, Fjm1))
        Yj = ((1.0 - coef.mu[j] - coef.nu[j]) * Y0 + coef.mu[j] * Yjm1 + coef.nu[j] * Yjm2
              + coef.mut[j] * dt * Fjm1 + coef.gt[j] * dt * F0)
        Yjm2, Yjm1 = Yjm1, Yj
    return Yjm1, calls


# ------------------------------------------------------- adaptive stepping
def stages_for(h: float, rho: float, s_max: int = 64):
    """Smallest s >= 2 whose stability interval covers h*rho (beta_s >= h rho);
    (s_max, beta_smax / rho) when even s_max does not: the step is cut."""
    for s in range(2, s_max + 1):
        if RKCCoefficients(s).beta >= h * rho:
            return s, h
    return s_max, RKCCoefficients(s_max).beta / rho


def error_estimate(h, y0, y1, F0, F1):
    """Local error estimate of the RKC scheme (ref. [9]):
    Est = (12 (y_n - y_{n+1}) + 6 h (F(t_n, y_n) + F(t_{n+1}, y_{n+1}))) / 15."""
    return (12.0 * (y0 - y1) + 6.0 * h * (F0 + F1)) / 15.0


def error_norm(est, y0, y1, atol, rtol):
    """Weighted RMS norm: sqrt(mean((Est_i / (atol + rtol max(|y0_i|, |y1_i|)))^2))."""
    w = atol + rtol * np.maximum(np.abs(y0), np.abs(y1))
    return float(np.sqrt(np.mean((est / w) ** 2)))


def step_factor(err: float) -> float:
    """Step size factor 0.8 err^(-1/3), kept in [0.1, 10] (second-order
    scheme: the local error scales like h^3)."""
    if err == 0.0:
        return 10.0
    return min(10.0, max(0.1, 0.8 * err ** (-1.0 / 3.0)))


def rkc_adaptive_step(F, t, y, F0, h, rho, atol, rtol, s_max=64, max_tries=50):
    """One accepted adaptive RKC step from (t, y) with F0 = F(t, y), trying
    step h first.  Each try: s from stages_for(h, rho), one RKC step,
    F1 = F(t + h, y1), the error norm of error_estimate; accept when
    err <= 1, else retry with h * step_factor(err).

    Returns (y1, F1, h_used, s, err, h_next, tries)."""
    for tries in range(1, max_tries + 1):
        s, h = stages_for(h, rho, s_max)
        y1, _ = rkc_step(F, t, y, h, RKCCoefficients(s))
        F1 = F(t + h, y1)
        err = error_norm(error_estimate(h, y, y1, F0, F1), y, y1, atol, rtol)
        if err <= 1.0:
            return y1, F1, h, s, err, h * step_factor(err), tries
        h = h * step_factor(err)
    raise RuntimeError("adaptive RKC: too many rejected steps")
