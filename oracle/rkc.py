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
