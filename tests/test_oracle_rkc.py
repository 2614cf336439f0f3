"""Pins of the oracle's RKC scheme (Section II; the scheme of its ref. [9])."""
import math

import numpy as np
import pytest

from oracle import rkc


@pytest.mark.parametrize("x", [1.0 + 2 / 13 / 100, 1.3, 0.37, -0.81])
def test_chebyshev_recurrence_closed_forms(x):
    s = 25
    T, dT, d2T = rkc.chebyshev_T(x, s)
    for j in range(s + 1):
        if x > 1:
            t = math.acosh(x)
            Tj = math.cosh(j * t)
            dTj = j * math.sinh(j * t) / math.sinh(t)
            d2Tj = j * (j * math.cosh(j * t) * math.sinh(t) - math.sinh(j * t) * math.cosh(t)) / math.sinh(t) ** 3
        else:
            t = math.acos(x)
            Tj = math.cos(j * t)
            dTj = j * math.sin(j * t) / math.sin(t)
            d2Tj = j * (math.sin(j * t) * math.cos(t) - j * math.cos(j * t) * math.sin(t)) / math.sin(t) ** 3
        assert T[j] == pytest.approx(Tj, rel=1e-11, abs=1e-11)
        assert dT[j] == pytest.approx(dTj, rel=1e-10, abs=1e-10)
        assert d2T[j] == pytest.approx(d2Tj, rel=1e-9, abs=1e-8)


@pytest.mark.parametrize("s", [2, 3, 10, 20])
def test_stage_recurrence_matches_stability_polynomial(s):
    c = rkc.RKCCoefficients(s)
    z = np.linspace(-c.beta, 0.0, 257)
    lam = z  # dt = 1
    F = lambda t, y: lam * y
    y1, calls = rkc.rkc_step(F, 0.0, np.ones_like(z), 1.0, c)
    np.testing.assert_allclose(y1, c.stability_poly(z), rtol=1e-9, atol=1e-12)
    for k, (_, Fk) in enumerate(calls):
        nz = z != 0
        np.testing.assert_allclose(Fk[nz] / lam[nz], c.stability_poly(z[nz], k), rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("s", [3, 10, 20])
def test_second_order_and_stability_interval(s):
    c = rkc.RKCCoefficients(s)
    for z in (1e-2, -1e-2, 2e-3):
        P = float(c.stability_poly(z))
        assert abs(P - (1 + z + z * z / 2)) <= 0.2 * abs(z) ** 3 * s ** 4
    zz = np.linspace(-c.beta, 0, 4001)
    assert np.max(np.abs(c.stability_poly(zz))) <= 1 + 1e-12
    if s >= 10:  # for few stages the true boundary lies somewhat beyond beta_s
        assert abs(float(c.stability_poly(-1.05 * c.beta))) > 1.0
    eps = rkc.DAMPING
    approx = 2.0 / 3.0 * (s * s - 1) * (1 - 2.0 * eps / 15.0)
    assert c.beta == pytest.approx(approx, rel=0.01 if s > 3 else 0.1)
    assert c.c[s] == pytest.approx(1.0, rel=1e-14)
    assert np.all(np.diff(c.c) > 0)


@pytest.mark.parametrize("s", [3, 10])
def test_order_two_time_dependent(s):
    """Nonlinear, non-autonomous scalar ODE: error ratios under step halving
    tend to 4 (second order), which also pins the stage times c_j."""
    F = lambda t, y: -(y - np.cos(t)) - np.sin(t) + 0.5 * y * y * np.sin(t)
    c = rkc.RKCCoefficients(s)

    def run(n):
        y, t, dt = np.array([1.0]), 0.0, 2.0 / n
        for _ in range(n):
            y, _ = rkc.rkc_step(F, t, y, dt, c)
            t += dt
        return y[0]

    ref = run(4096)
    errs = [abs(run(n) - ref) for n in (8, 16, 32, 64)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.8 < r < 4.4 for r in ratios), ratios
