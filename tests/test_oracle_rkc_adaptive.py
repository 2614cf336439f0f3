"""Pins of the oracle's adaptive RKC stepping (the local error control of
the scheme of ref. [9]; the paper runs with a local error below 1e-2)."""
import numpy as np
import pytest

import eqs_inputs as ei
from oracle import dtbound, rkc, system


@pytest.mark.parametrize("s", [2, 5, 13])
def test_estimate_vanishes_where_the_scheme_is_exact(s):
    """F = a + b t: the solution is quadratic in t, a second-order scheme
    reproduces it and the estimate (12 (y_n - y_n+1) + 6h (F_n + F_n+1))/15
    is zero."""
    a, b, h = 0.7, -1.3, 0.37
    F = lambda t, y: np.full_like(y, a + b * t)
    y0 = np.array([2.0])
    y1, _ = rkc.rkc_step(F, 0.4, y0, h, rkc.RKCCoefficients(s))
    exact = y0 + a * h + b * (0.4 * h + h * h / 2)
    np.testing.assert_allclose(y1, exact, rtol=1e-14)
    est = rkc.error_estimate(h, y0, y1, F(0.4, y0), F(0.4 + h, y1))
    assert abs(est[0]) <= 1e-14


def test_estimate_is_third_order():
    """F = t^2 (y''' = 2): Est = (2 h^3 - 12 le)/15 with le the step's local
    error; halving h divides it by 8."""
    F = lambda t, y: np.full_like(y, t * t)
    c = rkc.RKCCoefficients(7)
    ests = []
    for h in (0.2, 0.1, 0.05):
        y1, _ = rkc.rkc_step(F, 0.0, np.zeros(1), h, c)
        le = y1[0] - h ** 3 / 3
        est = rkc.error_estimate(h, np.zeros(1), y1, F(0.0, y1), F(h, y1))[0]
        assert est == pytest.approx((2 * h ** 3 - 12 * le) / 15, rel=1e-12)
        ests.append(est)
    assert ests[0] / ests[1] == pytest.approx(8.0, rel=1e-9)
    assert ests[1] / ests[2] == pytest.approx(8.0, rel=1e-9)


def test_stage_choice_against_brute_force():
    rho = 2.9153e4
    betas = {s: rkc.RKCCoefficients(s).beta for s in range(2, 41)}
    for h in np.geomspace(1e-6, 5e-2, 60):
        s, hh = rkc.stages_for(h, rho, 40)
        ok = [k for k in range(2, 41) if betas[k] >= h * rho]
        if ok:
            assert s == ok[0] and hh == h
        else:
            assert s == 40 and hh == pytest.approx(betas[40] / rho) and hh < h


def _integrate(F, y0, T, rho, tol, h0=1e-2):
    t, y, Fy, h, steps, rej = 0.0, y0.copy(), F(0.0, y0), h0, 0, 0
    while t < T - 1e-15:
        h = min(h, T - t)
        y, Fy, hu, s, err, h, tries = rkc.rkc_adaptive_step(F, t, y, Fy, h, rho, tol, tol)
        t += hu
        steps += 1
        rej += tries - 1
    return y, steps, rej


def test_global_error_and_step_counts_follow_second_order():
    F = lambda t, y: -(y - np.cos(t)) - np.sin(t) + 0.5 * y * y * np.sin(t)
    y0 = np.array([1.0])
    ref, _, _ = _integrate(F, y0, 2.0, 2.0, 1e-12, h0=1e-4)
    y4, n4, _ = _integrate(F, y0, 2.0, 2.0, 1e-4)
    y6, n6, _ = _integrate(F, y0, 2.0, 2.0, 1e-6)
    e4, e6 = abs(y4[0] - ref[0]), abs(y6[0] - ref[0])
    assert e6 < e4 and 5.0 < e4 / e6 < 200.0      # about 100^(2/3) = 21.5
    assert 3.0 < n6 / n4 < 7.0                    # about 100^(1/3) = 4.6


def test_rejection_shrinks_the_step():
    F = lambda t, y: -50.0 * (y - np.sin(t))
    y0 = np.array([0.0])
    y1, F1, h, s, err, hn, tries = rkc.rkc_adaptive_step(F, 0.0, y0, F(0.0, y0), 1.0, 50.0, 1e-8, 1e-8)
    assert tries > 1 and h < 0.8 and err <= 1.0


def test_eqs_relaxation_closed_form():
    """Homogeneous slab with g = 0: M_ff^-1 K_ff = (kappa/eps) I, so every
    component decays as exp(-kappa t / eps); adaptive RKC at a local error
    of 1e-6 follows it to about that accuracy."""
    p = ei.make_problem(4, varistor="none", V0=0.0, jitter=0.2, seed=11)
    p.materials = (ei.Material(3.0, 1e-9, 1e-9),)
    S = system.EQSSystem(p)
    rho = dtbound.rho_bound(p.materials)
    rng = np.random.default_rng(2)
    x0 = rng.standard_normal(p.n_free)
    tau = 3.0 * 8.8541878128e-12 / 1e-9
    y, steps, _ = _integrate(S.F, x0, 2 * tau, rho, 1e-6, h0=1e-3)
    np.testing.assert_allclose(y, x0 * np.exp(-2.0), rtol=2e-4, atol=2e-4 * np.abs(x0).max())
    assert steps >= 3
