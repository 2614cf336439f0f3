"""Pins of the oracle's semi-discrete system (Eq. 2) and full integrator."""
import numpy as np
import pytest
import scipy.linalg as sla

import eqs_inputs as ei
from oracle import dtbound, fem, rkc, system


def _homog(N, kappa=1e-9, eps_r=3.0, V0=0.0, jitter=0.0):
    p = ei.make_problem(N, varistor="none", V0=V0, jitter=jitter, seed=11)
    p.materials = (ei.Material(eps_r, kappa, kappa),)
    return p


def test_lift_is_linear_in_z():
    """Homogeneous slab, sides natural: M_ff^-1 (-M_fd 1_top) = z/L exactly."""
    p = _homog(5, jitter=0.2)
    S = system.EQSSystem(p)
    H = S.solve_direct(-S.m_top)
    np.testing.assert_allclose(H, p.xyz[S.free, 2] / ei.L_CUBE, rtol=1e-12, atol=1e-13)


def test_homogeneous_relaxation_discrete_closed_form():
    """Uniform eps, kappa: M_ff^-1 K_ff = (kappa/eps) I, so with g = 0 the RKC
    step multiplies by P_s(-dt kappa/eps) exactly."""
    p = _homog(4, jitter=0.2)
    S = system.EQSSystem(p)
    rng = np.random.default_rng(5)
    x0 = rng.standard_normal(p.n_free)
    lam = 1e-9 / (3.0 * fem.EPS0)
    for s in (3, 10):
        c = rkc.RKCCoefficients(s)
        dt = 0.7 * c.beta / lam
        x, t = x0.copy(), 0.0
        for _ in range(4):
            x, _ = rkc.rkc_step(S.F, t, x, dt, c)
            t += dt
        np.testing.assert_allclose(x, float(c.stability_poly(-dt * lam)) ** 4 * x0,
                                   rtol=1e-10, atol=1e-12 * np.abs(x0).max())


def test_driven_slab_second_order():
    """Driven homogeneous slab started on its lift: x_f(t) = (z/L) g(t) exactly
    (u = x_f - Hg obeys u' = -(kappa/eps) u, u(0) = 0).  RKC errors against
    it fall 4x per step halving."""
    p = _homog(3, kappa=1e-9, V0=1e4)
    S = system.EQSSystem(p)
    zf = p.xyz[S.free, 2] / ei.L_CUBE
    T = 0.004
    exact = zf * (p.V0 * np.sin(2 * np.pi * p.freq * T))
    for s in (4, 10):
        c = rkc.RKCCoefficients(s)
        errs = []
        for n in (8, 16, 32):
            x, t, dt = np.zeros(p.n_free), 0.0, T / n
            for _ in range(n):
                x, _ = rkc.rkc_step(S.F, t, x, dt, c)
                t += dt
            errs.append(np.abs(x - exact).max())
        r = [errs[0] / errs[1], errs[1] / errs[2]]
        assert all(3.9 < v < 4.2 for v in r), r


def test_stability_bound_against_generalised_eigenvalues():
    """rho_bound >= lambda_max(J_ff, M_ff); tight for an all-varistor slab at
    the peak field."""
    mats = (ei.BACKGROUND, ei.VARISTOR)
    rho = dtbound.rho_bound(mats)
    assert rho == pytest.approx(2.9153e4, rel=1e-4)
    p = ei.make_problem(3, varistor="block", block=(-1, 2))  # every tet varistor
    S = system.EQSSystem(p)
    for Emag in (1e5, 5.195e5, 8e5):
        x = -Emag * p.xyz[:, 2]
        J = fem.assemble_dKx(p.xyz, p.tets, p.tet_mat, p.materials, x)
        Jff = J[S.free][:, S.free].toarray()
        lam = sla.eigh(Jff, S.Mff.toarray(), eigvals_only=True)
        assert lam.max() <= rho * (1 + 1e-9)
        if Emag == 5.195e5:
            assert lam.max() >= 0.95 * rho


def test_step_at_bound_is_stable_beyond_is_not():
    """Constant kappa = max sigma_d: dt = beta/rho keeps |x| bounded, 1.05x grows."""
    sig = dtbound.max_sigma_d(ei.VARISTOR.as_tuple())
    p = _homog(3, kappa=sig, eps_r=12.0)
    S = system.EQSSystem(p)
    rho = sig / (12.0 * fem.EPS0)
    c = rkc.RKCCoefficients(10)
    x0 = np.random.default_rng(1).standard_normal(p.n_free)
    for fac, grows in ((1.0, False), (1.05, True)):
        x, t = x0.copy(), 0.0
        for _ in range(20):
            x, _ = rkc.rkc_step(S.F, t, x, fac * c.beta / rho, c)
            t += fac * c.beta / rho
        assert (np.abs(x).max() > 10 * np.abs(x0).max()) == grows


def test_nonlinear_switching_run_is_second_order_against_radau():
    """The nonlinear system (Eq. 2 with the field-dependent varistor
    conductivity) stepped by the oracle's RKC scheme (Section II, s = 10)
    converges at second order to an independent stiff integrator (SciPy's
    Radau IIA at rtol 1e-12) over ten steps of the stability-bound size, on
    a drive strong enough that the varistor switches (its field passes E0
    and its conductivity rises by orders of magnitude).  A dropped stage
    term, a wrong stage time or a wrong coefficient breaks the order."""
    from scipy.integrate import solve_ivp

    p = ei.make_problem(3, V0=2e5)
    Sy = system.EQSSystem(p)
    s = 10
    coef = rkc.RKCCoefficients(s)
    T = 10 * dtbound.dt_bound(p.materials, s, coef)
    ref = solve_ivp(lambda t, y: Sy.F(t, y), (0.0, T), np.zeros(p.n_free), method="Radau", rtol=1e-12,
                    atol=1e-9)
    assert ref.status == 0
    kap, _ = fem.tet_kappa(p.xyz, p.tets, p.tet_mat, p.materials, Sy.full(T, ref.y[:, -1]))
    lo = min(m.kappa_lo for m in p.materials if m.kappa_hi != m.kappa_lo)
    assert kap.max() > 1e3 * lo  # switched
    yT = ref.y[:, -1]
    errs = []
    for n in (10, 20, 40):
        dt = T / n
        xf, t = np.zeros(p.n_free), 0.0
        for _ in range(n):
            xf, _ = rkc.rkc_step(Sy.F, t, xf, dt, coef)
            t += dt
        errs.append(np.linalg.norm(xf - yT) / np.linalg.norm(yT))
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert errs[0] < 0.1
    assert all(3.5 < r < 4.7 for r in ratios), (errs, ratios)
