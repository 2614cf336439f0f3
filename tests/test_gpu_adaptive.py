"""Adaptive RKC stepping (local error control of the scheme of ref. [9]) on
the GPU against the oracle's adaptive stepping."""
import os

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import dtbound, rkc, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_09447_gb300 import build, eqs
    if not os.path.exists(build.LIB):
        build.build()
    return eqs


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6)])
def test_adaptive_steps_match_oracle(E, prec, tol):
    """Same stage counts, tries and step sizes as the oracle, and the same
    states; the first try from a too large step is rejected."""
    p = ei.config_problem(0)
    S = E.Solver(p, precision=prec, rtol=1e-13)
    Sy = system.EQSSystem(p)
    rho = dtbound.rho_bound(p.materials)
    atol, rtol = 1e-4 * p.V0, 1e-4
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    xf = np.zeros(p.n_free)
    F0 = Sy.F(0.0, xf)
    t_g, t_o, h_g, h_o = 0.0, 0.0, 5e-3, 5e-3
    for k in range(5):
        st = E.eqs_rkc_adaptive_step(S.ctx, x, t_g, h_g, atol, rtol, 20)
        xf, F0, hu, s, err, hn, tries = rkc.rkc_adaptive_step(Sy.F, t_o, xf, F0, h_o, rho, atol, rtol, 20)
        assert st.s == s and st.tries == tries, (k, st.s, s, st.tries, tries)
        assert st.h_used == pytest.approx(hu, rel=1e-9)
        assert st.err == pytest.approx(err, rel=1e-4 if prec else 1e-7)
        assert st.err <= 1.0
        t_g += st.h_used
        t_o += hu
        h_g, h_o = st.h_next, hn
        got = x.cpu().numpy()
        ref = Sy.full(t_o, xf)
        assert np.linalg.norm(got - ref) <= tol * max(np.linalg.norm(ref), 1.0)
        if k == 0:
            assert tries > 1  # 5 ms is far too long for a local error of 1e-4
    S.close()


def test_adaptive_rejects_bad_arguments(E):
    p = ei.make_problem(3)
    S = E.Solver(p)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    for args in ((0.0, 0.0, 1e-3, 1e-3, 10), (0.0, 1e-3, 0.0, 0.0, 10), (0.0, 1e-3, 1e-3, 1e-3, 1)):
        with pytest.raises(E.EqsError) as ex:
            E.eqs_rkc_adaptive_step(S.ctx, x, *args)
        assert ex.value.status == E.EQS_ERR_ARG
    S.close()
