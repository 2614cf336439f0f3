"""Failure paths on the GPU, made on the host side: an iteration limit that
runs out, a non-finite input, and grid-barrier waits with a zero budget.
None of them faults or hangs the device; the context stays usable."""
import os

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import fem

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


def _check_apply_K(E, S, p):
    x = np.random.default_rng(0).standard_normal(p.n_nodes) * 1e3
    got = S.apply_K(torch.tensor(x, dtype=torch.float64, device="cuda")).cpu().numpy()
    ref = fem.apply_K(p.xyz, p.tets, p.tet_mat, p.materials, x)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("persistent", [0, 1])
def test_iteration_limit_reports_noconv(E, persistent):
    p = ei.config_problem(0)
    S = E.Solver(p, rtol=1e-13, max_iter=2, persistent=persistent)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EqsError) as ex:
        S.step(x, 0.0, S.dt_bound(10), 10)
    assert ex.value.status == E.EQS_ERR_NOCONV
    R = torch.ones(p.n_free, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EqsError) as ex:
        S.solve_M(R)
    assert ex.value.status == E.EQS_ERR_NOCONV
    _check_apply_K(E, S, p)
    S.close()


def test_non_finite_input_reports_nan(E):
    p = ei.config_problem(0)
    S = E.Solver(p)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    x[p.n_nodes // 2] = float("nan")
    with pytest.raises(E.EqsError) as ex:
        S.step(x, 0.0, S.dt_bound(10), 10)
    assert ex.value.status == E.EQS_ERR_NAN
    _check_apply_K(E, S, p)
    S.close()


def test_barrier_wait_budget_reports_timeout(E):
    """Persistent solve whose barrier waits give up at once: every CTA
    returns, the host reads EQS_ERR_TIMEOUT, and the device keeps working."""
    p = ei.config_problem(0)
    S = E.Solver(p, persistent=1, barrier_polls=-1)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EqsError) as ex:
        S.step(x, 0.0, S.dt_bound(10), 10)
    assert ex.value.status == E.EQS_ERR_TIMEOUT
    _check_apply_K(E, S, p)
    S.close()
    S2 = E.Solver(p, persistent=1)  # the normal budget on the same device still solves
    st = S2.step(x.zero_(), 0.0, S2.dt_bound(10), 10)
    assert st.status == 0
    S2.close()
