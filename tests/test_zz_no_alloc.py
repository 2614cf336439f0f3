"""eqs_apply_K_static, the allocation-free variant of eqs_apply_K.

Some callers cannot allocate device memory at call time (a fixed device
memory budget claimed up front, a real-time or callback path where an
allocation may block or fail); this entry point serves them from a static
device array inside the library.  Checked here through the C ABI against
eqs_apply_K on two calls in a row, for linear tets (the Kuhn-cell and the
jittered mesh) and quadratic (10-node) tets.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import os

import numpy as np
import pytest

import eqs_inputs as ei

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


def _state(p, seed):
    rng = np.random.default_rng(seed)
    x = -5.2e5 * p.xyz[:, 2] + 0.3 * 5.2e5 * (0.1 / p.N) * rng.standard_normal(p.n_nodes)
    return torch.tensor(x, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
@pytest.mark.parametrize("problem", ["cube12", "jitter10", "p2_cube8"])
def test_static_matches_apply_K_twice(E, prec, tol, problem):
    p = {"cube12": lambda: ei.config_problem(0), "jitter10": lambda: ei.config_problem(2, N=10),
         "p2_cube8": lambda: ei.make_problem_p2(8)}[problem]()
    S = E.Solver(p, precision=prec)
    for seed in (11, 12):  # two calls in a row: the shared scratch is reused
        x = _state(p, seed)
        y_ref = torch.empty_like(x)
        y_static = torch.full_like(x, float("nan"))
        E.eqs_apply_K(S.ctx, x, y_ref)
        E.eqs_apply_K_static(S.ctx, x, y_static)
        torch.cuda.synchronize()
        ref = y_ref.cpu().numpy()
        got = y_static.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    S.close()


def test_static_rejects_too_many_nodes(E):
    p = ei.make_problem(80)  # 531441 nodes > 524288
    ctx = E.eqs_mesh_create(p.xyz, p.tets, p.node_tag)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EqsError) as ex:
        E.eqs_apply_K_static(ctx, x, x)
    assert ex.value.status == E.EQS_ERR_ARG
    assert "524288" in str(ex.value)
    E.eqs_destroy(ctx)
