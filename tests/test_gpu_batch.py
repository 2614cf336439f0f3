"""Batched serving: every instance of a batched step matches its solo run."""
import os

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import rkc, system

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


def _instances(k):
    """Reduced-size instances of the batched-serving recipe (seeded sizes,
    block fractions and amplitudes; N scaled down to 5..9)."""
    out = []
    for i in range(k):
        Ni, _, _ = ei.batch_instance_params(i)
        out.append(ei.config_problem(4, N=5 + (Ni - 16) // 8, instance=i))
    return out


@pytest.mark.parametrize("rows_per_block", [64, 512])
def test_batch_matches_solo_and_oracle(E, rows_per_block):
    probs = _instances(7)
    s, steps = 10, 3
    solvers = [E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-12) for p in probs]
    solos = [E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-12) for p in probs]
    b = E.eqs_batch_create([S.ctx for S in solvers], rows_per_block)
    tb, rpb = E.eqs_batch_info(b)
    assert tb >= len(probs)
    dt = solvers[0].dt_bound(s)
    xs = [torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda") for p in probs]
    xsolo = [torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda") for p in probs]
    t = 0.0
    for _ in range(steps):
        st = E.eqs_batch_rkc_step(b, xs, t, dt, s)
        assert st.status == 0 and st.max_relres <= 1e-12 and st.total_iters > 0
        assert st.launches == s + 2  # drive table + s stages + last recurrence
        for S, x in zip(solos, xsolo):
            S.step(x, t, dt, s)
        t += dt
    for k, p in enumerate(probs):
        got, ref = xs[k].cpu().numpy(), xsolo[k].cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-7 * np.abs(ref).max(), k
    # one instance against the FP64 oracle (mixed-precision bar)
    p = probs[3]
    Sy = system.EQSSystem(p)
    coef = rkc.RKCCoefficients(s)
    xf, tt = np.zeros(p.n_free), 0.0
    for _ in range(steps):
        xf, _ = rkc.rkc_step(Sy.F, tt, xf, dt, coef)
        tt += dt
    ref = Sy.full(tt, xf)
    assert np.linalg.norm(xs[3].cpu().numpy() - ref) <= 1e-6 * np.linalg.norm(ref)
    E.eqs_batch_destroy(b)
    for S in solvers + solos:
        S.close()


def test_batch_rejects_fp64_contexts(E):
    p = _instances(1)[0]
    S = E.Solver(p, precision=E.EQS_PREC_FP64)
    with pytest.raises(E.EqsError):
        E.eqs_batch_create([S.ctx], 256)
    S.close()
