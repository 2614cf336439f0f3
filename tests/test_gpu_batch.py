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


def test_batch_spe_matches_solo_and_oracle(E):
    """Batched instances starting every solve from their SPE vectors (the
    Gram pass and small solve inside each instance's CTA group) against the
    same instances stepped alone with SPE, and one against the oracle; the
    SPE starts take fewer CG iterations than the previous-solution starts."""
    probs = _instances(6)
    s, steps = 10, 4
    iters = {}
    for guess in (E.EQS_GUESS_PREV, E.EQS_GUESS_SPE):
        solvers = [E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-12, spe_n=6) for p in probs]
        for S in solvers:
            E.eqs_set_guess(S.ctx, guess)
        b = E.eqs_batch_create([S.ctx for S in solvers], 128)
        dt = solvers[0].dt_bound(s)
        xs = [torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda") for p in probs]
        t, tot = 0.0, 0
        for _ in range(steps):
            st = E.eqs_batch_rkc_step(b, xs, t, dt, s)
            assert st.status == 0 and st.max_relres <= 1e-12
            tot += st.total_iters
            t += dt
        iters[guess] = tot
        E.eqs_batch_destroy(b)
        if guess == E.EQS_GUESS_SPE:
            for k, p in enumerate(probs):
                solo = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-12, spe_n=6)
                E.eqs_set_guess(solo.ctx, E.EQS_GUESS_SPE)
                x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
                tt = 0.0
                for _ in range(steps):
                    solo.step(x, tt, dt, s)
                    tt += dt
                got, ref = xs[k].cpu().numpy(), x.cpu().numpy()
                assert np.abs(got - ref).max() <= 1e-7 * np.abs(ref).max(), k
                solo.close()
            p = probs[2]
            Sy = system.EQSSystem(p)
            coef = rkc.RKCCoefficients(s)
            xf, tt = np.zeros(p.n_free), 0.0
            for _ in range(steps):
                xf, _ = rkc.rkc_step(Sy.F, tt, xf, dt, coef)
                tt += dt
            ref = Sy.full(tt, xf)
            assert np.linalg.norm(xs[2].cpu().numpy() - ref) <= 1e-6 * np.linalg.norm(ref)
        for S in solvers:
            S.close()
    assert iters[E.EQS_GUESS_SPE] < iters[E.EQS_GUESS_PREV]


def test_batch_barrier_timeout_then_recovers(E):
    """A group-barrier wait budget of one poll runs out during a batched step
    (instances spread over many CTAs): the step reports EQS_ERR_TIMEOUT and
    every CTA returns.  With the default budget restored, the same batch
    steps again from the saved state and matches the solo runs."""
    probs = _instances(4)
    s = 10
    solvers = [E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-10) for p in probs]
    b = E.eqs_batch_create([S.ctx for S in solvers], 32)
    dt = solvers[0].dt_bound(s)
    xs = [torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda") for p in probs]
    E.eqs_batch_rkc_step(b, xs, 0.0, dt, s)
    saved = [x.clone() for x in xs]
    E.eqs_batch_set_barrier_polls(b, 1)
    with pytest.raises(E.EqsError) as ex:
        E.eqs_batch_rkc_step(b, xs, dt, dt, s)
    assert ex.value.status == E.EQS_ERR_TIMEOUT
    E.eqs_batch_set_barrier_polls(b, 0)
    for x, sv in zip(xs, saved):
        x.copy_(sv)
    st = E.eqs_batch_rkc_step(b, xs, dt, dt, s)
    assert st.status == 0
    for k, p in enumerate(probs):
        solo = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-10)
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        solo.step(x, 0.0, dt, s)
        solo.step(x, dt, dt, s)
        got, ref = xs[k].cpu().numpy(), x.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-7 * np.abs(ref).max(), k
        solo.close()
    E.eqs_batch_destroy(b)
    for S in solvers:
        S.close()


@pytest.mark.parametrize("opts", [dict(cheb_degree=1, coarse_max=300), dict(cheb_degree=2, coarse_max=2500)])
def test_every_autotune_candidate_gives_the_solo_result(E, opts):
    """Every launch candidate of the autotuner (rows per CTA of the batched
    launch) and every solver-option candidate it chooses between gives the
    batched result of the solo runs, SPE start vectors on (the tuner only
    picks among equal answers)."""
    from paper_1612_09447_gb300 import autotune

    probs = _instances(5)
    s, steps = 10, 2
    solvers = [E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-12, fill_lanes=0, spe_n=6, **opts) for p in probs]
    for S in solvers:
        E.eqs_set_guess(S.ctx, E.EQS_GUESS_SPE)
    dt = solvers[0].dt_bound(s)
    refs = []
    for p in probs:
        solo = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-12, spe_n=6, **opts)
        E.eqs_set_guess(solo.ctx, E.EQS_GUESS_SPE)
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        for k in range(steps):
            solo.step(x, k * dt, dt, s)
        refs.append(x.cpu().numpy())
        solo.close()
    for rpb in (64, 256, 1024, 4096):
        b = E.eqs_batch_create([S.ctx for S in solvers], rpb)
        xs = [torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda") for p in probs]
        for k in range(steps):
            st = E.eqs_batch_rkc_step(b, xs, k * dt, dt, s)
            assert st.status == 0
        for k in range(len(probs)):
            got = xs[k].cpu().numpy()
            assert np.abs(got - refs[k]).max() <= 1e-7 * np.abs(refs[k]).max(), (rpb, k)
        E.eqs_batch_destroy(b)
    best, res, _ = autotune.tune_batch(E, solvers, candidates=(128, 1024), s=s, steps=1, warmup=1, repeats=2)
    assert best in (128, 1024) and all(v[0] > 0 and v[1] >= 0 for v in res.values())
    for S in solvers:
        S.close()
