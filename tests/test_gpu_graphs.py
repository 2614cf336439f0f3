"""Step graphs and the one-kernel launch entry point.

The captured step reads and writes the caller's x through the per-call
parameter block, so one graph per stage count serves every x buffer: a run
that hands a different buffer to every step must equal a run with one
buffer.  eqs_launch_kernel enqueues one kernel of the last step alone (for
timing) and leaves later steps unaffected."""
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


@pytest.mark.parametrize("prec", [0, 1])
def test_fresh_buffer_every_step(E, prec):
    p = ei.config_problem(0)
    s, steps = 10, 4
    A = E.Solver(p, precision=prec, rtol=1e-12)
    B = E.Solver(p, precision=prec, rtol=1e-12)
    dt = A.dt_bound(s)
    xa = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    xb = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    t = 0.0
    for _ in range(steps):
        A.step(xa, t, dt, s)
        xb = xb.clone()  # a new allocation: another device address
        B.step(xb, t, dt, s)
        t += dt
    a, b = xa.cpu().numpy(), xb.cpu().numpy()
    tol = 1e-12 if prec == 0 else 1e-6
    assert np.abs(a - b).max() <= tol * np.abs(a).max()
    A.close()
    B.close()


def test_ensemble_fresh_buffer_every_step(E):
    p = ei.config_problem(0)
    s = 10
    A = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-12)
    B = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-12)
    dt = A.dt_bound(s)
    scales = (0.5, 1.0, 1.5, 2.0)
    xa = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    xb = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    t = 0.0
    for _ in range(3):
        E.eqs_ens_rkc_step(A.ctx, xa, scales, t, dt, s)
        xb = xb.clone()
        E.eqs_ens_rkc_step(B.ctx, xb, scales, t, dt, s)
        t += dt
    a, b = xa.cpu().numpy(), xb.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
    A.close()
    B.close()


def test_launch_kernel(E):
    p = ei.config_problem(0)
    s = 10
    S = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-10, spe_n=6)
    E.eqs_set_guess(S.ctx, E.EQS_GUESS_SPE)
    with pytest.raises(E.EqsError) as ex:  # no step yet
        E.eqs_launch_kernel(S.ctx, E.EQS_KERNEL_ELEM)
    assert ex.value.status == E.EQS_ERR_STATE
    ref = E.Solver(p, precision=E.EQS_PREC_MIXED, rtol=1e-10, spe_n=6)
    E.eqs_set_guess(ref.ctx, E.EQS_GUESS_SPE)
    dt = S.dt_bound(s)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    xr = torch.zeros_like(x)
    S.step(x, 0.0, dt, s)
    ref.step(xr, 0.0, dt, s)
    for kid in (E.EQS_KERNEL_SPE_GRAM, E.EQS_KERNEL_ELEM, E.EQS_KERNEL_PCG_PQ):
        for _ in range(3):
            E.eqs_launch_kernel(S.ctx, kid)
    with pytest.raises(E.EqsError) as ex:
        E.eqs_launch_kernel(S.ctx, 99)
    assert ex.value.status == E.EQS_ERR_ARG
    with pytest.raises(E.EqsError) as ex:  # no ensemble step yet
        E.eqs_launch_kernel(S.ctx, E.EQS_KERNEL_ENS_PCG_PQ)
    assert ex.value.status == E.EQS_ERR_STATE
    # the next step is unaffected by the lone launches
    st = S.step(x, dt, dt, s)
    ref.step(xr, dt, dt, s)
    assert st.status == 0
    a, b = x.cpu().numpy(), xr.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max()
    # ensemble kernels after an ensemble step
    X = torch.zeros((4, p.n_nodes), dtype=torch.float64, device="cuda")
    E.eqs_ens_rkc_step(S.ctx, X, (0.5, 1.0, 1.5, 2.0), 0.0, dt, s)
    for kid in (E.EQS_KERNEL_ENS_SPE_GRAM, E.EQS_KERNEL_ENS_ELEM, E.EQS_KERNEL_ENS_PCG_PQ):
        E.eqs_launch_kernel(S.ctx, kid)
    torch.cuda.synchronize()
    S.close()
    ref.close()


def test_integer_widening_is_exact(E):
    """The CG kernels' FP32 -> FP64 widening by integer operations equals the
    exact conversion bit for bit: random values over the whole exponent
    range, zeros of both signs, the smallest and largest normals,
    subnormals, infinities and NaN."""
    rng = np.random.default_rng(21)
    n = 1 << 20
    bits = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32).copy()
    edges = np.array([0.0, -0.0, 1.0, -1.5, np.finfo(np.float32).max, np.finfo(np.float32).tiny,
                      np.float32(1e-40), -np.float32(1e-45), np.inf, -np.inf, np.nan], dtype=np.float32)
    f[: len(edges)] = edges
    with np.errstate(invalid="ignore"):  # the random bit patterns include NaNs
        want = f.astype(np.float64)
    fw = torch.empty(n, dtype=torch.float64, device="cuda")
    E.eqs_convert_check(torch.tensor(f, device="cuda"), fw)
    got = fw.cpu().numpy()
    ok = (got.view(np.uint64) == want.view(np.uint64)) | (np.isnan(got) & np.isnan(want))
    assert ok.all(), f[~ok][:5]
