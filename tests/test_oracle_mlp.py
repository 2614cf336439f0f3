"""Pins of the oracle's learned start-vector network."""
import math

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import mlp, system


def _theta(seed=5, scale_out=0.3):
    th = ei.mlp_init(seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    th[256:288] = 0.1 * rng.standard_normal(32)
    th[1312:1344] = 0.1 * rng.standard_normal(32)
    th[1344:1376] = scale_out * rng.standard_normal(32)
    th[1376] = 0.05
    return th


def test_gelu_definition_and_derivative():
    x = np.array([-3.0, -1.0, -0.1, 0.0, 0.5, 2.0])
    want = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in x])
    np.testing.assert_allclose(mlp.gelu(x), want, rtol=1e-15, atol=1e-300)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, rtol=1e-8, atol=1e-10)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0 and mlp.gelu_grad(np.array([0.0]))[0] == 0.5


def test_gradient_against_central_differences():
    rng = np.random.default_rng(0)
    th = _theta()
    X = rng.standard_normal((64, 8))
    T = rng.standard_normal(64)

    def loss(t):  # full precision (no BF16) for the difference quotient
        o, _ = mlp.forward(t, X)
        return float(np.mean((o - T) ** 2))

    o, cache = mlp.forward(th, X)
    g = mlp.backward(th, cache, 2.0 * (o - T) / len(T))
    idx = np.r_[0:8, 250:262, 300:310, 1330:1340, 1344:1350, 1376]
    for k in idx:
        e = np.zeros_like(th)
        e[k] = 1e-6
        fd = (loss(th + e) - loss(th - e)) / 2e-6
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.14159], dtype=np.float32)
    b = mlp.to_bf16(v)
    assert b[0] == 1.0 and b[3] == -2.5
    assert b[1] == 1.0  # 1 + 2^-8 lies halfway; the even neighbour is 1.0
    assert b[2] == 1.0 + 2 ** -7  # above halfway rounds up
    assert abs(b[4] - 3.14159) <= 2 ** -7 * 4


def test_zero_output_layer_returns_previous_solution():
    p = ei.make_problem(3)
    S = system.EQSSystem(p)
    A = mlp.free_adjacency(p.tets, S.free, p.n_nodes)
    rng = np.random.default_rng(1)
    H = [rng.standard_normal(p.n_free) for _ in range(4)]
    z0 = mlp.guess(ei.mlp_init(), A, H)
    assert np.array_equal(z0, H[0])


def test_ring_means_against_dense_count():
    p = ei.make_problem(3)
    S = system.EQSSystem(p)
    A = mlp.free_adjacency(p.tets, S.free, p.n_nodes)
    # adjacency equals the off-diagonal structural pattern of M_ff
    pat = S.Mff.copy()
    pat.data[:] = 1.0
    pat.setdiag(0)
    pat.eliminate_zeros()
    assert (abs(pat - A)).max() == 0
    h = np.arange(p.n_free, dtype=float)
    m = mlp.ring_means(A, [h])[0]
    D = A.toarray()
    for i in (0, 5, p.n_free - 1):
        nb = np.nonzero(D[i])[0]
        assert m[i] == pytest.approx(h[nb].mean())


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(2)
    th = rng.standard_normal(10)
    g = rng.standard_normal(10)
    th1, m, v = mlp.adam_step(th, g, np.zeros(10), np.zeros(10), 1, lr=1e-3)
    np.testing.assert_allclose(th1, th - 1e-3 * np.sign(g), rtol=0, atol=1e-8)
