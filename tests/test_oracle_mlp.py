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


def test_adam_second_step_bias_correction():
    """Hand-computed second Adam step (Kingma & Ba, Algorithm 1) of a scalar
    with gradients g1 = 1, g2 = -1: m2 = 0.9*0.1 - 0.1 = -0.01, so the
    bias-corrected m2 / (1 - 0.9^2) = -1/19; v2 = 0.999*0.001 + 0.001 =
    0.001999 = 1 - 0.999^2, so the corrected v2 is 1.  The step is
    +lr/19/(1 + eps).  With g2 = +1 both corrected moments are 1."""
    lr, eps = 1e-3, 1e-8
    th1, m, v = mlp.adam_step(np.array([0.5]), np.array([1.0]), np.zeros(1), np.zeros(1), 1, lr=lr, eps=eps)
    th2, m2, v2 = mlp.adam_step(th1, np.array([-1.0]), m, v, 2, lr=lr, eps=eps)
    assert m2[0] == pytest.approx(-0.01, rel=1e-14)
    assert v2[0] == pytest.approx(0.001999, rel=1e-13)
    assert th2[0] - th1[0] == pytest.approx(lr / 19.0 / (1.0 + eps), rel=1e-10)
    th2b, _, _ = mlp.adam_step(th1, np.array([1.0]), m, v, 2, lr=lr, eps=eps)
    assert th2b[0] - th1[0] == pytest.approx(-lr / (1.0 + eps), rel=1e-10)
    # third step, g3 = 0: m3 = 0.9 m2, v3 = 0.999 v2; corrected with 1 - b^3
    th3, _, _ = mlp.adam_step(th2, np.array([0.0]), m2, v2, 3, lr=lr, eps=eps)
    mh = 0.9 * -0.01 / (1 - 0.9 ** 3)
    vh = 0.999 * 0.001999 / (1 - 0.999 ** 3)
    assert th3[0] - th2[0] == pytest.approx(-lr * mh / (math.sqrt(vh) + eps), rel=1e-10)


def test_spe_correction_inputs_and_line_search():
    """SPE-correction mode: inputs are increments (adding one vector to x0
    and every h changes neither inputs nor scale), the 1-ring columns are
    the means of the increment columns; the zero output layer gives no
    direction and returns x0; the line search never increases the M-norm
    error (any direction) and returns the solution exactly when the
    direction is the error itself (alpha = 1 for d = z - x0, alpha = 1/2
    for d = 2(z - x0))."""
    p = ei.make_problem(4)
    S = system.EQSSystem(p)
    A = mlp.free_adjacency(p.tets, S.free, p.n_nodes)
    rng = np.random.default_rng(6)
    n = p.n_free
    H = [np.sin(np.arange(n) * 0.1 + k) + 0.01 * rng.standard_normal(n) for k in range(4)]
    x0 = H[0] + 0.02 * rng.standard_normal(n)
    X, s = mlp.spe_features(A, x0, H)
    assert s == pytest.approx(np.sqrt(np.mean((x0 - H[0]) ** 2)))
    np.testing.assert_allclose(X[:, 0] * s, x0 - H[0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(X[:, 3] * s, H[2] - H[3], rtol=0, atol=1e-15)
    D = A.toarray()
    i = 7
    nb = np.nonzero(D[i])[0]
    assert X[i, 5] * s == pytest.approx(np.mean(H[0][nb] - H[1][nb]))
    off = 3.7 * np.cos(np.arange(n))
    X2, s2 = mlp.spe_features(A, x0 + off, [h + off for h in H])
    assert s2 == pytest.approx(s, rel=1e-12)
    np.testing.assert_allclose(X2, X, rtol=0, atol=1e-9)
    R = rng.standard_normal(n)
    z = S.solve_direct(R)
    z0, alpha = mlp.spe_corrected_start(S.Mff, ei.mlp_init(), A, x0, H, R)
    assert alpha == 0.0 and np.array_equal(z0, x0)

    def err_M(v):
        e = v - z
        return float(e @ (S.Mff @ e))

    th = _theta(3)
    z1, _ = mlp.spe_corrected_start(S.Mff, th, A, x0, H, R)
    assert err_M(z1) <= err_M(x0) * (1 + 1e-12)
    for scale, want in ((1.0, 1.0), (2.0, 0.5)):
        d = scale * (z - x0)
        alpha = float(d @ (R - S.Mff @ x0)) / float(d @ (S.Mff @ d))
        assert alpha == pytest.approx(want, rel=1e-9)
    T = mlp.spe_target(z, x0)
    assert np.sqrt(np.mean(T * T)) == pytest.approx(1.0)
    np.testing.assert_allclose(T * np.sqrt(np.mean((z - x0) ** 2)), z - x0, rtol=1e-12, atol=0)


def test_features_hand_computed_on_a_path_graph():
    """Inputs of the previous-solution mode on the free path graph 0-1-2:
    columns h1..h4 and their neighbour means, all divided by s_h = RMS(h1)
    (values worked out by hand; a normalisation by another history vector
    or a ring mean that counted the node itself would differ)."""
    import scipy.sparse as sp

    A = sp.csr_matrix(np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]], dtype=float))
    H = [np.array([3.0, 0.0, 4.0]), np.array([1.0, 2.0, 3.0]), np.array([0.0, 0.0, 6.0]),
         np.array([-2.0, 2.0, 0.0])]
    X, s_h = mlp.features(A, H)
    assert s_h == pytest.approx(math.sqrt(25.0 / 3.0), rel=1e-15)
    means = [np.array([0.0, 3.5, 0.0]), np.array([2.0, 2.0, 2.0]), np.array([0.0, 3.0, 0.0]),
             np.array([2.0, -1.0, 2.0])]
    want = np.stack(H + means, axis=1) / math.sqrt(25.0 / 3.0)
    np.testing.assert_allclose(X, want, rtol=1e-15, atol=0)
    # z0 = h1 + s_h o: an output layer with bias b alone shifts h1 by s_h b
    th = ei.mlp_init().astype(np.float64)
    th[1376] = 0.5  # output bias (a BF16-exact value)
    np.testing.assert_allclose(mlp.guess(th, A, H), H[0] + 0.5 * math.sqrt(25.0 / 3.0), rtol=1e-15)
