"""Pins of the oracle's SPE start vector (Section IV, Eq. 4-5)."""
import numpy as np

import eqs_inputs as ei
from oracle import spe, system


def _M():
    return system.EQSSystem(ei.make_problem(4, jitter=0.2, seed=2)).Mff


def test_mgs_orthonormal_span_and_dropping():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((200, 4))
    V = spe.mgs(X)
    np.testing.assert_allclose(V.T @ V, np.eye(4), atol=1e-13)
    # span preserved: X = V (V^T X)
    np.testing.assert_allclose(V @ (V.T @ X), X, atol=1e-12)
    Xd = np.column_stack([X[:, 0], X[:, 1], X[:, 0] + 2 * X[:, 1], X[:, 2]])
    assert spe.mgs(Xd).shape[1] == 3


def test_reproduces_solution_in_span():
    M = _M()
    rng = np.random.default_rng(1)
    H = [rng.standard_normal(M.shape[0]) for _ in range(4)]
    x = 0.3 * H[0] - 1.2 * H[2] + 0.5 * H[3]
    x0 = spe.spe_start(M, H, M @ x)
    np.testing.assert_allclose(x0, x, rtol=1e-10, atol=1e-10 * np.abs(x).max())


def test_error_is_M_orthogonal_and_order_free():
    M = _M()
    rng = np.random.default_rng(2)
    H = [rng.standard_normal(M.shape[0]) for _ in range(5)]
    xs = rng.standard_normal(M.shape[0])
    b = M @ xs
    x0 = spe.spe_start(M, H, b)
    X = np.stack(H, axis=1)
    np.testing.assert_allclose(X.T @ (M @ (xs - x0)), 0, atol=1e-10 * np.abs(X.T @ b).max())
    x1 = spe.spe_start(M, H[::-1], b)
    np.testing.assert_allclose(x1, x0, rtol=1e-9, atol=1e-9 * np.abs(x0).max())
    assert not spe.spe_start(M, [], b).any()
