"""Pins of the oracle's POD-MOR start vectors (Section IV)."""
import numpy as np

import eqs_inputs as ei
from oracle import pod, system


def _M():
    return system.EQSSystem(ei.make_problem(4, jitter=0.2, seed=2)).Mff


def test_singular_values_match_gram_eigenvalues():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((300, 7)) @ np.diag([5, 3, 2, 1, 0.5, 0.1, 0.01])
    V, sig = pod.pod_basis(X, 7)
    lam = np.sort(np.linalg.eigvalsh(X.T @ X))[::-1]
    np.testing.assert_allclose(sig ** 2, lam, rtol=1e-10)
    np.testing.assert_allclose(V.T @ V, np.eye(7), atol=1e-12)


def test_eckart_young_projection_error():
    """Projecting the snapshots on the m leading modes leaves exactly the
    energy of the discarded singular values."""
    rng = np.random.default_rng(1)
    X = rng.standard_normal((250, 6)) * np.array([4.0, 2.0, 1.0, 0.3, 0.1, 0.05])
    for m in (1, 3, 5):
        V, sig = pod.pod_basis(X, m)
        err2 = np.linalg.norm(X - V @ (V.T @ X), "fro") ** 2
        np.testing.assert_allclose(err2, np.sum(sig[m:] ** 2), rtol=1e-9)


def test_rank_deficient_snapshots_are_truncated():
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal(100), rng.standard_normal(100)
    X = np.column_stack([a, b, a + 2 * b, 3 * a, b - a])  # rank 2
    V, _ = pod.pod_basis(X, 5)
    assert V.shape[1] == 2
    np.testing.assert_allclose(V @ (V.T @ X), X, atol=1e-12 * np.abs(X).max())


def test_start_reproduces_span_and_is_M_orthogonal():
    M = _M()
    rng = np.random.default_rng(3)
    X = rng.standard_normal((M.shape[0], 5))
    V, _ = pod.pod_basis(X, 5)
    x = X @ np.array([0.5, -1.0, 0.25, 2.0, -0.7])
    np.testing.assert_allclose(pod.pod_start(M, V, M @ x), x, rtol=1e-9, atol=1e-9 * np.abs(x).max())
    xs = rng.standard_normal(M.shape[0])
    V3, _ = pod.pod_basis(X, 3)
    x0 = pod.pod_start(M, V3, M @ xs)
    np.testing.assert_allclose(V3.T @ (M @ (xs - x0)), 0, atol=1e-10 * np.abs(V3.T @ (M @ xs)).max())
    assert not pod.pod_start(M, np.zeros((M.shape[0], 0)), M @ xs).any()


def test_mor_fixes_its_first_basis():
    M = _M()
    rng = np.random.default_rng(4)
    est = pod.MOR(M, K=3, m=2)
    prev = rng.standard_normal(M.shape[0])
    b = rng.standard_normal(M.shape[0])
    np.testing.assert_array_equal(est.start(b, prev), prev)  # no basis yet
    snaps = [rng.standard_normal(M.shape[0]) for _ in range(5)]
    for k, x in enumerate(snaps):
        est.after_solve(x, 10)
        if k == 2:
            V_first = est.V.copy()
    np.testing.assert_array_equal(est.V, V_first)  # later solutions do not change it
    V_ref, _ = pod.pod_basis(np.stack(snaps[:3], axis=1), 2)
    np.testing.assert_allclose(np.abs(V_first.T @ V_ref), np.eye(2), atol=1e-12)


def test_mor2_threshold_and_overwrite():
    M = _M()
    rng = np.random.default_rng(5)
    est = pod.MOR2(M, K=3, m=3, min_iters=4)
    xs = [rng.standard_normal(M.shape[0]) for _ in range(6)]
    est.after_solve(xs[0], 4)  # not above the threshold: ignored
    assert est.V is None and est.rebuilds == 0
    for x in xs[1:5]:
        est.after_solve(x, 9)
    assert est.rebuilds == 4 and len(est.snaps) == 3
    np.testing.assert_array_equal(est.snaps[0], xs[2])  # xs[1] was overwritten
    V_ref, _ = pod.pod_basis(np.stack(xs[2:5], axis=1), 3)
    np.testing.assert_allclose(est.V @ est.V.T, V_ref @ V_ref.T, atol=1e-12)
