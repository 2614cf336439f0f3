"""Seeded input generators: counts, volumes, generator test vector."""
import os

import numpy as np
import pytest

import eqs_inputs as ei


def _edges(N):
    return 3 * N * (N + 1) ** 2 + 3 * N * N * (N + 1) + N ** 3


def test_splitmix64_reference_sequence(golden_dir):
    want = [int(l, 16) for l in open(os.path.join(golden_dir, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    got = ei.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in got] == want


@pytest.mark.parametrize("N", [1, 2, 5, 12])
def test_kuhn_counts_and_volume(N):
    xyz, tets = ei.kuhn_cube(N)
    assert len(xyz) == (N + 1) ** 3 and len(tets) == 6 * N ** 3
    p = xyz[tets]
    J = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], axis=2)
    det = np.linalg.det(J)
    assert np.all(det > 0)
    assert abs(det.sum() / 6 - ei.L_CUBE ** 3) <= 1e-14 * ei.L_CUBE ** 3
    # conforming: every edge appears, #edges matches the closed count
    e = np.sort(tets[:, [[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3]]].reshape(-1, 2), axis=1)
    assert len(np.unique(e, axis=0)) == _edges(N)


def test_jitter_interior_only_and_volume():
    N = 10
    xyz0, _ = ei.kuhn_cube(N)
    xyz, tets = ei.kuhn_cube(N, jitter=0.2, seed=ei.mesh.CONFIG_SEED)
    moved = np.any(xyz != xyz0, axis=1)
    n1 = N + 1
    idx = np.arange(n1 ** 3)
    i, j, k = idx % n1, (idx // n1) % n1, idx // (n1 * n1)
    interior = (i > 0) & (i < N) & (j > 0) & (j < N) & (k > 0) & (k < N)
    assert np.array_equal(moved, interior)
    assert np.max(np.abs(xyz - xyz0)) <= 0.2 * ei.L_CUBE / N
    p = xyz[tets]
    J = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], axis=2)
    det = np.linalg.det(J)
    assert np.all(det > 0)
    assert abs(det.sum() / 6 - ei.L_CUBE ** 3) <= 1e-13 * ei.L_CUBE ** 3


def test_config_sizes():
    p0 = ei.config_problem(0)
    assert (p0.n_nodes, p0.n_tets, p0.n_free) == (2197, 10368, 1859)
    assert p0.tet_mat.sum() == 6 * 4 ** 3  # central 4^3 cells of 12^3
    N, frac, V0 = ei.batch_instance_params(0)
    assert 16 <= N <= 48 and 0.2 <= frac <= 0.5 and 5e3 <= V0 <= 2e4
