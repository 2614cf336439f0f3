"""POD-MOR start vectors (oracle), Section IV, second half.

Proper orthogonal decomposition: solutions ("snapshots") of earlier M-solves
are collected in a snapshot matrix X (n x K), which is decomposed by a
singular value decomposition; the left singular vectors of the m largest
singular values form the basis V (n x m) and the start vector of the next
solve with right-hand side b is the projection of Eq. 5 with that basis,

    x0 = V (V^T M V)^-1 V^T b.

Two ways of collecting snapshots (Section IV):

* ``MOR``  - the first K solutions are taken, the basis is computed once and
  kept for the rest of the simulation (one reduced system).
* ``MOR2`` - like SPE, the latest solutions: a solution is added to the
  snapshot set only when its solve needed more than a given number of PCG
  iterations; when the set is full the oldest snapshot is overwritten, and
  the basis and reduced system are recomputed after every addition.

Readings where the paper is silent: the SVD is the Euclidean one of the
snapshot matrix (classical POD); singular values below ``drop`` times the
largest are discarded (rank deficiency of nearly repeated snapshots);
before MOR's set is complete, and while MOR2's set is empty, the start
vector is the previous solution.

Pins (tests/test_oracle_pod.py): the singular values equal the square roots
of the eigenvalues of the Gram matrix X^T X; V is orthonormal; the
snapshot projection error equals the discarded singular values
(Eckart-Young); a solution inside span(V) is reproduced; the error of x0 is
M-orthogonal to span(V); MOR keeps its first basis; MOR2 adds a snapshot
only above the iteration threshold and overwrites the oldest.
"""
from __future__ import annotations

import numpy as np


def pod_basis(X, m, drop=1e-8):
    """Leading left singular vectors of the snapshot matrix X (n x K).

    Returns (V, sigma): V has min(m, numerical rank) columns (singular
    values below drop * sigma_1 are discarded), sigma all singular values."""
    X = np.asarray(X, dtype=np.float64)
    if X.shape[1] == 0:
        return np.zeros((X.shape[0], 0)), np.zeros(0)
    U, sig, _ = np.linalg.svd(X, full_matrices=False)
    if sig[0] == 0.0:
        return np.zeros((X.shape[0], 0)), sig
    keep = int(np.count_nonzero(sig > drop * sig[0]))
    return U[:, :min(m, keep)], sig


def pod_start(M, V, b):
    """x0 = V (V^T M V)^-1 V^T b (Eq. 5 with the POD basis V)."""
    if V.shape[1] == 0:
        return np.zeros_like(b)
    A = V.T @ (M @ V)
    return V @ np.linalg.solve(A, V.T @ b)


class MOR:
    """Fixed POD basis from the first K solutions (one reduced system)."""

    def __init__(self, M, K, m, drop=1e-8):
        self.M, self.K, self.m, self.drop = M, K, m, drop
        self.snaps = []
        self.V = None

    def start(self, b, prev):
        return prev.copy() if self.V is None else pod_start(self.M, self.V, b)

    def after_solve(self, x, iters):
        if self.V is None:
            self.snaps.append(np.array(x, dtype=np.float64, copy=True))
            if len(self.snaps) == self.K:
                self.V, _ = pod_basis(np.stack(self.snaps, axis=1), self.m, self.drop)


class MOR2:
    """Rolling POD basis: a solution whose solve took more than ``min_iters``
    PCG iterations enters the set of at most K snapshots (the oldest is
    overwritten when full); the basis is recomputed after every addition."""

    def __init__(self, M, K, m, min_iters, drop=1e-8):
        self.M, self.K, self.m, self.min_iters, self.drop = M, K, m, min_iters, drop
        self.snaps = []   # oldest first
        self.V = None
        self.rebuilds = 0

    def start(self, b, prev):
        return prev.copy() if self.V is None else pod_start(self.M, self.V, b)

    def after_solve(self, x, iters):
        if iters <= self.min_iters:
            return
        if len(self.snaps) == self.K:
            self.snaps.pop(0)
        self.snaps.append(np.array(x, dtype=np.float64, copy=True))
        self.V, _ = pod_basis(np.stack(self.snaps, axis=1), self.m, self.drop)
        self.rebuilds += 1
