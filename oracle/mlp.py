"""Learned per-node start vector for the M-solves (oracle).

Section IV estimates start vectors for the multiple right-hand-side M-solves
from earlier solutions.  The learned estimator (a project addition, no
counterpart in the paper) is a per-node network:

  inputs  x = [h1, h2, h3, h4, m1, m2, m3, m4] / s_h   at free node i
          h_k = k-th most recent M-solve solution, m_k = mean of h_k over the
          free graph neighbours of i (mesh edges, self excluded; 0 without
          neighbours), s_h = RMS of h1 over the free nodes
  network a1 = W1 x + b1, g1 = GELU(a1), a2 = W2 g1 + b2, g2 = GELU(a2),
          o = w3 . g2 + b3          (8 -> 32 -> 32 -> 1, exact-erf GELU)
  guess   z0 = h1 + s_h o
  loss    mean over the batch of (o - (z - h1)/s_h)^2
  update  Adam (Kingma & Ba 2015) on FP32 master weights; forward and backward
          use the weights rounded to BF16 (round to nearest even).

A second mode corrects the SPE start vector from solution increments
(spe_features / spe_guess below).

Everything here is FP64 numpy.  Pins (tests/test_oracle_mlp.py): central
finite differences of the loss against the analytic gradient; GELU against
its erf definition and derivative; the zero output layer returns h1 exactly;
Adam's first step equals -lr * sign(g) and its hand-computed second and
third steps; 1-ring means against a dense adjacency count; the SPE-correction
inputs are increments (a common offset of all vectors changes nothing), the
zero output layer returns x0, the line search never increases the M-norm
error and lands on the solution when the direction is the error itself.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT2PI = 1.0 / math.sqrt(2.0 * math.pi)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    W1 = theta[0:256].reshape(32, 8)
    b1 = theta[256:288]
    W2 = theta[288:1312].reshape(32, 32)
    b2 = theta[1312:1344]
    w3 = theta[1344:1376]
    b3 = theta[1376]
    return W1, b1, W2, b2, w3, b3


def to_bf16(a):
    """Round float32 values to BF16 (nearest, ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / SQRT2)) + x * INV_SQRT2PI * np.exp(-0.5 * x * x)


def forward(theta, X):
    """X: (B, 8) -> o (B,), cache."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    a1 = X @ W1.T + b1
    g1 = gelu(a1)
    a2 = g1 @ W2.T + b2
    g2 = gelu(a2)
    o = g2 @ w3 + b3
    return o, (X, a1, g1, a2, g2)


def backward(theta, cache, do):
    """Gradient of sum(do * o) with respect to the packed parameters."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    X, a1, g1, a2, g2 = cache
    gw3 = g2.T @ do
    gb3 = do.sum()
    dg2 = np.outer(do, w3)
    da2 = dg2 * gelu_grad(a2)
    gW2 = da2.T @ g1
    gb2 = da2.sum(axis=0)
    dg1 = da2 @ W2
    da1 = dg1 * gelu_grad(a1)
    gW1 = da1.T @ X
    gb1 = da1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


def loss_and_grad(theta, X, T):
    """MSE loss and its gradient, with the BF16-rounded weights."""
    tb = to_bf16(theta)
    o, cache = forward(tb, X)
    e = o - T
    loss = float(np.mean(e * e))
    return loss, backward(tb, cache, 2.0 * e / len(T))


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step t >= 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def free_adjacency(tets, free_nodes, n_nodes):
    """CSR (indptr, indices) of the mesh-edge graph among free nodes, in the
    free numbering (ascending mesh order), self excluded."""
    import scipy.sparse as sp

    e = tets[:, [[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3]]].reshape(-1, 2)
    fidx = -np.ones(n_nodes, dtype=np.int64)
    fidx[free_nodes] = np.arange(len(free_nodes))
    a, b = fidx[e[:, 0]], fidx[e[:, 1]]
    keep = (a >= 0) & (b >= 0)
    a, b = a[keep], b[keep]
    nf = len(free_nodes)
    A = sp.coo_matrix((np.ones(2 * len(a)), (np.r_[a, b], np.r_[b, a])), shape=(nf, nf)).tocsr()
    A.data[:] = 1.0
    A.sort_indices()
    return A


def ring_means(A, H):
    """m_k = mean of h_k over the neighbours (rows of the adjacency A)."""
    deg = np.asarray(A.sum(axis=1)).ravel()
    with np.errstate(invalid="ignore", divide="ignore"):
        inv = np.where(deg > 0, 1.0 / np.where(deg > 0, deg, 1.0), 0.0)
    return [inv * (A @ h) for h in H]


def features(A, H):
    """(n, 8) normalised inputs and s_h for the history H = [h1, h2, h3, h4]."""
    s_h = float(np.sqrt(np.mean(H[0] * H[0])))
    M = ring_means(A, H)
    X = np.stack(list(H) + M, axis=1)
    return (X / s_h if s_h > 0 else X), s_h


def guess(theta, A, H):
    """z0 = h1 + s_h * MLP(x) (h1 when s_h = 0)."""
    X, s_h = features(A, H)
    if s_h == 0.0:
        return np.array(H[0], dtype=np.float64, copy=True)
    o, _ = forward(to_bf16(theta), X)
    return H[0] + s_h * o


# ------------------------------------------------ correction of the SPE start
# The second mode of the learned estimator proposes a correction direction
# for the SPE start vector x0 (Eq. 4-5) and takes the step along it that
# minimises the M-norm error (an exact line search; M is SPD):
#
#   inputs  x = [d0, d1, d2, d3, m(d0), m(d1), m(d2), m(d3)] / s   at free node i
#           d0 = x0 - h1 (the SPE step from the previous solution),
#           d_k = h_k - h_{k+1} (k = 1..3; h1 the most recent solution),
#           m(d) = mean of d over the free graph neighbours of i (self
#           excluded), s = RMS of d0 over the free nodes
#   direction  d = s o  (0 when s = 0)
#   start      z0 = x0 + alpha d,  alpha = d.(R - M x0) / d.(M d)  (0 when d.Md = 0)
#   target     (z - x0) / RMS(z - x0)   (the scale of d is immaterial to z0)
#
# with the same 8-32-32-1 network, loss and optimizer as above.  The inputs
# are increments: the information is in how the solutions change, which is
# small against the solutions themselves; fed raw, those inputs would ask
# BF16 weights to cancel them to better than their 8-bit precision.  The
# line search keeps a poor direction harmless: ||z0 - z||_M <= ||x0 - z||_M.
def spe_increments(x0, H):
    """[d0, d1, d2, d3] of the SPE-correction mode (H = [h1, h2, h3, h4])."""
    return [x0 - H[0], H[0] - H[1], H[1] - H[2], H[2] - H[3]]


def spe_features(A, x0, H):
    """(n, 8) normalised inputs and s of the SPE-correction mode."""
    D = spe_increments(x0, H)
    s = float(np.sqrt(np.mean(D[0] * D[0])))
    M = ring_means(A, D)
    X = np.stack(D + M, axis=1)
    return (X / s if s > 0 else X), s


def spe_direction(theta, A, x0, H):
    """d = s * MLP(x) (0 when s = 0)."""
    X, s = spe_features(A, x0, H)
    if s == 0.0:
        return np.zeros_like(x0)
    o, _ = forward(to_bf16(theta), X)
    return s * o


def spe_corrected_start(Mff, theta, A, x0, H, R):
    """z0 = x0 + alpha d with the M-norm optimal alpha along the direction d."""
    d = spe_direction(theta, A, x0, H)
    Md = Mff @ d
    den = float(d @ Md)
    alpha = float(d @ (R - Mff @ x0)) / den if den > 0 else 0.0
    return x0 + alpha * d, alpha


def spe_target(z, x0):
    """Normalised training target (z - x0) / RMS(z - x0) of one solve (0 when z = x0)."""
    e = z - x0
    r = float(np.sqrt(np.mean(e * e)))
    return e / r if r > 0 else np.zeros_like(e)
