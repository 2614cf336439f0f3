"""Kuhn-split cube meshes, seeded jitter, material and Dirichlet tagging.

Node (i, j, k), 0 <= i, j, k <= N, has index ``i + (N+1)*(j + (N+1)*k)`` and
sits at ``(i, j, k) * h`` with ``h = L/N``.  Each of the N^3 cells is split
into 6 tetrahedra along its main diagonal (the Kuhn/Freudenthal split): for
every permutation (a, b, c) of the axes, in lexicographic order, the tet is
``v0, v0+e_a, v0+e_a+e_b, v0+e_a+e_b+e_c``.  All cells use the same
orientation, so the split is conforming.  For odd permutations the last two
vertices are swapped so that every tet has a positive Jacobian determinant.
Tets are numbered cell-major (cell ``ci + N*(cj + N*ck)``), 6 per cell.

Random numbers come from the counter-based splitmix64 finaliser (Steele,
Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
value ``k`` of stream ``seed`` is ``mix(seed + (k+1)*0x9E3779B97F4A7C15)``,
so every draw is independent of evaluation order.
"""

from __future__ import annotations

import dataclasses
import itertools

import numpy as np

L_CUBE = 0.1  # cube edge [m]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, k) -> np.ndarray:
    """Counter-based splitmix64: the k-th 64-bit output of stream ``seed``."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (k + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, k) -> np.ndarray:
    """Uniform double in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclasses.dataclass(frozen=True)
class Material:
    """Material law: eps = eps0*eps_r and
    kappa(E) = kappa_lo + (kappa_hi - kappa_lo) * logistic((E - E0)/w);
    kappa_hi == kappa_lo marks a constant conductivity."""

    eps_r: float
    kappa_lo: float
    kappa_hi: float
    E0: float = 1.0
    w: float = 1.0

    def as_tuple(self):
        return (self.eps_r, self.kappa_lo, self.kappa_hi, self.E0, self.w)


BACKGROUND = Material(3.0, 1e-14, 1e-14, 1.0, 1.0)
VARISTOR = Material(12.0, 1e-12, 1e-6, 5e5, 5e4)


def kuhn_cube(N: int, L: float = L_CUBE, jitter: float = 0.0, seed: int = 0):
    """Return (xyz[n,3] float64, tets[n_tet,4] int32) for the N^3-cell cube.

    ``jitter`` > 0 moves every strictly interior node by ``u*jitter*h`` per
    coordinate, u ~ U[-1, 1) drawn as value ``3*node + coord`` of stream
    ``seed``.
    """
    n1 = N + 1
    h = L / N
    i, j, k = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    # node index i + n1*(j + n1*k): order with i fastest
    ii = i.transpose(2, 1, 0).reshape(-1)
    jj = j.transpose(2, 1, 0).reshape(-1)
    kk = k.transpose(2, 1, 0).reshape(-1)
    xyz = np.stack([ii * h, jj * h, kk * h], axis=1).astype(np.float64)
    if jitter > 0.0:
        interior = (ii > 0) & (ii < N) & (jj > 0) & (jj < N) & (kk > 0) & (kk < N)
        nodes = np.nonzero(interior)[0].astype(np.uint64)
        for c in range(3):
            u = 2.0 * uniform01(seed, np.uint64(3) * nodes + np.uint64(c)) - 1.0
            xyz[nodes, c] += u * jitter * h

    ci, cj, ck = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    ci = ci.transpose(2, 1, 0).reshape(-1)
    cj = cj.transpose(2, 1, 0).reshape(-1)
    ck = ck.transpose(2, 1, 0).reshape(-1)
    v0 = ci + n1 * (cj + n1 * ck)
    step = (1, n1, n1 * n1)
    tets = np.empty((N ** 3, 6, 4), dtype=np.int64)
    for p, perm in enumerate(itertools.permutations(range(3))):
        a, b, c = perm
        verts = [v0, v0 + step[a], v0 + step[a] + step[b], v0 + step[a] + step[b] + step[c]]
        inversions = sum(1 for x in range(3) for y in range(x + 1, 3) if perm[x] > perm[y])
        if inversions % 2 == 1:
            verts[2], verts[3] = verts[3], verts[2]
        for q in range(4):
            tets[:, p, q] = verts[q]
    return xyz, tets.reshape(-1, 4).astype(np.int32)


# P2 (10-node) tets: vertex order as kuhn_cube, then the midpoints of the
# edges (0,1), (0,2), (0,3), (1,2), (1,3), (2,3).
P2_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def kuhn_cube_p2(N: int, L: float = L_CUBE, jitter: float = 0.0, seed: int = 0):
    """Return (xyz[(2N+1)^3, 3], tets[6 N^3, 10]) of the quadratic mesh.

    Every node of the (2N+1)^3 refined grid is a vertex (even refined
    coordinates) or the midpoint of exactly one edge of the Kuhn split.
    Vertices sit where ``kuhn_cube`` puts them (same jitter draws), edges are
    straight: a midpoint node is the mean of its edge's two vertices.  Node
    index I + R (J + R K), R = 2N + 1, refined coordinates (I, J, K).
    """
    xyz1, tets1 = kuhn_cube(N, L, jitter, seed)
    n1, R = N + 1, 2 * N + 1
    v = tets1.astype(np.int64)
    vi, vj, vk = v % n1, (v // n1) % n1, v // (n1 * n1)
    ref = np.stack([2 * vi, 2 * vj, 2 * vk], axis=2)  # (T, 4, 3) refined coordinates
    ids = np.empty((len(tets1), 10), dtype=np.int64)
    ids[:, :4] = ref[:, :, 0] + R * (ref[:, :, 1] + R * ref[:, :, 2])
    xyz = np.full((R ** 3, 3), np.nan)
    xyz[ids[:, :4].reshape(-1)] = xyz1[v.reshape(-1)]
    for e, (a, b) in enumerate(P2_EDGES):
        m = (ref[:, a] + ref[:, b]) // 2
        ids[:, 4 + e] = m[:, 0] + R * (m[:, 1] + R * m[:, 2])
        xyz[ids[:, 4 + e]] = 0.5 * (xyz1[v[:, a]] + xyz1[v[:, b]])
    if np.isnan(xyz).any():
        raise AssertionError("refined grid node without an edge")
    return xyz, ids.astype(np.int32)


def dirichlet_tags_p2(N: int) -> np.ndarray:
    """Refined-grid tags: 1 on z = 0, 2 on z = L, 0 elsewhere."""
    R = 2 * N + 1
    tag = np.zeros(R ** 3, dtype=np.uint8)
    tag[: R * R] = 1
    tag[-R * R:] = 2
    return tag


def _centroids(xyz, tets):
    return xyz[tets].mean(axis=1)


def tag_materials_block(xyz, tets, lo: float, hi: float) -> np.ndarray:
    """Material 1 (varistor) where the tet centroid lies in the closed cube
    [lo, hi]^3, material 0 (background) elsewhere."""
    c = _centroids(xyz, tets)
    inside = np.all((c >= lo) & (c <= hi), axis=1)
    return inside.astype(np.uint8)


def tag_materials_spheres(xyz, tets, centres, radius: float) -> np.ndarray:
    """Material 1 where the tet centroid lies in any closed ball."""
    c = _centroids(xyz, tets)
    inside = np.zeros(len(tets), dtype=bool)
    for cen in np.asarray(centres, dtype=np.float64):
        inside |= np.sum((c - cen) ** 2, axis=1) <= radius * radius
    return inside.astype(np.uint8)


def dirichlet_tags(N: int) -> np.ndarray:
    """0 = free, 1 = grounded (z = 0), 2 = driven (z = L); side faces free."""
    n1 = N + 1
    tag = np.zeros(n1 ** 3, dtype=np.uint8)
    tag[: n1 * n1] = 1
    tag[-n1 * n1:] = 2
    return tag


@dataclasses.dataclass
class Problem:
    """One EQS instance: mesh, materials, Dirichlet tags and the drive
    g(t) = V0*sin(2*pi*freq*t + phase) on tag-2 nodes (0 on tag-1 nodes)."""

    N: int
    xyz: np.ndarray
    tets: np.ndarray
    tet_mat: np.ndarray
    node_tag: np.ndarray
    materials: tuple
    V0: float = 1e4
    freq: float = 50.0
    phase: float = 0.0
    s: int = 10
    steps: int = 1
    name: str = ""

    @property
    def n_nodes(self):
        return len(self.xyz)

    @property
    def n_tets(self):
        return len(self.tets)

    @property
    def n_free(self):
        return int(np.count_nonzero(self.node_tag == 0))


CONFIG_SEED = 1612094470


def make_problem(N, *, jitter=0.0, seed=CONFIG_SEED, varistor="block", block=(1 / 3, 2 / 3),
                 spheres=None, radius=0.02, V0=1e4, freq=50.0, phase=0.0, s=10, steps=1,
                 name=""):
    xyz, tets = kuhn_cube(N, L_CUBE, jitter, seed)
    if varistor == "block":
        mat = tag_materials_block(xyz, tets, block[0] * L_CUBE, block[1] * L_CUBE)
    elif varistor == "spheres":
        mat = tag_materials_spheres(xyz, tets, spheres, radius)
    elif varistor == "none":
        mat = np.zeros(len(tets), dtype=np.uint8)
    else:
        raise ValueError(varistor)
    return Problem(N, xyz, tets, mat, dirichlet_tags(N), (BACKGROUND, VARISTOR),
                   V0, freq, phase, s, steps, name)


def make_problem_p2(N, *, jitter=0.0, seed=CONFIG_SEED, block=(1 / 3, 2 / 3), V0=1e4, freq=50.0,
                    phase=0.0, s=10, steps=1, name=""):
    """Quadratic (P2) problem on the N^3-cell Kuhn cube with the block
    varistor (material by the centroid of the tet's four vertices)."""
    xyz, tets = kuhn_cube_p2(N, L_CUBE, jitter, seed)
    mat = tag_materials_block(xyz, tets[:, :4], block[0] * L_CUBE, block[1] * L_CUBE)
    return Problem(N, xyz, tets, mat, dirichlet_tags_p2(N), (BACKGROUND, VARISTOR),
                   V0, freq, phase, s, steps, name or f"p2_cube{N}")


def sphere_centres(seed: int, count: int = 2, radius: float = 0.02):
    """Centres ~ U[r, L-r]^3, value 3*sphere + axis of stream ``seed``."""
    u = uniform01(seed, np.arange(3 * count, dtype=np.uint64)).reshape(count, 3)
    return radius + (L_CUBE - 2 * radius) * u


def batch_instance_params(i: int, seed: int = CONFIG_SEED):
    """Seeded parameters of batched instance i: (N in 16..48, block fraction
    in [0.2, 0.5], V0 in [5e3, 2e4]); values 0, 1, 2 of stream seed + i."""
    u = uniform01(seed + i, np.arange(3, dtype=np.uint64))
    N = 16 + int(np.floor(u[0] * 33))
    frac = 0.2 + 0.3 * u[1]
    V0 = 5e3 + 1.5e4 * u[2]
    return N, float(frac), float(V0)


def config_problem(idx: int, N: int | None = None, instance: int = 0):
    """The five synthetic workloads.  ``N`` overrides the mesh size (for
    reduced-size tests of the same recipe)."""
    if idx == 0:
        return make_problem(N or 12, s=10, steps=200, name="cube12_block")
    if idx == 1:
        return make_problem(N or 64, s=20, steps=100, name="cube64_block")
    if idx in (2, 3):
        cen = sphere_centres(CONFIG_SEED + 1)
        return make_problem(N or 128, jitter=0.2, seed=CONFIG_SEED, varistor="spheres",
                            spheres=cen, radius=0.02, s=20, steps=50 if idx == 2 else 200,
                            name="cube128_jitter_spheres")
    if idx == 4:
        Ni, frac, V0 = batch_instance_params(instance)
        lo = 0.5 - frac / 2
        return make_problem(N or Ni, block=(lo, lo + frac), V0=V0, s=10, steps=100,
                            name=f"batch{instance}_cube{N or Ni}")
    raise ValueError(idx)


# ------------------------------------------------------------------ guess MLP
MLP_SIZES = (8, 32, 32, 1)
MLP_NPARAM = 8 * 32 + 32 + 32 * 32 + 32 + 32 + 1  # 1377


def mlp_init(seed: int = CONFIG_SEED + 3) -> np.ndarray:
    """Initial FP32 parameters of the 8-32-32-1 guess network, packed as
    [W1 (32x8, row-major), b1 (32), W2 (32x32), b2 (32), w3 (32), b3 (1)].
    W1 ~ U(-1/sqrt(8), 1/sqrt(8)), W2 ~ U(-1/sqrt(32), 1/sqrt(32)) drawn as
    values 0.. of stream ``seed``; biases and the output layer are zero so the
    untrained network returns the previous-solution guess."""
    u = uniform01(seed, np.arange(256 + 1024, dtype=np.uint64))
    W1 = (2 * u[:256] - 1) / np.sqrt(8.0)
    W2 = (2 * u[256:] - 1) / np.sqrt(32.0)
    out = np.zeros(MLP_NPARAM, dtype=np.float32)
    out[:256] = W1
    out[288:288 + 1024] = W2
    return out
