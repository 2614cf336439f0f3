"""The semi-discrete EQS system with Dirichlet elimination (oracle).

Eq. 2 reads M dx/dt + K(x) x = b, b holding the inhomogeneous Dirichlet
data.  Nodes split into free (f) and Dirichlet (d) sets; on d the potential
is prescribed, x_d = g(t): 0 on tag-1 nodes, V0 sin(2 pi freq t + phase) on
tag-2 nodes.  With x~ = [x_f; g(t)] the free rows of Eq. 2 give

    M_ff dx_f/dt = -[K(x~) x~]_f - M_fd g'(t) =: R(t, x_f)
    F(t, x_f)    = M_ff^-1 R(t, x_f)

(the reading of "b" used throughout: Dirichlet elimination, evaluated at
the stage time, which the second-order RKC scheme needs).  Side faces carry
natural (homogeneous Neumann) conditions.

Pins: tests/test_oracle_system.py (homogeneous slab against the
closed-form exponential relaxation with time constant eps/kappa; the static
lift is exactly linear in z; a driven slab converges at second order; a
nonlinear run in which the varistor switches converges at second order to
an independent stiff integrator, SciPy's Radau IIA).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem


class EQSSystem:
    def __init__(self, problem):
        p = problem
        self.p = p
        self.free = np.nonzero(p.node_tag == 0)[0]
        self.dir = np.nonzero(p.node_tag != 0)[0]
        self.top = (p.node_tag[self.dir] == 2).astype(np.float64)  # indicator on d
        self.M = fem.assemble_M(p.xyz, p.tets, p.tet_mat, p.materials)
        self.Mff = self.M[self.free][:, self.free].tocsr()
        self.Mff.sort_indices()
        self.Mfd = self.M[self.free][:, self.dir].tocsr()
        self.m_top = self.Mfd @ self.top  # M_fd 1_top
        self._lu = None
        self._geom = None

    def geometry(self):
        """(G, V) of every P1 tet, computed once (None for P2 meshes)."""
        if self._geom is None and self.p.tets.shape[1] == 4:
            self._geom = fem.tet_geometry(self.p.xyz, self.p.tets)
        return self._geom

    # Dirichlet data g(t) and g'(t) on the d nodes
    def g(self, t):
        p = self.p
        return self.top * (p.V0 * np.sin(2 * np.pi * p.freq * t + p.phase))

    def gdot(self, t):
        p = self.p
        return self.top * (p.V0 * 2 * np.pi * p.freq * np.cos(2 * np.pi * p.freq * t + p.phase))

    def full(self, t, xf):
        """x~ = [x_f; g(t)] as a full node vector (mesh order)."""
        x = np.zeros(self.p.n_nodes)
        x[self.free] = xf
        x[self.dir] = self.g(t)
        return x

    def rhs(self, t, xf):
        """R(t, x_f) = -[K(x~)x~]_f - M_fd g'(t)."""
        p = self.p
        x = self.full(t, xf)
        y = fem.apply_K(p.xyz, p.tets, p.tet_mat, p.materials, x, geometry=self.geometry())
        return -y[self.free] - self.Mfd @ self.gdot(t)

    def solve_direct(self, R):
        """M_ff^-1 R by a sparse LU factorisation computed once (the plain
        definition of the M-solve's result)."""
        if self._lu is None:
            self._lu = spla.splu(self.Mff.tocsc())
        return self._lu.solve(R)

    def F(self, t, xf, solve=None):
        return (solve or self.solve_direct)(self.rhs(t, xf))
