"""Structured Cartesian mesh, Q2 velocity / Q1 pressure numbering, constraints (oracle).

TEST INFRASTRUCTURE: only tests, smoke() and bench.py's CPU-baseline leg use this.

Spaces: Taylor-Hood Q2-Q1 on quadrilaterals / hexahedra (Sec. 3.2, Eq. "spaces",
p1 = 2, p2 = 1; Sec. 5 first paragraph).  The paper uses deal.II numbering, which
is not reproducible here; this library fixes a lexicographic, component-blocked
numbering (x fastest):

  velocity node (I, J[, K]) on the (2 n_x + 1) x (2 n_y + 1) [x (2 n_z + 1)] grid
      -> I + (2 n_x + 1) * (J + (2 n_y + 1) * K)
  DoF of component a at velocity node v -> a * N_v + v
  pressure node (i, j[, k]) on the (n_x + 1) x ... grid -> i + (n_x + 1)(j + (n_y + 1) k),
      DoF -> d * N_v + q
  cell (i, j[, k]) -> i + n_x (j + n_y k); its local velocity node (a, b[, c]) in {0,1,2}^d is
      global node (2i + a, 2j + b, 2k + c), local index a + 3 b + 9 c;
      local pressure node (a, b[, c]) in {0,1}^d, local index a + 2 b + 4 c.

Constraints: a velocity node is constrained (all components) if it lies on a
Dirichlet face or belongs to an obstacle ("void") cell; a pressure node is
constrained if no active cell touches it.  Parity: pinned by the DoF-count
closed forms d (2n+1)^d and (n+1)^d and by direct index checks in the tests.
"""
from __future__ import annotations

import itertools

import numpy as np


class Mesh:
    def __init__(self, dim, n, length, void=None, dirichlet_faces=None):
        self.dim = int(dim)
        self.n = tuple(int(k) for k in n)
        self.length = tuple(float(x) for x in length)
        assert len(self.n) == self.dim and len(self.length) == self.dim
        self.h = tuple(self.length[a] / self.n[a] for a in range(self.dim))
        self.nv_axis = tuple(2 * k + 1 for k in self.n)
        self.np_axis = tuple(k + 1 for k in self.n)
        self.Nv = int(np.prod(self.nv_axis))
        self.Np = int(np.prod(self.np_axis))
        self.Nc = int(np.prod(self.n))
        self.n_u = self.dim * self.Nv
        self.N = self.n_u + self.Np
        self.faces = (1 << (2 * self.dim)) - 1 if dirichlet_faces is None else int(dirichlet_faces)
        if void is None:
            self.void = np.zeros(self.Nc, dtype=bool)
        else:
            self.void = np.asarray(void).astype(bool).reshape(self.Nc)

    # ---- index helpers -------------------------------------------------
    def cell_index_tuples(self):
        """(N_c, d) integer cell coordinates, row c = cell c (x fastest)."""
        idx = np.arange(self.Nc)
        out = np.zeros((self.Nc, self.dim), dtype=np.int64)
        for a in range(self.dim):
            out[:, a] = idx % self.n[a]
            idx = idx // self.n[a]
        return out

    def vnode_flat(self, I):
        """Flat velocity node index from an (..., d) array of grid coordinates."""
        I = np.asarray(I, dtype=np.int64)
        flat = np.zeros(I.shape[:-1], dtype=np.int64)
        stride = 1
        for a in range(self.dim):
            flat = flat + I[..., a] * stride
            stride *= self.nv_axis[a]
        return flat

    def pnode_flat(self, I):
        I = np.asarray(I, dtype=np.int64)
        flat = np.zeros(I.shape[:-1], dtype=np.int64)
        stride = 1
        for a in range(self.dim):
            flat = flat + I[..., a] * stride
            stride *= self.np_axis[a]
        return flat

    def vnode_tuples(self):
        idx = np.arange(self.Nv)
        out = np.zeros((self.Nv, self.dim), dtype=np.int64)
        for a in range(self.dim):
            out[:, a] = idx % self.nv_axis[a]
            idx = idx // self.nv_axis[a]
        return out

    def pnode_tuples(self):
        idx = np.arange(self.Np)
        out = np.zeros((self.Np, self.dim), dtype=np.int64)
        for a in range(self.dim):
            out[:, a] = idx % self.np_axis[a]
            idx = idx // self.np_axis[a]
        return out

    @staticmethod
    def local_offsets(dim, per_axis):
        """Local node offsets, local index = a + per_axis*b + per_axis^2*c (x fastest)."""
        offs = []
        for t in itertools.product(range(per_axis), repeat=dim):
            offs.append(t[::-1])  # itertools varies the last entry fastest
        return np.array(offs, dtype=np.int64)

    def cell_vnodes(self):
        """(N_c, 3^d) global velocity node of each local Q2 node."""
        cells = self.cell_index_tuples()
        offs = self.local_offsets(self.dim, 3)
        return self.vnode_flat(2 * cells[:, None, :] + offs[None, :, :])

    def cell_pnodes(self):
        cells = self.cell_index_tuples()
        offs = self.local_offsets(self.dim, 2)
        return self.pnode_flat(cells[:, None, :] + offs[None, :, :])

    def cell_udofs(self):
        """(N_c, d * 3^d) global velocity DoFs, local order component-major."""
        vn = self.cell_vnodes()
        return np.concatenate([a * self.Nv + vn for a in range(self.dim)], axis=1)

    def active_cells(self):
        return np.nonzero(~self.void)[0]

    # ---- constraints ---------------------------------------------------
    def vnode_constrained(self):
        t = self.vnode_tuples()
        c = np.zeros(self.Nv, dtype=bool)
        for a in range(self.dim):
            if self.faces & (1 << (2 * a)):
                c |= t[:, a] == 0
            if self.faces & (1 << (2 * a + 1)):
                c |= t[:, a] == self.nv_axis[a] - 1
        if self.void.any():
            vn = self.cell_vnodes()[self.void]
            c[np.unique(vn.ravel())] = True
        return c

    def pnode_constrained(self):
        touched = np.zeros(self.Np, dtype=bool)
        pn = self.cell_pnodes()[~self.void]
        touched[np.unique(pn.ravel())] = True
        return ~touched

    def dof_constrained(self):
        """Boolean mask over the full vector [u_x | u_y | (u_z) | p]."""
        vc = self.vnode_constrained()
        return np.concatenate([np.tile(vc, self.dim), self.pnode_constrained()])

    def has_pressure_nullspace(self):
        """Constant pressure is in the kernel of B^T iff every boundary face is Dirichlet."""
        return self.faces == (1 << (2 * self.dim)) - 1

    # ---- levels --------------------------------------------------------
    def coarsen(self):
        """Mesh with half the cells per axis.  A coarse cell is an obstacle cell iff all of its
        2^d children are (so the coarse active region covers the fine one)."""
        assert all(k % 2 == 0 for k in self.n), "mesh not coarsenable"
        nc = tuple(k // 2 for k in self.n)
        coarse = Mesh(self.dim, nc, self.length, None, self.faces)
        ch = children(coarse)
        coarse.void = np.all(self.void[ch], axis=1)
        return coarse


def children(coarse: Mesh):
    """(N_c_coarse, 2^d) fine cell indices of each coarse cell's children."""
    cells = coarse.cell_index_tuples()
    offs = Mesh.local_offsets(coarse.dim, 2)
    fine_n = tuple(2 * k for k in coarse.n)
    I = 2 * cells[:, None, :] + offs[None, :, :]
    flat = np.zeros(I.shape[:-1], dtype=np.int64)
    stride = 1
    for a in range(coarse.dim):
        flat = flat + I[..., a] * stride
        stride *= fine_n[a]
    return flat


def coarsen_eta(fine: Mesh, coarse: Mesh, eta_fine):
    """Coarse eta = arithmetic mean of the active children (1.0 for all-void coarse cells)."""
    ch = children(coarse)
    act = ~fine.void[ch]
    vals = np.where(act, eta_fine[ch], 0.0)
    cnt = act.sum(axis=1)
    return np.where(cnt > 0, vals.sum(axis=1) / np.maximum(cnt, 1), 1.0)


def mesh_from_problem(p):
    return Mesh(p.dim, p.n, p.length, p.void, p.dirichlet_faces)
