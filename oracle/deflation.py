"""Rigid-body deflation of stiff inclusions in the velocity V-cycle (oracle).

TEST INFRASTRUCTURE: only tests, smoke() and bench.py's CPU-baseline leg use this.

The paper's FSI meshes resolve the solid-fluid interface on the coarsest level (Sec. 4), so every
level's rediscretised operator carries the solid's near-rigid motions.  Stiff inclusions smaller
than a coarse cell break that: the motions of each inclusion as a rigid body have almost no
strain energy (only the fluid layer around it deforms), their Jacobi-scaled eigenvalues lie far
below the Chebyshev smoother's interval, and no coarse level represents them, so the V-cycle
leaves them untouched and FGMRES stalls.  This option (not part of the paper's method) adds those
motions as an explicit coarse space on the finest level:

* stiff cells: active cells with eta >= sqrt(eta_min eta_max) over the active cells, considered
  only when eta_max / eta_min >= 1e3; an inclusion is a connected component of stiff cells, two
  cells being connected when they share a velocity node;
* Z: for each inclusion its rigid motions, evaluated at the velocity nodes of its cells: the d
  translations e_a and the rotations about the mean c of those nodes' coordinates, 2D
  (-(y - c_y), x - c_x), 3D omega x (x - c) for omega = e_x, e_y, e_z; constrained entries
  zeroed, columns that vanish entirely dropped;
* E = Z^T A Z (A: constrained velocity block of the finest level);
* in the V-cycle of the finest level, with r = b - A x after pre-smoothing, the coarse-grid
  correction becomes x += P V(P^T r) + Z E^{-1} Z^T r (additive), followed by post-smoothing.

A rigid motion is linear, hence exactly a Q2 field with zero symmetric gradient: inside an
inclusion its viscous energy vanishes and E does not depend on the inclusion's eta (pinned).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import Mesh

CONTRAST_MIN = 1e3


def stiff_cells(mesh: Mesh, eta) -> np.ndarray:
    """Boolean mask of stiff active cells (empty if the contrast is below CONTRAST_MIN)."""
    eta = np.asarray(eta, dtype=float)
    act = ~mesh.void
    if not act.any():
        return np.zeros(mesh.Nc, dtype=bool)
    lo, hi = eta[act].min(), eta[act].max()
    if hi < CONTRAST_MIN * lo:
        return np.zeros(mesh.Nc, dtype=bool)
    return act & (eta >= np.sqrt(lo * hi))


def inclusion_labels(mesh: Mesh, stiff: np.ndarray) -> np.ndarray:
    """Label (1, 2, ...) of each stiff cell's inclusion, 0 elsewhere.  Cells are connected when
    they share a velocity node (cell coordinates differ by at most 1 along every axis).  Labels
    are numbered in the order of each inclusion's first cell (cell index order)."""
    n = mesh.n
    labels = np.zeros(mesh.Nc, dtype=np.int64)
    cells = mesh.cell_index_tuples()
    strides = [int(np.prod(n[:a])) for a in range(mesh.dim)]
    offsets = [o for o in np.ndindex(*(3,) * mesh.dim) if any(v != 1 for v in o)]
    nxt = 0
    for c0 in range(mesh.Nc):
        if not stiff[c0] or labels[c0]:
            continue
        nxt += 1
        labels[c0] = nxt
        stack = [c0]
        while stack:
            c = stack.pop()
            ci = cells[c]
            for o in offsets:
                nb = ci + np.array(o) - 1
                if np.any(nb < 0) or np.any(nb >= np.array(n)):
                    continue
                cn = int(sum(int(nb[a]) * strides[a] for a in range(mesh.dim)))
                if stiff[cn] and not labels[cn]:
                    labels[cn] = nxt
                    stack.append(cn)
    return labels


def rigid_basis(mesh: Mesh, labels: np.ndarray) -> sp.csc_matrix:
    """Z (n_u x m): per inclusion (label order) the d translations, then the rotations (2D: one,
    3D: about x, y, z), on the velocity nodes of the inclusion's cells; constrained rows zero;
    all-zero columns removed."""
    dim, Nv = mesh.dim, mesh.Nv
    con = mesh.vnode_constrained()
    X = mesh.vnode_tuples().astype(float) * (np.array(mesh.h) / 2.0)[None, :]
    cv = mesh.cell_vnodes()
    cols = []
    for k in range(1, int(labels.max(initial=0)) + 1):
        nodes = np.unique(cv[labels == k].ravel())
        c = X[nodes].mean(axis=0)
        d = X[nodes] - c[None, :]
        free = ~con[nodes]
        modes = []
        for a in range(dim):
            v = np.zeros((len(nodes), dim))
            v[:, a] = 1.0
            modes.append(v)
        if dim == 2:
            v = np.zeros((len(nodes), 2))
            v[:, 0], v[:, 1] = -d[:, 1], d[:, 0]
            modes.append(v)
        else:
            for ax in range(3):  # omega = e_ax: omega x d
                om = np.zeros(3)
                om[ax] = 1.0
                modes.append(np.cross(om[None, :], d))
        for v in modes:
            col = np.zeros(dim * Nv)
            for a in range(dim):
                col[a * Nv + nodes[free]] = v[free, a]
            if np.any(col != 0.0):
                cols.append(col)
    if not cols:
        return sp.csc_matrix((dim * Nv, 0))
    return sp.csc_matrix(np.array(cols).T)


class Deflation:
    """Z, E = Z^T A Z and the correction Z E^{-1} Z^T r for one level's operator A."""

    def __init__(self, mesh: Mesh, eta, A):
        self.labels = inclusion_labels(mesh, stiff_cells(mesh, eta))
        self.Z = rigid_basis(mesh, self.labels)
        self.m = self.Z.shape[1]
        self.E = (self.Z.T @ (A @ self.Z)).toarray() if self.m else np.zeros((0, 0))
        self.Einv = np.linalg.inv(self.E) if self.m else self.E

    def correction(self, r):
        if self.m == 0:
            return np.zeros_like(r)
        return self.Z @ (self.Einv @ (self.Z.T @ r))
