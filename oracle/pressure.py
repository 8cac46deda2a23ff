"""Pressure Laplacian and its multigrid (Cahouet-Chabard term of the Schur approximation) (oracle).

TEST INFRASTRUCTURE: only tests, smoke() and bench.py's CPU-baseline leg use this.

For the generalized Stokes operator alpha M - div(2 eta eps) the Schur complement behaves like
eta^{-1} M_p on fine scales but like (div alpha^{-1} grad) on scales where alpha dominates
(alpha L^2 / eta >> 1; the channel workload has alpha = 1e3, eta_f = 1).  The 1/eta-weighted
pressure mass alone (Sec. 4's block variant) then leaves FGMRES with hundreds of iterations.
The Cahouet-Chabard approximation adds the reaction part:

    S^{-1} ~ M_p(1/eta)^{-1} + alpha K_p^{-1},

(with alpha per cell: K_p(1/alpha)^{-1}, the Laplacian weighted by 1/alpha_K on each cell, applied
as abar (K_p^w)^{-1} with weights w_K = abar / alpha_K and abar = max alpha; w = 1 for one alpha)

K_p = Q1 stiffness matrix int grad psi_q . grad psi_r over active cells, with p = 0 on faces
without a velocity Dirichlet condition (do-nothing outflow) and on pressure nodes touched by no
active cell.  K_p^{-1} is applied by one V-cycle of the same kind as the velocity one (nested
levels, Q1 interpolation, Chebyshev-Jacobi degree k on [lambda_hi/15, lambda_hi] from 12
Lanczos steps, dense coarse solve).  With every velocity face Dirichlet, K_p is singular (the
constant); the coarse matrix then gets the rank-one term 1 1^T / n_free, which leaves its
action on mean-free vectors unchanged.

Parity pins (tests): Q1 1D stiffness closed form, constant null space / positive
definiteness, Q1 prolongation reproduces bilinear fields, V-cycle symmetry and contraction.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .fem import Q1_NODES, lagrange_1d, tensor_basis
from .mesh import Mesh, coarsen_eta
from .mg import chebyshev, lanczos_max, lanczos_start

LANCZOS_PRESSURE_LEVEL = 0x80  # level field of the start-vector counter: pressure level l -> 0x80 | l


def q1_stiffness_cell(dim, h):
    _, g, w = tensor_basis(dim, h, Q1_NODES, 3)
    return np.einsum("q,qid,qjd->ij", w, g, g)


def laplacian_constraints(mesh: Mesh):
    """Pressure nodes fixed to zero in K_p: no active cell, or on a face without velocity BC."""
    c = mesh.pnode_constrained().copy()
    t = mesh.pnode_tuples()
    for a in range(mesh.dim):
        if not (mesh.faces & (1 << (2 * a))):
            c |= t[:, a] == 0
        if not (mesh.faces & (1 << (2 * a + 1))):
            c |= t[:, a] == mesh.np_axis[a] - 1
    return c


def pressure_laplacian(mesh: Mesh, w=None):
    """(K_p with constraints eliminated, constraint mask); w: optional weight per cell."""
    Ke = q1_stiffness_cell(mesh.dim, mesh.h)
    act = mesh.active_cells()
    pd = mesh.cell_pnodes()[act]
    n = pd.shape[1]
    wa = np.ones(len(act)) if w is None else np.asarray(w, dtype=float)[act]
    vals = (wa[:, None, None] * Ke[None]).reshape(len(act), -1)
    K = sp.coo_matrix((vals.ravel(), (np.repeat(pd, n, axis=1).ravel(), np.tile(pd, (1, n)).ravel())),
                      shape=(mesh.Np, mesh.Np)).tocsr()
    c = laplacian_constraints(mesh)
    keep = sp.diags((~c).astype(float))
    K = (keep @ K @ keep + sp.diags(c.astype(float))).tocsr()
    K.eliminate_zeros()
    return K, c


def q1_prolongation_1d(n_coarse: int) -> sp.csr_matrix:
    """(2 n_c + 1) x (n_c + 1): fine node I in coarse cell c at local t in {0, 1/2, 1}."""
    nf = 2 * n_coarse + 1
    rows, cols, vals = [], [], []
    for I in range(nf):
        c = min(I // 2, n_coarse - 1)
        t = (I - 2 * c) / 2.0
        v, _ = lagrange_1d(Q1_NODES, [t])
        for a in range(2):
            if v[a, 0] != 0.0:
                rows.append(I)
                cols.append(c + a)
                vals.append(v[a, 0])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, n_coarse + 1))


def q1_prolongation(coarse: Mesh, fine: Mesh, c_coarse, c_fine) -> sp.csr_matrix:
    P = q1_prolongation_1d(coarse.n[0])
    for a in range(1, coarse.dim):
        P = sp.kron(q1_prolongation_1d(coarse.n[a]), P)
    P = P.tocsr()
    P = (sp.diags((~c_fine).astype(float)) @ P @ sp.diags((~c_coarse).astype(float))).tocsr()
    P.eliminate_zeros()
    return P


class PressureHierarchy:
    """Multigrid for K_p on the nested meshes (levels[0] = coarsest)."""

    def __init__(self, fine: Mesh, nlevels, degree=4, seed=0, lanczos_steps=12, safety=1.2, ratio=15.0,
                 coarse="cholesky", alpha=None):
        meshes = [fine]
        for _ in range(nlevels - 1):
            meshes.append(meshes[-1].coarsen())
        # alpha per cell: weights w = abar / alpha_K, coarse alpha = mean of the active children
        weights = [None] * nlevels
        self.abar = None
        if alpha is not None and np.ndim(alpha) > 0:
            a = [np.asarray(alpha, dtype=float)]
            for i in range(nlevels - 1):
                a.append(coarsen_eta(meshes[i], meshes[i + 1], a[-1]))
            self.abar = float(a[0].max())
            weights = [self.abar / ai for ai in a]
        meshes, weights = meshes[::-1], weights[::-1]
        self.degree, self.ratio = degree, ratio
        self.levels = []
        for i, m in enumerate(meshes):
            K, c = pressure_laplacian(m, weights[i])
            self.levels.append(dict(mesh=m, K=K, c=c, D=K.diagonal(), P=None, lam_hi=None))
        for i in range(1, len(meshes)):
            lo, hi = self.levels[i - 1], self.levels[i]
            hi["P"] = q1_prolongation(lo["mesh"], hi["mesh"], lo["c"], hi["c"])
        self.coarse = coarse
        for i, lv in enumerate(self.levels):
            if i == 0 and coarse != "chebyshev":
                continue
            v0 = lanczos_start(lv["mesh"].Np, seed, LANCZOS_PRESSURE_LEVEL | i)
            v0[lv["c"]] = 0.0
            lv["lam_hi"] = safety * lanczos_max(lv["K"], lv["D"], v0, lanczos_steps)
        # pure Neumann (every velocity face Dirichlet): the constant is in the kernel of K_p
        self.singular = fine.has_pressure_nullspace()
        if coarse == "cholesky":
            K0 = self.levels[0]["K"].toarray()
            c0 = self.levels[0]["c"]
            if self.singular:
                free = (~c0).astype(float)
                K0 = K0 + np.outer(free, free) / free.sum()
            self.chol = sla.cho_factor(K0, lower=True)

    def vcycle(self, b, level=None):
        if level is None:
            level = len(self.levels) - 1
        lv = self.levels[level]
        if level == 0:
            if self.coarse == "chebyshev":
                return chebyshev(lv["K"], 1.0 / lv["D"], b, None, self.degree, lv["lam_hi"] / self.ratio, lv["lam_hi"])
            return sla.cho_solve(self.chol, b)
        lo, hi = lv["lam_hi"] / self.ratio, lv["lam_hi"]
        Dinv = 1.0 / lv["D"]
        x = chebyshev(lv["K"], Dinv, b, None, self.degree, lo, hi)
        r = b - lv["K"] @ x
        x = x + lv["P"] @ self.vcycle(lv["P"].T @ r, level - 1)
        return chebyshev(lv["K"], Dinv, b, x, self.degree, lo, hi)

    def apply_inverse(self, r):
        """alpha-free Cahouet-Chabard term: K_p^{-1} r by one V-cycle, constrained entries zero."""
        c = self.levels[-1]["c"]
        y = self.vcycle(np.where(c, 0.0, r))
        return np.where(c, 0.0, y)
