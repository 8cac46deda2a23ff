"""Corrector-mode momentum block: convection by a given velocity and streamline diffusion (oracle).

TEST INFRASTRUCTURE: only tests, smoke() and bench.py's CPU-baseline leg use this.

In the corrector stage (Sec. 3.1.2, Eq. "v_star") the convective velocity is the unknown itself
while v° = v# - w# is given, so the form of Eq. "form_a_j" gains the linear, non-symmetric term
rho ((v° . grad) v, w).  Eq. "a_stab" adds the streamline diffusion
sum_K int_K r_K (v° . grad v) . (v° . grad w) with the cell parameter of Brooks-Hughes, zero where
the cell Peclet number is below 1.  The velocity block becomes

    A_c = alpha M + 2 eta eps:eps + rho C(v°) + rho S(v°, r),

non-symmetric; the saddle system keeps B and B^T.  Readings taken here:

* v° is a Q2 nodal field (the velocity space), evaluated at the 3^d Gauss points of each cell
  (3-point Gauss per direction as for every other cell matrix: exact for the convection term when
  v° has degree <= 1 per direction, not for the streamline term with a quadratic v°);
* |v°|_K = Euclidean norm of v° at the cell centre (the Q2 centre node); h_K = the cell diameter;
  p1 = 2 (Q2); Pe_K = rho |v°|_K h_K / (2 eta_K p1) (the momentum equation as written: convection
  carries rho, the viscous term eta);
* r_K = h_K / (2 |v°|_K p1) xi(Pe_K) with xi(Pe) = coth(Pe) - 1 / Pe (the Brooks-Hughes function;
  the printed formula reads (coth(Pe) - 1) / Pe, which vanishes as Pe grows and would switch the
  stabilisation off where it is needed), r_K = 0 where Pe_K < 1;
* the streamline term is scaled by rho, like the convection it stabilises (rho r (v°.grad v)
  (v°.grad w) has the units of rho (v°.grad v) w);
* coarse levels: v° injected (coarse node I = fine node 2 I), r_K from the coarse cells;
* the block-triangular preconditioner of the predictor mode with A_c in the velocity V-cycle;
  the Chebyshev interval of A_c comes from 12 Lanczos steps on its symmetric part (A_c + A_c^T)/2
  (1.2 safety, [lambda / 15, lambda], as in mg.py); dense LU on the coarsest level.

Parity pins (tests): v° = 0 gives the predictor system; for a constant v° the convection matrix
of a cell equals the Kronecker closed form of the 1D Q2 matrices; for a linear divergence-free
v° with every face Dirichlet the free block of C is skew-symmetric; the streamline term is
symmetric positive semi-definite and vanishes where Pe_K < 1; r_K against the closed form;
FGMRES reaches the sparse direct solution of the non-symmetric system.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .fem import Q2_NODES, System, tensor_basis, _eliminate
from .krylov import fgmres
from .mesh import Mesh
from .mg import Hierarchy, chebyshev, lanczos_max, lanczos_start, schur_apply_inv
from .pressure import PressureHierarchy

P1 = 2  # polynomial degree of the velocity space


def xi(pe):
    """Brooks-Hughes streamline function coth(Pe) - 1 / Pe (Pe > 0)."""
    pe = np.asarray(pe, dtype=float)
    return 1.0 / np.tanh(pe) - 1.0 / pe


def cell_parameters(mesh: Mesh, vcirc, eta, rho):
    """|v°| at the cell centres, Pe_K and r_K for every cell (r_K = 0 where Pe_K < 1)."""
    d = mesh.dim
    centres = mesh.cell_vnodes()[:, (3 ** d) // 2]          # the centre node of each cell
    vn = np.sqrt(sum(vcirc[a * mesh.Nv + centres] ** 2 for a in range(d)))
    hK = float(np.sqrt(sum(hh * hh for hh in mesh.h)))
    eta = np.asarray(eta, dtype=float)
    pe = rho * vn * hK / (2.0 * eta * P1)
    r = np.zeros_like(pe)
    big = pe >= 1.0
    r[big] = hK / (2.0 * vn[big] * P1) * xi(pe[big])
    return vn, pe, r


def convection_matrices(mesh: Mesh, vcirc, eta, rho):
    """Unconstrained rho C(v°) and rho S(v°, r) (n_u x n_u), assembled cell by cell with 3-point Gauss:
    C[i a, j a] = int phi_i (v° . grad phi_j),  S[i a, j a] = r_K int (v° . grad phi_i)(v° . grad phi_j)."""
    d = mesh.dim
    vals, grads, w = tensor_basis(d, mesh.h, Q2_NODES)          # (nq, nb), (nq, nb, d), (nq,)
    act = mesh.active_cells()
    vn = mesh.cell_vnodes()[act]                                 # (nc, nb)
    vloc = np.stack([vcirc[a * mesh.Nv + vn] for a in range(d)], axis=1)  # (nc, d, nb)
    vq = np.einsum("qi,cai->cqa", vals, vloc)                    # v° at the quadrature points
    adv = np.einsum("cqa,qja->cqj", vq, grads)                   # v° . grad phi_j
    Cl = rho * np.einsum("q,qi,cqj->cij", w, vals, adv)
    _, _, r = cell_parameters(mesh, vcirc, eta, rho)
    Sl = rho * r[act][:, None, None] * np.einsum("q,cqi,cqj->cij", w, adv, adv)
    nb = vals.shape[1]
    rows = np.repeat(vn, nb, axis=1)
    cols = np.tile(vn, (1, nb))
    out = []
    for loc in (Cl, Sl):
        blocks = []
        for a in range(d):
            blocks.append(sp.coo_matrix((loc.reshape(len(act), -1).ravel(),
                                         ((rows + a * mesh.Nv).ravel(), (cols + a * mesh.Nv).ravel())),
                                        shape=(mesh.n_u, mesh.n_u)))
        out.append(sum(blocks).tocsr())
    return out[0], out[1]


class CorrectorSystem:
    """Saddle system of the corrector stage: K_c = [[A_c, B^T], [B, C]] with constraints eliminated."""

    def __init__(self, mesh: Mesh, eta, alpha, vcirc, rho):
        self.mesh = mesh
        self.base = System(mesh, eta, alpha)
        Craw, Sraw = convection_matrices(mesh, vcirc, eta, rho)
        self.C_raw, self.S_raw = Craw, Sraw
        vc = self.base.u_constrained
        self.A_raw = (self.base.A_raw + Craw + Sraw).tocsr()
        self.A = _eliminate(self.A_raw, vc)
        b = self.base
        self.B = b.B
        self.K = sp.bmat([[self.A, b.B.T], [b.B, b.C]]).tocsr()
        self.K_raw = sp.bmat([[self.A_raw, b.B_raw.T], [b.B_raw, None]]).tocsr()
        self.constrained = b.constrained
        self.p_constrained = b.p_constrained
        self.Mpw = b.Mpw

    def lift_rhs(self, f, g):
        n_u = self.mesh.n_u
        F = np.concatenate([self.base.Mu @ f[:n_u], self.base.Mp1 @ f[n_u:]])
        gc = np.where(self.constrained, g, 0.0)
        bb = F - self.K_raw @ gc
        return np.where(self.constrained, g, bb)


def inject(fine: Mesh, coarse: Mesh, vcirc):
    """Coarse nodal field: coarse node I takes the fine node 2 I (nested Q2 nodes)."""
    d = fine.dim
    ct = coarse.vnode_tuples()
    fn = fine.vnode_flat(2 * ct)
    return np.concatenate([vcirc[a * fine.Nv + fn] for a in range(d)])


class CorrectorOracle:
    """FGMRES with the block-triangular preconditioner on the corrector system."""

    def __init__(self, mesh: Mesh, eta, alpha, vcirc, rho, levels, degree=4, seed=0, restart=50,
                 lanczos_steps=12, safety=1.2, ratio=15.0, pdegree=2):
        self.mesh = mesh
        self.sys = CorrectorSystem(mesh, eta, alpha, vcirc, rho)
        base = Hierarchy(mesh, eta, alpha, levels, degree=degree, seed=seed)
        self.degree, self.ratio = degree, ratio
        self.levels = []
        v = np.asarray(vcirc, dtype=float)
        fields = [v]
        for i in range(levels - 1, 0, -1):
            fields.append(inject(base.levels[i].mesh, base.levels[i - 1].mesh, fields[-1]))
        fields = fields[::-1]
        for i, lv in enumerate(base.levels):
            Craw, Sraw = convection_matrices(lv.mesh, fields[i], lv.eta, rho)
            A = _eliminate((lv.sys.A_raw + Craw + Sraw).tocsr(), lv.sys.u_constrained)
            D = A.diagonal()
            lam = None
            if i > 0:
                v0 = lanczos_start(lv.mesh.n_u, seed, i)
                v0[lv.sys.u_constrained] = 0.0
                lam = safety * lanczos_max(((A + A.T) * 0.5).tocsr(), D, v0, lanczos_steps)
            self.levels.append(dict(mesh=lv.mesh, A=A, D=D, P=lv.P, lam=lam))
        self.coarse_lu = sla.lu_factor(self.levels[0]["A"].toarray())
        self.alpha = float(np.max(alpha)) if np.ndim(alpha) > 0 else float(alpha)
        self.pmg = PressureHierarchy(mesh, levels, degree=pdegree, seed=seed,
                                     alpha=alpha if np.ndim(alpha) > 0 else None) if self.alpha > 0 else None
        self.restart = restart
        self.nullspace = mesh.has_pressure_nullspace()

    def vcycle(self, b, level=None):
        if level is None:
            level = len(self.levels) - 1
        lv = self.levels[level]
        if level == 0:
            return sla.lu_solve(self.coarse_lu, b)
        A, Dinv = lv["A"], 1.0 / lv["D"]
        lo, hi = lv["lam"] / self.ratio, lv["lam"]
        x = chebyshev(A, Dinv, b, None, self.degree, lo, hi)
        r = b - A @ x
        x = x + lv["P"] @ self.vcycle(lv["P"].T @ r, level - 1)
        return chebyshev(A, Dinv, b, x, self.degree, lo, hi)

    def precond(self, r):
        n_u = self.mesh.n_u
        ru, rp = r[:n_u], r[n_u:]
        zp = -schur_apply_inv(self.sys.Mpw, rp, self.mesh.dim)
        if self.pmg is not None:
            zp = zp - self.alpha * self.pmg.apply_inverse(rp)
        zu = self.vcycle(ru - self.sys.B.T @ zp)
        z = np.concatenate([zu, zp])
        z[self.sys.constrained] = r[self.sys.constrained]
        if self.nullspace:
            p = z[n_u:]
            free = ~self.sys.p_constrained
            p[free] -= p[free].mean()
        return z

    def solve(self, b, tol=1e-8, max_iter=1000):
        return fgmres(lambda x: self.sys.K @ x, self.precond, b, tol=tol, restart=self.restart, max_iter=max_iter)
