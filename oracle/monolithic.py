"""Monolithic multigrid on the saddle system with the block smoother K_j (oracle).

TEST INFRASTRUCTURE: only tests, smoke() and bench.py's CPU-baseline leg use this.

Sec. 4 preconditions FGMRES with n V-cycles of multigrid on the whole saddle matrix
M_j = [A_j B_j^T; B_j 0] of every level (Zulehner's class of smoothers), each level smoothing
with m steps of the block smoother of Eq. "smoother",

    K_j = [Ahat  B^T ; B  B Ahat^{-1} B^T - Shat]^{-1},

where Ahat^{-1} = Cheb(A, diag A, k_A) and Shat^{-1} = ChebMINRES(n_S, k_S): n_S steps of MINRES
on S = B Ahat^{-1} B^T, preconditioned by Cheb(S, diag(B diag(A)^{-1} B^T), k_S), all from zero.
Table "NS-solver-parameters-1" fixes n = 1, m = 2, k_A = 4, n_S = 1, k_S = 1 (predictor).

Readings taken here (the paper gives the ingredients, not the loop):

* K_j is applied through its factorisation [Ahat 0; B -Shat] [I Ahat^{-1} B^T; 0 I]:
      w~  = Ahat^{-1} r_u,   w_p = Shat^{-1} (B w~ - r_p),   w_u = w~ - Ahat^{-1} B^T w_p,
  which takes the two Ahat solves and the one Shat solve that Sec. 4 counts;
* one smoothing step is x <- x + K_j (b - M_j x); m steps before the coarse correction (the
  first one from x = 0) and m after it; n cycles are the stationary iteration
  x <- x + V(b - M x) from x = 0;
* transfers: Q2 interpolation for the velocity (mg.prolongation) and Q1 interpolation for the
  pressure, rows and columns of constrained nodes removed; restriction = transpose;
* coarsest level: dense solve of M_0 on its free unknowns.  With every face Dirichlet the
  constant pressure is in the kernel of M_0; its pressure block then gets -1 1^T / n_free, which
  leaves the mean-free solution of a consistent system unchanged.  Option "chebyshev": m
  smoothing steps from zero instead (coarse meshes too large to factor);
* Ahat uses the velocity hierarchy's Chebyshev bounds [lambda_hi / 15, lambda_hi] (mg.py);
* k_S = 1: one Chebyshev step from zero is D_S^{-1} r / theta, and MINRES does not depend on a
  positive scaling of its preconditioner, so theta = 1 and no eigenvalue bound of S is needed;
  other k_S are not provided;
* diag(B diag(A)^{-1} B^T) is zero on constrained pressure nodes (their rows of B vanish); its
  inverse is taken as zero there, so the smoother leaves those entries at zero.  Constrained
  rows of M_j are identity rows that never couple to free entries; the preconditioner returns
  z = r on them, as the block-triangular one does.

Corrector mode (option corrector = (v°, rho), Sec. 4 for a non-symmetric A): every level's
velocity block is the corrector block of corrector.py (convection by v° injected to the level,
streamline diffusion), diag and the Chebyshev bounds are those of that block (Lanczos on its
symmetric part), and Shat^{-1} = ChebBiCGStab(n_S, k_S = 1): n_S BiCGStab steps on
S = B Ahat^{-1} B^T with the same preconditioner (the paper replaces MINRES by BiCGStab when A is
not symmetric).

Parity pins (tests): the smoother inverts the block matrix of Eq. "smoother" when Shat^{-1} is
an exact inverse; one MINRES step equals the closed-form minimiser of the preconditioned
residual norm, is invariant to scaling the preconditioner, and n MINRES steps solve an n x n
SPD system; diag(B D^{-1} B^T) equals the dense triple product; the coarse solve satisfies
M_0 x = b; a one-level hierarchy is an exact preconditioner; without smoothing a two-level
cycle is the dense coarse-grid correction P M_0^{-1} P^T; FGMRES reaches the direct solution.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .fem import System
from .mesh import Mesh
from .mg import Hierarchy, chebyshev, lanczos_max, lanczos_start
from .pressure import q1_prolongation


def bicgstab(apply_S, apply_P, b, steps):
    """`steps` iterations of preconditioned BiCGStab for S x = b from x = 0 (van der Vorst 1992, with
    the preconditioner P applied to the search directions; shadow residual = b)."""
    x = np.zeros_like(b)
    r = b.copy()
    rh = b.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for _ in range(steps):
        rho_new = float(rh @ r)
        if rho_new == 0.0:
            break
        beta = (rho_new / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = apply_P(p)
        v = apply_S(ph)
        den = float(rh @ v)
        if den == 0.0:
            break
        alpha = rho_new / den
        s_ = r - alpha * v
        sh = apply_P(s_)
        t = apply_S(sh)
        tt = float(t @ t)
        omega = float(t @ s_) / tt if tt > 0.0 else 0.0
        x = x + alpha * ph + omega * sh
        r = s_ - omega * t
        rho_old = rho_new
        if omega == 0.0:
            break
    return x


def minres(apply_S, apply_P, b, steps):
    """`steps` iterations of preconditioned MINRES for S x = b from x = 0 (S symmetric, P = the
    preconditioner's inverse action, symmetric positive definite): each iterate minimises the
    P-norm of the residual, sqrt(r^T P r), over the preconditioned Krylov space (Paige-Saunders
    recurrences in the preconditioned form of Elman, Silvester and Wathen, Sec. 4.2)."""
    x = np.zeros_like(b)
    v_prev = np.zeros_like(b)
    v = b.copy()
    z = apply_P(v)
    gamma = float(np.sqrt(max(z @ v, 0.0)))
    if gamma == 0.0:
        return x
    eta = gamma
    gamma_prev = 1.0
    c_prev = c = 1.0
    s_prev = s = 0.0
    w_prev = np.zeros_like(b)
    w = np.zeros_like(b)
    for _ in range(steps):
        z = z / gamma
        Sz = apply_S(z)
        delta = float(Sz @ z)
        v_new = Sz - (delta / gamma) * v - (gamma / gamma_prev) * v_prev
        z_new = apply_P(v_new)
        gamma_new = float(np.sqrt(max(z_new @ v_new, 0.0)))
        # QR factorisation of the Lanczos tridiagonal by Givens rotations
        a0 = c * delta - c_prev * s * gamma
        a1 = float(np.hypot(a0, gamma_new))
        a2 = s * delta + c_prev * c * gamma
        a3 = s_prev * gamma
        if a1 == 0.0:
            break
        c_new, s_new = a0 / a1, gamma_new / a1
        w_new = (z - a3 * w_prev - a2 * w) / a1
        x = x + c_new * eta * w_new
        eta = -s_new * eta
        if gamma_new == 0.0:
            break
        v_prev, v, z = v, v_new, z_new
        gamma_prev, gamma = gamma, gamma_new
        c_prev, c, s_prev, s = c, c_new, s, s_new
        w_prev, w = w, w_new
    return x


class SaddleLevel:
    def __init__(self, mesh: Mesh, eta, alpha, index, A=None):
        """A: the level's velocity block when it is not System's (corrector mode)."""
        self.mesh = mesh
        self.index = index
        self.sys = System(mesh, eta, alpha)
        self.A = self.sys.A if A is None else A
        self.K = self.sys.K if A is None else sp.bmat([[A, self.sys.B.T], [self.sys.B, self.sys.C]]).tocsr()
        self.B = self.sys.B
        self.n_u = mesh.n_u
        self.Pp = None  # pressure prolongation from level index-1
        self.Pu = None
        self.D = self.A.diagonal()
        self.lam_hi = None
        # D_S = diag(B diag(A)^{-1} B^T): sum over velocity entries j of B_qj^2 / A_jj
        D = self.D
        ds = np.asarray(self.B.multiply(self.B) @ (1.0 / D)).ravel()
        self.ds = ds
        self.dsinv = np.where(ds > 0.0, 1.0 / np.where(ds > 0.0, ds, 1.0), 0.0)


class MonolithicHierarchy:
    """Saddle-point multigrid of Sec. 4, levels[0] = coarsest."""

    def __init__(self, fine: Mesh, eta_fine, alpha, nlevels, degree=4, smooth=2, cycles=1, schur_steps=1,
                 seed=0, coarse="dense", corrector=None):
        self.vel = Hierarchy(fine, eta_fine, alpha, nlevels, degree=degree, seed=seed,
                             coarse="chebyshev" if coarse == "chebyshev" else "cholesky")
        meshes = [lv.mesh for lv in self.vel.levels]
        etas = [lv.eta for lv in self.vel.levels]
        alphas = [lv.alpha for lv in self.vel.levels]
        self.degree = degree
        self.smooth = smooth
        self.cycles = cycles
        self.schur_steps = schur_steps
        self.coarse = coarse
        self.corrector = corrector is not None
        blocks = [None] * len(meshes)
        if corrector is not None:
            from .corrector import convection_matrices, inject
            from .fem import _eliminate
            vcirc, rho = corrector
            fields = [np.asarray(vcirc, dtype=float)]
            for i in range(len(meshes) - 1, 0, -1):
                fields.append(inject(meshes[i], meshes[i - 1], fields[-1]))
            fields = fields[::-1]
            for i, lv in enumerate(self.vel.levels):
                Craw, Sraw = convection_matrices(lv.mesh, fields[i], lv.eta, rho)
                blocks[i] = _eliminate((lv.sys.A_raw + Craw + Sraw).tocsr(), lv.sys.u_constrained)
        self.levels = [SaddleLevel(m, e, a, i, blocks[i]) for i, (m, e, a) in enumerate(zip(meshes, etas, alphas))]
        for i, lv in enumerate(self.levels):
            if corrector is None:
                lv.lam_hi = self.vel.levels[i].lam_hi
            elif i > 0 or coarse == "chebyshev":
                v0 = lanczos_start(lv.mesh.n_u, seed, i)
                v0[lv.sys.u_constrained] = 0.0
                lv.lam_hi = 1.2 * lanczos_max(((lv.A + lv.A.T) * 0.5).tocsr(), lv.D, v0, 12)
        for i in range(1, len(self.levels)):
            lo, hi = self.levels[i - 1], self.levels[i]
            hi.Pu = self.vel.levels[i].P
            hi.Pp = q1_prolongation(lo.mesh, hi.mesh, lo.sys.p_constrained, hi.sys.p_constrained)
        self.nullspace = fine.has_pressure_nullspace()
        if coarse == "dense":
            c0 = self.levels[0]
            free = ~c0.sys.constrained
            M0 = c0.K.toarray()[np.ix_(free, free)]
            if self.nullspace:
                e = (np.arange(c0.mesh.N) >= c0.n_u)[free].astype(float)
                M0 = M0 - np.outer(e, e) / e.sum()
            self.coarse_free = free
            self.coarse_lu = sla.lu_factor(M0)

    # ---- pieces ----------------------------------------------------------------------------------
    def ahat_inv(self, level, r):
        """Ahat^{-1} r = Cheb(A, diag A, k_A) from zero."""
        lv = self.levels[level]
        return chebyshev(lv.A, 1.0 / lv.D, r, None, self.degree, lv.lam_hi / self.vel.ratio, lv.lam_hi)

    def schur_inv(self, level, v):
        """Shat^{-1} v = ChebMINRES(n_S, k_S = 1): MINRES on S = B Ahat^{-1} B^T, preconditioner
        one Chebyshev step with diag(B diag(A)^{-1} B^T)."""
        lv = self.levels[level]
        B = lv.B
        krylov = bicgstab if self.corrector else minres   # ChebBiCGStab for a non-symmetric A
        return krylov(lambda z: B @ self.ahat_inv(level, B.T @ z), lambda r: lv.dsinv * r, v, self.schur_steps)

    def smoother(self, level, r, schur=None):
        """w = K_j r (Eq. "smoother") by the block factorisation; `schur` replaces Shat^{-1}."""
        lv = self.levels[level]
        n_u = lv.n_u
        ru, rp = r[:n_u], r[n_u:]
        B = lv.B
        wt = self.ahat_inv(level, ru)
        v = B @ wt - rp
        wp = self.schur_inv(level, v) if schur is None else schur(v)
        wu = wt - self.ahat_inv(level, B.T @ wp)
        return np.concatenate([wu, wp])

    def coarse_solve(self, b):
        c0 = self.levels[0]
        x = np.zeros(c0.mesh.N)
        x[self.coarse_free] = sla.lu_solve(self.coarse_lu, b[self.coarse_free])
        return x

    def vcycle(self, b, level=None):
        """One V-cycle of the saddle-point multigrid on level `level` for right-hand side b."""
        if level is None:
            level = len(self.levels) - 1
        lv = self.levels[level]
        if level == 0 and self.coarse == "dense":
            return self.coarse_solve(b)
        x = np.zeros_like(b)
        for s in range(self.smooth):
            x = x + self.smoother(level, b if s == 0 else b - lv.K @ x)
        if level == 0:
            return x
        cl = self.levels[level - 1]
        n_u, nc_u = lv.n_u, cl.n_u
        r = b - lv.K @ x
        rc = np.concatenate([lv.Pu.T @ r[:n_u], lv.Pp.T @ r[n_u:]])
        ec = self.vcycle(rc, level - 1)
        x = x + np.concatenate([lv.Pu @ ec[:nc_u], lv.Pp @ ec[nc_u:]])
        for _ in range(self.smooth):
            x = x + self.smoother(level, b - lv.K @ x)
        return x

    def apply(self, b):
        """n cycles from zero: x <- x + V(b - M x)."""
        lv = self.levels[-1]
        x = self.vcycle(b)
        for _ in range(self.cycles - 1):
            x = x + self.vcycle(b - lv.K @ x)
        return x
