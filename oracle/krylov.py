"""Right-preconditioned FGMRES with CGS2 and the block-triangular Stokes preconditioner (oracle).

TEST INFRASTRUCTURE: only tests, smoke() and bench.py's CPU-baseline leg use this.

Sec. 5 ("Linear solver settings") solves the saddle system of Eq.
"stokes-discrete-block" with FGMRES preconditioned by the multilevel method of
Sec. 4; it stops on the Euclidean norm of the residual.  Readings taken here:

* stopping test: relative residual ||r|| / ||b|| <= tol (zero initial guess by
  default), with the implicit (Givens) estimate during the cycle and an explicit
  check b - K x at exit; if the explicit check fails, the method restarts, at
  most 3 extra times;
* restart length m = 50; orthogonalisation = classical Gram-Schmidt applied twice ("cgs2");
  option "selective": the second pass only when the new vector's norm drops below 1/sqrt(2)
  of its value before the projection (Daniel-Gragg-Kaufman-Stewart criterion);
* Schur approximation S^{-1} ~ M_p(1/eta)^{-1} (+ alpha K_p^{-1}, Cahouet-Chabard, when alpha > 0;
  see pressure.py; K_p^{-1} by one V-cycle with Chebyshev degree 2, which keeps the FGMRES
  iteration count of degree 4 on the channel workload);
* preconditioner (block upper triangular):  z_p = -S^{-1} r_p,
  z_u = V-cycle(r_u - B^T z_p); on constrained entries (identity rows of K) z = r;
  precond="monolithic": Sec. 4's own preconditioner, n V-cycles of saddle-point multigrid with
  the block smoother K_j (monolithic.py), constrained entries and pressure mean as above;
* pure-Dirichlet problems have the constant pressure in the kernel; the mean of
  the free pressure entries is subtracted from every preconditioned vector and
  from the final iterate.

Parity pins (tests): brute-force dense solve of the full saddle system on tiny
meshes; one-iteration convergence with an exact preconditioner; unpreconditioned
convergence within the dimension of the space.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse.linalg as spla

from .fem import System
from .mesh import Mesh
from .mg import Hierarchy, schur_apply_inv
from .pressure import PressureHierarchy


REORTH_KAPPA = 1.0 / math.sqrt(2.0)


def fgmres(apply_K, apply_M, b, x0=None, tol=1e-8, restart=50, max_iter=1000, max_extra=3,
           orth="cgs2"):
    """Returns (x, iterations, explicit relative residual, history of implicit estimates).

    orth = "cgs2": classical Gram-Schmidt applied twice; "selective": classical Gram-Schmidt
    with a second pass only when the norm of the new vector drops below 1/sqrt(2) of its norm
    before the projection (Daniel, Gragg, Kaufman, Stewart 1976)."""
    n = len(b)
    bnorm = float(np.linalg.norm(b))
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float)
    if bnorm == 0.0:
        return np.zeros(n), 0, 0.0, []
    it = 0
    extra = 0
    hist = []
    while True:
        r = b - apply_K(x)
        beta = float(np.linalg.norm(r))
        if beta / bnorm <= tol or it >= max_iter:
            return x, it, beta / bnorm, hist
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        converged = False
        for j in range(restart):
            Z[j] = apply_M(V[j])
            w = apply_K(Z[j])
            wn0 = float(np.linalg.norm(w))
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            hn = float(np.linalg.norm(w))
            if orth == "cgs2" or hn < REORTH_KAPPA * wn0:
                h2 = V[:j + 1] @ w
                w = w - V[:j + 1].T @ h2
                h = h + h2
                hn = float(np.linalg.norm(w))
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rr = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / rr
            sn[j] = H[j + 1, j] / rr
            H[j, j] = rr
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or hn == 0.0:
                converged = True
                break
            if it >= max_iter:
                break
            V[j + 1] = w / hn
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        if converged:
            rel = float(np.linalg.norm(b - apply_K(x))) / bnorm
            if rel <= tol or extra >= max_extra:
                return x, it, rel, hist
            extra += 1
        elif it >= max_iter:
            rel = float(np.linalg.norm(b - apply_K(x))) / bnorm
            return x, it, rel, hist


class StokesOracle:
    """FP64 reference solver for one problem: assembled system + velocity hierarchy."""

    def __init__(self, mesh: Mesh, eta, alpha, levels, degree=4, seed=0, restart=50, schur="auto",
                 coarse="cholesky", orth="cgs2", pdegree=2, deflate=False, precond="block", smooth=2, cycles=1):
        self.mesh = mesh
        # alpha: a scalar, or one value per cell (then the Cahouet-Chabard term is
        # K_p(1/alpha)^{-1} = abar (K_p^w)^{-1}, w = abar / alpha_K, abar = max alpha; pressure.py)
        self.alpha_cells = alpha if np.ndim(alpha) > 0 else None
        self.alpha = float(np.max(alpha)) if np.ndim(alpha) > 0 else float(alpha)
        self.sys = System(mesh, eta, alpha)
        self.levels = levels
        self.restart = restart
        self.orth = orth
        # precond = "block": the block-triangular variant below; "monolithic": Sec. 4's saddle-point
        # multigrid with the block smoother K_j (monolithic.py), m = smooth, n = cycles
        self.mono = None
        if precond == "monolithic":
            from .monolithic import MonolithicHierarchy
            self.mono = MonolithicHierarchy(mesh, eta, alpha, levels, degree=degree, smooth=smooth, cycles=cycles,
                                            seed=seed, coarse="chebyshev" if coarse == "chebyshev" else "dense")
            self.mg = self.mono.vel
            self.schur = "mono"
            self.pmg = None
            self.nullspace = mesh.has_pressure_nullspace()
            self.free_p = ~self.sys.p_constrained
            return
        self.mg = Hierarchy(mesh, eta, alpha, levels, degree=degree, seed=seed, coarse=coarse, deflate=deflate)
        # Schur approximation: "mass" = M_p(1/eta) only; "cc" = Cahouet-Chabard
        # M_p(1/eta)^{-1} + alpha K_p^{-1}; "auto" = cc when alpha > 0
        self.schur = ("cc" if self.alpha > 0 else "mass") if schur == "auto" else schur
        self.pmg = (PressureHierarchy(mesh, levels, degree=pdegree, seed=seed, coarse=coarse, alpha=self.alpha_cells)
                    if self.schur == "cc" else None)
        # the finest level of the hierarchy re-assembles A; both are identical by construction
        self.nullspace = mesh.has_pressure_nullspace()
        self.free_p = ~self.sys.p_constrained

    def project(self, x):
        if not self.nullspace:
            return x
        x = x.copy()
        n_u = self.mesh.n_u
        p = x[n_u:]
        p[self.free_p] -= p[self.free_p].mean()
        return x

    def apply_K(self, x):
        return self.sys.K @ x

    def precond(self, r):
        if self.mono is not None:
            z = self.mono.apply(r)
            z[self.sys.constrained] = r[self.sys.constrained]
            return self.project(z)
        n_u = self.mesh.n_u
        ru, rp = r[:n_u], r[n_u:]
        zp = -schur_apply_inv(self.sys.Mpw, rp, self.mesh.dim)
        if self.pmg is not None:
            zp = zp - self.alpha * self.pmg.apply_inverse(rp)
        zu = self.mg.vcycle(ru - self.sys.B.T @ zp)
        z = np.concatenate([zu, zp])
        # K is the identity on constrained rows: invert that block exactly
        z[self.sys.constrained] = r[self.sys.constrained]
        return self.project(z)

    def solve(self, b, tol=1e-8, x0=None, max_iter=1000):
        x, it, rel, hist = fgmres(self.apply_K, self.precond, b, x0, tol, self.restart, max_iter,
                                  orth=self.orth)
        return self.project(x), it, rel, hist


def normalize_pressure(mesh: Mesh, sysm: System, x):
    """Shift the pressure so that int p dx = 1^T M_p p = 0 (comparison of pure-Dirichlet solutions)."""
    x = x.copy()
    n_u = mesh.n_u
    p = x[n_u:]
    free = ~sysm.p_constrained
    w = sysm.Mp1 @ np.ones(mesh.Np)
    c = (w[free] @ p[free]) / w[free].sum()
    p[free] -= c
    return x


def direct_solve(sysm: System, b):
    """Sparse direct solve of K x = b; with a pressure null space the system is bordered by the
    constraint sum of free pressure entries = 0."""
    mesh = sysm.mesh
    K = sysm.K
    if mesh.has_pressure_nullspace():
        import scipy.sparse as sp
        e = np.zeros(mesh.N)
        e[mesh.n_u:][~sysm.p_constrained] = 1.0
        Kb = sp.bmat([[K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]]).tocsc()
        sol = spla.spsolve(Kb, np.concatenate([b, [0.0]]))
        return sol[:-1]
    return spla.spsolve(K.tocsc(), b)
