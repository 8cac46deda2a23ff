"""Mesh-extension solve: CG preconditioned by the velocity multigrid (oracle).

TEST INFRASTRUCTURE: only tests, smoke() and bench.py's CPU-baseline leg use this.

Sec. 2 extends the solid displacement into the fluid by the pseudo-elastic problem of Eq.
"extenstion": -div(mu_A eps(u)) = 0 in the fluid, u = u_s on the solid boundary, u = 0 on the
rest of the fluid boundary.  Sec. 5 solves it by CG preconditioned with a matrix-free multigrid
with a fourth-order Chebyshev smoother based on the diagonal, and stops when the Euclidean norm
of the residual drops below 1e-6; Eq. "mu_distribution" gives the coefficient
mu_A = 1 + 50 exp(-800 ((x - A_x)^2 + (y - A_y)^2)).

Readings taken here:

* the weak form int mu_A eps(u) : eps(v) is the velocity block A of this library with alpha = 0
  and eta_K = mu_A(centroid of K) / 2 (A carries 2 eta eps : eps); the solid cells are obstacle
  cells, their nodes carry u_s as Dirichlet data, every outer face is Dirichlet (u = 0);
* preconditioner: one V-cycle of the velocity hierarchy (mg.py: Chebyshev degree 4, one pre- and
  one post-smoothing call, dense coarse solve); constrained rows are identity rows, z = r there;
* CG in its flexible (Polak-Ribiere) form, beta = z_new . (r_new - r_old) / (z_old . r_old): for
  a fixed SPD preconditioner it is the textbook PCG in exact arithmetic, and it stays robust when
  the preconditioner is applied in lower precision;
* stopping test: ||r|| / ||b|| <= tol (relative, as for the Stokes solve); x0 = the Dirichlet
  data on constrained rows, 0 elsewhere.

Parity pins (tests): with the exact inverse as preconditioner CG stops after one step; without
a preconditioner it solves an n x n SPD system within n steps; the multigrid-preconditioned
solution equals the sparse direct solution; rigid motions have eps = 0, so with rigid-motion
boundary data the discrete extension is that rigid motion for any mu_A.
"""
from __future__ import annotations

import numpy as np

from .fem import System
from .mesh import Mesh
from .mg import Hierarchy


def pcg(apply_A, apply_M, b, x0=None, tol=1e-6, max_iter=1000):
    """Flexible preconditioned CG; returns (x, iterations, relative residual ||b - A x|| / ||b||)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=float)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - apply_A(x)
    if np.linalg.norm(r) / bnorm <= tol:
        return x, 0, float(np.linalg.norm(r)) / bnorm
    z = apply_M(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < max_iter:
        q = apply_A(p)
        a = rz / float(p @ q)
        x = x + a * p
        r_old = r
        r = r - a * q
        it += 1
        if np.linalg.norm(r) / bnorm <= tol:
            break
        z = apply_M(r)
        beta = float(z @ (r - r_old)) / rz
        rz = float(r @ z)
        p = z + beta * p
    return x, it, float(np.linalg.norm(b - apply_A(x))) / bnorm


class ExtensionOracle:
    """A u = b on the velocity block (alpha = 0, eta = mu_A / 2), CG + velocity V-cycle."""

    def __init__(self, mesh: Mesh, eta, levels, degree=4, seed=0):
        self.mesh = mesh
        self.sys = System(mesh, eta, 0.0, need_pressure=False)
        self.mg = Hierarchy(mesh, eta, 0.0, levels, degree=degree, seed=seed)
        self.con = self.sys.u_constrained

    def apply_A(self, x):
        return self.sys.A @ x

    def precond(self, r):
        z = self.mg.vcycle(r)
        z[self.con] = r[self.con]
        return z

    def lift_rhs(self, g_u):
        """b = -A_raw g on free rows, g on constrained rows (Dirichlet data u_s and 0)."""
        gc = np.where(self.con, g_u, 0.0)
        b = -(self.sys.A_raw @ gc)
        return np.where(self.con, g_u, b)

    def solve(self, b, tol=1e-6, max_iter=1000):
        """x0 = b on the constrained (identity) rows, 0 elsewhere: the residual vanishes there and
        stays zero, so the Dirichlet data is reproduced exactly."""
        x0 = np.where(self.con, b, 0.0)
        return pcg(self.apply_A, self.precond, b, x0=x0, tol=tol, max_iter=max_iter)
