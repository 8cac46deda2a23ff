"""Geometric multigrid pieces for the velocity block (oracle).

TEST INFRASTRUCTURE: only tests, smoke() and bench.py's CPU-baseline leg use this.

Sec. 4 builds the preconditioner on nested meshes T_0 (coarsest) ... T_J obtained
by uniform refinement, and applies the viscous block through k_A steps of the
Chebyshev smoother preconditioned with diag(A), Cheb(A, diag(A), k_A), after
Adams et al. (2003), with zero initial guesses for inner iterations.  The
velocity-only V-cycle and the eta^{-1}-weighted pressure-mass Schur
approximation are the block-triangular variant this library solves; the paper
is silent on several details, read here as follows:

* coarse operators are rediscretised on each level (no Galerkin products);
  coarse eta = mean of the active children; a coarse cell is an obstacle cell
  iff all children are;
* prolongation = Q2 interpolation of the coarse field at the fine nodes,
  with constrained fine rows and constrained coarse columns removed;
  restriction = its transpose;
* Chebyshev interval [lambda_hi / 15, lambda_hi], lambda_hi = 1.2 * the largest
  Ritz value of 12 Lanczos steps on D^{-1/2} A D^{-1/2} from a start vector drawn
  with SplitMix64 (constrained entries zeroed);
* one pre- and one post-smoothing Chebyshev call per level, degree k_A = 4
  (Table "NS-solver-parameters-1", predictor column);
* coarsest level solved exactly by a dense FP64 Cholesky factorisation (option: Chebyshev
  smoothing only, for meshes whose coarsest level is too large to factor);
* Schur approximation S^ = M_p(1/eta); S^{-1} applied by 4 Chebyshev-Jacobi
  steps on the fixed interval [2^-d, (3/2)^d] (Wathen's bounds for the
  Jacobi-scaled Q1 mass matrix, which hold for any positive cell weights).

Parity pins (tests): prolongation reproduces quadratics exactly and matches the
1D stencil (3/8, 3/4, -1/8); restriction is the bitwise transpose; Chebyshev on
a diagonal matrix equals the closed form T_k((theta - lambda)/delta) /
T_k(theta/delta); Lanczos Ritz values are bracketed by the dense spectrum; the
V-cycle is a symmetric operator and contracts the error; Wathen bounds hold.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .fem import Q2_NODES, System, lagrange_1d
from .mesh import Mesh, coarsen_eta

MASK64 = (1 << 64) - 1


def splitmix64(z: int) -> int:
    """One output of the SplitMix64 generator (Steele, Lea, Flood, OOPSLA 2014) for state z."""
    z = (z + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def lanczos_start(n: int, seed: int, level: int) -> np.ndarray:
    """Uniform(-1, 1) start vector: entry i = 2 * (splitmix64(c_i) >> 11) * 2^-53 - 1 with the
    64-bit counter c_i = ((seed mod 2^32) << 32) XOR ((level mod 256) << 56) XOR i."""
    base = ((seed & 0xFFFFFFFF) << 32) ^ ((level & 0xFF) << 56)
    z = np.uint64(base) ^ np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return 2.0 * ((z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)) - 1.0


def prolongation_1d(n_coarse: int) -> sp.csr_matrix:
    """(4 n_c + 1) x (2 n_c + 1) matrix: fine node I lies in coarse cell c at local position
    t in {0, 1/4, 1/2, 3/4, 1}; its row holds the coarse Q2 basis values at t."""
    nf = 4 * n_coarse + 1
    rows, cols, vals = [], [], []
    for I in range(nf):
        c = min(I // 4, n_coarse - 1)
        t = (I - 4 * c) / 4.0
        v, _ = lagrange_1d(Q2_NODES, [t])
        for a in range(3):
            if v[a, 0] != 0.0:
                rows.append(I)
                cols.append(2 * c + a)
                vals.append(v[a, 0])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, 2 * n_coarse + 1))


def prolongation(coarse: Mesh, fine: Mesh) -> sp.csr_matrix:
    P1 = [prolongation_1d(coarse.n[a]) for a in range(coarse.dim)]
    Ps = P1[0]
    for a in range(1, coarse.dim):
        Ps = sp.kron(P1[a], Ps)  # x fastest: later axes are the outer Kronecker factors
    Ps = Ps.tocsr()
    keep_f = sp.diags((~fine.vnode_constrained()).astype(float))
    keep_c = sp.diags((~coarse.vnode_constrained()).astype(float))
    Ps = (keep_f @ Ps @ keep_c).tocsr()
    Ps.eliminate_zeros()
    return sp.block_diag([Ps] * coarse.dim).tocsr()


class Level:
    def __init__(self, mesh: Mesh, eta, alpha, index):
        self.mesh = mesh
        self.eta = eta
        self.alpha = alpha
        self.index = index
        self.sys = System(mesh, eta, alpha, need_pressure=False)
        self.A = self.sys.A
        self.D = self.A.diagonal()
        self.P = None          # prolongation from level index-1
        self.lam_hi = None
        self.chol = None


def lanczos_max(A, D, v0, steps=12):
    """Largest Ritz value after `steps` Lanczos steps on S = D^{-1/2} A D^{-1/2}."""
    s = 1.0 / np.sqrt(D)
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    beta_prev = 0.0
    alphas, betas = [], []
    for j in range(steps):
        w = s * (A @ (s * v)) - beta_prev * v_prev
        a = w @ v
        w = w - a * v
        b = np.linalg.norm(w)
        alphas.append(a)
        if j == steps - 1 or b == 0.0:
            break
        betas.append(b)
        v_prev, v, beta_prev = v, w / b, b
    T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
    return float(np.linalg.eigvalsh(T)[-1])


def chebyshev(A, Dinv, b, x0, degree, lam_lo, lam_hi):
    """Chebyshev iteration preconditioned with D (Saad, Iterative Methods, Alg. 12.1) as used
    for Cheb(M, D, k): degree k updates of x; the residual is recomputed as b - A x."""
    theta = 0.5 * (lam_hi + lam_lo)
    delta = 0.5 * (lam_hi - lam_lo)
    sigma = theta / delta
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b.copy() if x0 is None else b - A @ x
    rho = 1.0 / sigma
    d = Dinv * r / theta
    for t in range(1, degree + 1):
        x = x + d
        if t < degree:
            r = b - A @ x
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * (Dinv * r)
            rho = rho_new
    return x


class Hierarchy:
    """Velocity multigrid hierarchy, levels[0] = coarsest."""

    def __init__(self, fine: Mesh, eta_fine, alpha, nlevels, degree=4, seed=0,
                 lanczos_steps=12, safety=1.2, ratio=15.0, coarse="cholesky", deflate=False):
        meshes = [fine]
        etas = [np.asarray(eta_fine, dtype=float)]
        # per-cell alpha (rho_s != rho_f) is coarsened like eta: mean of the active children
        per_cell = np.ndim(alpha) > 0
        alphas = [np.asarray(alpha, dtype=float) if per_cell else alpha]
        for _ in range(nlevels - 1):
            c = meshes[-1].coarsen()
            etas.append(coarsen_eta(meshes[-1], c, etas[-1]))
            alphas.append(coarsen_eta(meshes[-1], c, alphas[-1]) if per_cell else alpha)
            meshes.append(c)
        meshes, etas, alphas = meshes[::-1], etas[::-1], alphas[::-1]
        self.degree = degree
        self.ratio = ratio
        self.levels = [Level(m, e, a, i) for i, (m, e, a) in enumerate(zip(meshes, etas, alphas))]
        for i in range(1, len(self.levels)):
            self.levels[i].P = prolongation(meshes[i - 1], meshes[i])
        self.coarse = coarse
        for lv in self.levels[(0 if coarse == "chebyshev" else 1):]:
            v0 = lanczos_start(lv.mesh.n_u, seed, lv.index)
            v0[lv.sys.u_constrained] = 0.0
            lv.lam_hi = safety * lanczos_max(lv.A, lv.D, v0, lanczos_steps)
        if coarse == "cholesky":
            A0 = self.levels[0].A.toarray()
            self.levels[0].chol = sla.cho_factor(A0, lower=True)
        # rigid-body deflation of stiff inclusions on the finest level (deflation.py)
        self.defl = None
        if deflate:
            from .deflation import Deflation
            fl = self.levels[-1]
            self.defl = Deflation(fl.mesh, fl.eta, fl.A)

    def vcycle(self, b, level=None):
        """Velocity V-cycle V(l, b) (Sec. 4): pre-smooth from 0, residual, restrict, recurse,
        prolongate and add, post-smooth."""
        if level is None:
            level = len(self.levels) - 1
        lv = self.levels[level]
        if level == 0:
            if self.coarse == "chebyshev":   # smoothing only, for coarse meshes too large to factor
                return chebyshev(lv.A, 1.0 / lv.D, b, None, self.degree, lv.lam_hi / self.ratio, lv.lam_hi)
            return sla.cho_solve(lv.chol, b)
        lo, hi = lv.lam_hi / self.ratio, lv.lam_hi
        Dinv = 1.0 / lv.D
        x = chebyshev(lv.A, Dinv, b, None, self.degree, lo, hi)
        r = b - lv.A @ x
        rc = lv.P.T @ r
        x = x + lv.P @ self.vcycle(rc, level - 1)
        if self.defl is not None and level == len(self.levels) - 1:
            x = x + self.defl.correction(r)
        x = chebyshev(lv.A, Dinv, b, x, self.degree, lo, hi)
        return x


def schur_apply_inv(Mpw, r, dim, degree=4):
    """S^{-1} r ~ Cheb(M_p(1/eta), diag, degree) from zero on the interval [2^-d, (3/2)^d]."""
    D = Mpw.diagonal()
    return chebyshev(Mpw, 1.0 / D, r, None, degree, 0.5 ** dim, 1.5 ** dim)
