"""Q2-Q1 cell matrices by Gauss quadrature and sparse assembly (oracle).

TEST INFRASTRUCTURE: only tests, smoke() and bench.py's CPU-baseline leg use this.

What is computed (the generalized Stokes system of the predictor mode, Sec. 3.1.2,
Eqs. "form_a_j" and "form_b", and its matrix form Eq. "stokes-discrete-block"):

  A[i a, j b] = sum_K  alpha * int_K phi_i phi_j delta_ab
                     + eta_K * int_K 2 eps(phi_j e_b) : eps(phi_i e_a)
  B[q, j b]   = - sum_K int_K psi_q  d(phi_j)/dx_b
  Mp_w[q, r]  = sum_K eta_K^{-1} int_K psi_q psi_r     (Schur approximation)

Readings of the paper: the viscous term carries the factor 2 of the stress
sigma = 2 eta eps - p I (Eq. "const_fluid"); the pressure is the physical one, so
B = -(div u, q) (the paper's p is its negative).  alpha = rho / (gamma tau) is one scalar, or one
value per cell when the solid and fluid densities differ (Sec. 5, FSI2i: rho_s = 10 rho_f); the
mass term is then sum_K alpha_K int_K phi_i phi_j.

Quadrature is tensor-product 3-point Gauss-Legendre, exact for these
polynomial integrands on Cartesian cells.  Constraints are imposed by symmetric
elimination: constrained rows and columns are zeroed and the diagonal set to 1.

Parity pins (tests/test_oracle_*.py): 1D closed forms of the Q2 / Q1 mass and
stiffness matrices, exact symbolic integration of the full cell matrices,
rigid-body kernel of the viscous form, symmetry / positive definiteness,
discrete-divergence invariants, a quadratic patch test, and manufactured-solution
convergence rates O(h^3) (velocity, L2) and O(h^2) (pressure, L2).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .mesh import Mesh

# 3-point Gauss-Legendre rule on [0, 1]
GAUSS3_POINTS = np.array([0.5 - 0.5 * math.sqrt(0.6), 0.5, 0.5 + 0.5 * math.sqrt(0.6)])
GAUSS3_WEIGHTS = np.array([5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0])

Q2_NODES = (0.0, 0.5, 1.0)
Q1_NODES = (0.0, 1.0)


def lagrange_1d(nodes, t):
    """Values and derivatives of the Lagrange polynomials on `nodes` at points t.
    Returns (vals[len(nodes), len(t)], ders[len(nodes), len(t)])."""
    t = np.atleast_1d(np.asarray(t, dtype=float))
    k = len(nodes)
    vals = np.ones((k, len(t)))
    ders = np.zeros((k, len(t)))
    for i in range(k):
        for j in range(k):
            if j == i:
                continue
            vals[i] *= (t - nodes[j]) / (nodes[i] - nodes[j])
        # product rule
        for m in range(k):
            if m == i:
                continue
            term = np.full(len(t), 1.0 / (nodes[i] - nodes[m]))
            for j in range(k):
                if j == i or j == m:
                    continue
                term = term * (t - nodes[j]) / (nodes[i] - nodes[j])
            ders[i] += term
    return vals, ders


def gauss_rule(npts):
    """Gauss-Legendre rule on [0,1] (npts = 3 uses the closed form above)."""
    if npts == 3:
        return GAUSS3_POINTS.copy(), GAUSS3_WEIGHTS.copy()
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (x + 1.0), 0.5 * w


def tensor_basis(dim, h, nodes, npts=3):
    """Values (nq, nb) and physical gradients (nq, nb, dim) of the tensor-product Lagrange
    basis on the cell [0,h_0] x ... , plus quadrature weights (nq,) including the Jacobian.
    Local basis index a + k b + k^2 c (x fastest); quadrature index likewise."""
    pts, wts = gauss_rule(npts)
    v1, d1 = lagrange_1d(nodes, pts)  # (k, nq1)
    k = len(nodes)
    nb = k ** dim
    nq = npts ** dim
    basis_offs = Mesh.local_offsets(dim, k)
    q_offs = Mesh.local_offsets(dim, npts)
    vals = np.ones((nq, nb))
    grads = np.ones((nq, nb, dim))
    w = np.ones(nq)
    for q in range(nq):
        for a in range(dim):
            w[q] *= wts[q_offs[q, a]] * h[a]
    for q in range(nq):
        for b in range(nb):
            for a in range(dim):
                vals[q, b] *= v1[basis_offs[b, a], q_offs[q, a]]
            for g in range(dim):
                prod = 1.0
                for a in range(dim):
                    if a == g:
                        prod *= d1[basis_offs[b, a], q_offs[q, a]] / h[a]
                    else:
                        prod *= v1[basis_offs[b, a], q_offs[q, a]]
                grads[q, b, g] = prod
    return vals, grads, w


class CellMatrices:
    """Reference matrices of one Cartesian cell with extents h (all cells of a level share them).

    mass   [d nb, d nb]  int phi_i phi_j delta_ab
    visc   [d nb, d nb]  int 2 eps(phi_j e_b) : eps(phi_i e_a)         (eta = 1)
    div    [np, d nb]    -int psi_q d phi_j / d x_b
    pmass  [np, np]      int psi_q psi_r
    Local velocity DoF = a * 3^d + local node; pressure local index as in mesh.py.
    """

    def __init__(self, dim, h, npts=3):
        self.dim = dim
        self.h = tuple(h)
        uv, ug, w = tensor_basis(dim, h, Q2_NODES, npts)
        pv, _, w2 = tensor_basis(dim, h, Q1_NODES, npts)
        assert np.allclose(w, w2)
        nb = uv.shape[1]
        nd = dim * nb
        self.nb = nb
        # symmetric gradients of the vector basis functions Phi_I = phi_i e_a at quadrature points
        eps = np.zeros((len(w), nd, dim, dim))
        for a in range(dim):
            for i in range(nb):
                G = np.zeros((len(w), dim, dim))
                G[:, a, :] = ug[:, i, :]           # grad(phi_i e_a)[r, s] = delta_ra d_s phi_i
                eps[:, a * nb + i] = 0.5 * (G + np.transpose(G, (0, 2, 1)))
        self.visc = 2.0 * np.einsum("q,qIrs,qJrs->IJ", w, eps, eps)
        m1 = np.einsum("q,qi,qj->ij", w, uv, uv)
        self.mass = np.kron(np.eye(dim), m1)
        divphi = np.zeros((len(w), nd))
        for a in range(dim):
            divphi[:, a * nb:(a + 1) * nb] = ug[:, :, a]
        self.div = -np.einsum("q,qp,qJ->pJ", w, pv, divphi)
        self.pmass = np.einsum("q,qp,qr->pr", w, pv, pv)


class System:
    """Assembled, constrained matrices of one mesh level.

    A   velocity block (constrained rows/cols eliminated, unit diagonal)
    B   divergence block (constrained velocity columns and pressure rows zeroed)
    C   pressure-pressure block: 1 on constrained pressure nodes, else 0
    K   full saddle matrix [[A, B^T], [B, C]]
    Mpw eta^{-1}-weighted pressure mass (constrained rows/cols -> identity)
    K_raw, Mu, Mp1   unconstrained saddle matrix, velocity mass, plain pressure mass
    """

    def __init__(self, mesh: Mesh, eta, alpha, need_pressure=True):
        self.mesh = mesh
        self.alpha = alpha
        self.alpha_cells = cell_alpha(mesh, alpha)
        self.eta = np.asarray(eta, dtype=float)
        cm = CellMatrices(mesh.dim, mesh.h)
        self.cm = cm
        act = mesh.active_cells()
        udofs = mesh.cell_udofs()[act]
        nloc = udofs.shape[1]
        e = self.eta[act]
        # velocity block: A_K = alpha * mass + eta_K * visc
        al = self.alpha_cells[act]
        vals = (al[:, None, None] * cm.mass[None] + e[:, None, None] * cm.visc[None]).reshape(len(act), -1)
        rows = np.repeat(udofs, nloc, axis=1)
        cols = np.tile(udofs, (1, nloc))
        A_raw = sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())),
                              shape=(mesh.n_u, mesh.n_u)).tocsr()
        mvals = np.broadcast_to(cm.mass[None], (len(act),) + cm.mass.shape).reshape(len(act), -1)
        self.Mu = sp.coo_matrix((mvals.ravel(), (rows.ravel(), cols.ravel())),
                                shape=(mesh.n_u, mesh.n_u)).tocsr()
        vc = np.tile(mesh.vnode_constrained(), mesh.dim)
        self.u_constrained = vc
        self.A_raw = A_raw
        self.A = _eliminate(A_raw, vc)
        if not need_pressure:
            return
        pdofs = mesh.cell_pnodes()[act]
        npl = pdofs.shape[1]
        bvals = np.broadcast_to(cm.div[None], (len(act),) + cm.div.shape).reshape(len(act), -1)
        brow = np.repeat(pdofs, nloc, axis=1)
        bcol = np.tile(udofs, (1, npl))
        B_raw = sp.coo_matrix((bvals.ravel(), (brow.ravel(), bcol.ravel())),
                              shape=(mesh.Np, mesh.n_u)).tocsr()
        pc = mesh.pnode_constrained()
        self.p_constrained = pc
        prow = np.repeat(pdofs, npl, axis=1)
        pcol = np.tile(pdofs, (1, npl))
        pm = np.broadcast_to(cm.pmass[None], (len(act),) + cm.pmass.shape).reshape(len(act), -1)
        self.Mp1 = sp.coo_matrix((pm.ravel(), (prow.ravel(), pcol.ravel())),
                                 shape=(mesh.Np, mesh.Np)).tocsr()
        pmw = (cm.pmass[None] / e[:, None, None]).reshape(len(act), -1)
        Mpw_raw = sp.coo_matrix((pmw.ravel(), (prow.ravel(), pcol.ravel())),
                                shape=(mesh.Np, mesh.Np)).tocsr()
        self.Mpw = _eliminate(Mpw_raw, pc)
        self.B_raw = B_raw
        keep_u = sp.diags((~vc).astype(float))
        keep_p = sp.diags((~pc).astype(float))
        self.B = (keep_p @ B_raw @ keep_u).tocsr()
        self.B.eliminate_zeros()
        self.C = sp.diags(pc.astype(float)).tocsr()
        self.K = sp.bmat([[self.A, self.B.T], [self.B, self.C]]).tocsr()
        self.K_raw = sp.bmat([[A_raw, B_raw.T], [B_raw, None]]).tocsr()
        self.constrained = np.concatenate([vc, pc])

    def lift_rhs(self, f, g):
        """Right-hand side with Dirichlet data: b = F - K_raw g on free rows, b = g on constrained
        rows, where F = [M_u f_u ; M_p f_p] is the load of the nodal field f."""
        n_u = self.mesh.n_u
        F = np.concatenate([self.Mu @ f[:n_u], self.Mp1 @ f[n_u:]])
        gc = np.where(self.constrained, g, 0.0)
        b = F - self.K_raw @ gc
        return np.where(self.constrained, g, b)


def cell_alpha(mesh: Mesh, alpha):
    """alpha per cell: a scalar broadcast to every cell, or an array of N_c values."""
    a = np.asarray(alpha, dtype=float)
    if a.ndim == 0:
        return np.full(int(np.prod(mesh.n)), float(a))
    assert a.shape == (int(np.prod(mesh.n)),), "alpha: a scalar or one value per cell"
    return a


def _eliminate(M, constrained):
    keep = sp.diags((~constrained).astype(float))
    out = (keep @ M @ keep + sp.diags(constrained.astype(float))).tocsr()
    out.eliminate_zeros()
    return out


def apply_A_rows(mesh: Mesh, eta, alpha, x, rows):
    """Selected rows of y = A x (constrained A), evaluated cell by cell from the reference cell
    matrices without assembling A (used to check full-size launches at sampled outputs)."""
    cm = CellMatrices(mesh.dim, mesh.h)
    vc = mesh.vnode_constrained()
    nb = cm.nb
    al = cell_alpha(mesh, alpha)
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros(len(rows))
    cell_vn = None
    vt = mesh.vnode_tuples()
    for r, row in enumerate(rows):
        comp, node = divmod(int(row), mesh.Nv)
        if vc[node]:
            out[r] = x[row]
            continue
        I = vt[node]
        # cells containing node I: i in {floor((I-1)/2), floor(I/2)} per axis, within range
        cand = []
        for a in range(mesh.dim):
            lo = (I[a] - 1) // 2 if I[a] % 2 == 0 else I[a] // 2
            hi = I[a] // 2
            cand.append(sorted({c for c in (lo, hi) if 0 <= c < mesh.n[a]}))
        acc = 0.0
        for cell in _product(cand):
            cflat = 0
            stride = 1
            for a in range(mesh.dim):
                cflat += cell[a] * stride
                stride *= mesh.n[a]
            if mesh.void[cflat]:
                continue
            loc = np.array([I[a] - 2 * cell[a] for a in range(mesh.dim)])
            li = int(sum(loc[a] * 3 ** a for a in range(mesh.dim)))
            offs = Mesh.local_offsets(mesh.dim, 3)
            gn = mesh.vnode_flat(2 * np.array(cell)[None, :] + offs)
            xl = np.concatenate([np.where(vc[gn], 0.0, x[b * mesh.Nv + gn]) for b in range(mesh.dim)])
            Arow = al[cflat] * cm.mass[comp * nb + li] + eta[cflat] * cm.visc[comp * nb + li]
            acc += Arow @ xl
        out[r] = acc
    return out


def _product(lists):
    if not lists:
        yield ()
        return
    for v in lists[0]:
        for rest in _product(lists[1:]):
            yield (v,) + rest


def mms_weak_rhs(mesh: Mesh, eta, alpha, u_fn, grad_fn, p_fn, npts=5):
    """Load F(v) = alpha (u, v) + sum_K 2 eta_K (eps(u), eps(v))_K - (p, div v) of exact fields
    (2D), integrated cell by cell with an npts-point Gauss rule (no interface deltas needed)."""
    assert mesh.dim == 2
    uv, ug, w = tensor_basis(2, mesh.h, Q2_NODES, npts)
    pts, _ = gauss_rule(npts)
    q_offs = Mesh.local_offsets(2, npts)
    nb = uv.shape[1]
    F = np.zeros(mesh.n_u)
    cells = mesh.cell_index_tuples()
    vn = mesh.cell_vnodes()
    for c in mesh.active_cells():
        x0 = cells[c] * np.array(mesh.h)
        xq = x0[0] + pts[q_offs[:, 0]] * mesh.h[0]
        yq = x0[1] + pts[q_offs[:, 1]] * mesh.h[1]
        ux, uy = u_fn(xq, yq)
        dxx, dxy, dyx, dyy = grad_fn(xq, yq)
        p = p_fn(xq, yq)
        e11, e22, e12 = dxx, dyy, 0.5 * (dxy + dyx)
        for a in range(2):
            uval = ux if a == 0 else uy
            for i in range(nb):
                g = ug[:, i, :]
                # eps(phi_i e_a) : eps(u)
                if a == 0:
                    ee = g[:, 0] * e11 + g[:, 1] * e12
                else:
                    ee = g[:, 0] * e12 + g[:, 1] * e22
                val = np.sum(w * (alpha * uval * uv[:, i] + 2.0 * eta[c] * ee - p * g[:, a]))
                F[a * mesh.Nv + vn[c, i]] += val
    return F
