"""Per-row error measure for operator applications (test helper).

A matrix-free operator computes y_i = sum_K (A_K x_K)_i cell by cell.  In floating point the
error of row i is bounded by a small multiple of the unit roundoff times

    s_i = sum_K (|A_K| |x_K|)_i        (the cellwise absolute sum),

so the check  max_i |y_i - y_ref,i| / s_i <= tol  holds every row to its own magnitude.  A
norm-wise check cannot do that at a viscosity contrast of 1e6: the rows of fluid cells are
about 1e-6 of the rows of stiff cells, so a 1e-7 relative error confined to fluid rows (for
instance an FP32 rounding of eta leaking into an FP64 path) moves the norm by ~1e-13.

The cellwise absolute matrices are assembled from the oracle's reference cell matrices with the
entries' absolute values; constrained rows are identity rows (s_i = |x_i|) and constrained columns
are dropped, exactly as the constrained operators treat them.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from oracle.fem import CellMatrices, cell_alpha
from oracle.mesh import Mesh


def _assemble(vals, rows, cols, shape):
    return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=shape).tocsr()


class AbsOperators:
    """Cellwise absolute operators |A|_c, |B|_c and the saddle |K|_c of one mesh level, constrained
    like oracle.fem.System (identity rows, zero columns at constrained entries)."""

    def __init__(self, mesh: Mesh, eta, alpha):
        self.mesh = mesh
        cm = CellMatrices(mesh.dim, mesh.h)
        act = mesh.active_cells()
        udofs = mesh.cell_udofs()[act]
        nloc = udofs.shape[1]
        e = np.asarray(eta, dtype=float)[act]
        al = cell_alpha(mesh, alpha)[act]
        vals = np.abs(al[:, None, None] * cm.mass[None] + e[:, None, None] * cm.visc[None])
        rows = np.repeat(udofs, nloc, axis=1)
        cols = np.tile(udofs, (1, nloc))
        A_raw = _assemble(vals.reshape(len(act), -1), rows, cols, (mesh.n_u, mesh.n_u))
        vc = np.tile(mesh.vnode_constrained(), mesh.dim)
        self.u_constrained = vc
        self.A_raw = A_raw
        self.A = self._eliminate(A_raw, vc)
        pdofs = mesh.cell_pnodes()[act]
        npl = pdofs.shape[1]
        bvals = np.broadcast_to(np.abs(cm.div)[None], (len(act),) + cm.div.shape).reshape(len(act), -1)
        B_raw = _assemble(bvals, np.repeat(pdofs, nloc, axis=1), np.tile(udofs, (1, npl)), (mesh.Np, mesh.n_u))
        pc = mesh.pnode_constrained()
        keep_u = sp.diags((~vc).astype(float))
        keep_p = sp.diags((~pc).astype(float))
        self.B = (keep_p @ B_raw @ keep_u).tocsr()
        self.K = sp.bmat([[self.A, self.B.T], [self.B, sp.diags(pc.astype(float))]]).tocsr()

    @staticmethod
    def _eliminate(M, constrained):
        keep = sp.diags((~constrained).astype(float))
        return (keep @ M @ keep + sp.diags(constrained.astype(float))).tocsr()


def row_error(y, y_ref, S_abs, x):
    """max_i |y_i - y_ref,i| / (S_abs |x|)_i over all rows; a row whose scale is 0 must match
    exactly (returns inf otherwise)."""
    y = np.asarray(y, dtype=float)
    y_ref = np.asarray(y_ref, dtype=float)
    s = S_abs @ np.abs(np.asarray(x, dtype=float))
    err = np.abs(y - y_ref)
    zero = s == 0.0
    if np.any(err[zero] != 0.0):
        return float("inf")
    if np.all(zero):
        return 0.0
    return float(np.max(err[~zero] / s[~zero]))


def abs_rows(mesh: Mesh, eta, alpha, x, rows):
    """Selected rows of s = sum_K |A_K| |x_K| (constrained velocity block) without assembling it:
    the scale of row_error at sampled outputs of a full-size launch."""
    cm = CellMatrices(mesh.dim, mesh.h)
    vc = mesh.vnode_constrained()
    nb = cm.nb
    al = cell_alpha(mesh, alpha)
    eta = np.asarray(eta, dtype=float)
    vt = mesh.vnode_tuples()
    offs = Mesh.local_offsets(mesh.dim, 3)
    out = np.zeros(len(rows))
    for r, row in enumerate(np.asarray(rows, dtype=np.int64)):
        comp, node = divmod(int(row), mesh.Nv)
        if vc[node]:
            out[r] = abs(x[row])
            continue
        I = vt[node]
        cand = []
        for a in range(mesh.dim):
            lo = (I[a] - 1) // 2 if I[a] % 2 == 0 else I[a] // 2
            cand.append(sorted({c for c in (lo, I[a] // 2) if 0 <= c < mesh.n[a]}))
        acc = 0.0
        for cell in np.array(np.meshgrid(*cand, indexing="ij")).reshape(mesh.dim, -1).T:
            cflat = int(sum(int(cell[a]) * int(np.prod(mesh.n[:a])) for a in range(mesh.dim)))
            if mesh.void[cflat]:
                continue
            li = int(sum((I[a] - 2 * int(cell[a])) * 3 ** a for a in range(mesh.dim)))
            gn = mesh.vnode_flat(2 * np.array(cell)[None, :] + offs)
            xl = np.concatenate([np.where(vc[gn], 0.0, np.abs(x[b * mesh.Nv + gn])) for b in range(mesh.dim)])
            acc += np.abs(al[cflat] * cm.mass[comp * nb + li] + eta[cflat] * cm.visc[comp * nb + li]) @ xl
        out[r] = acc
    return out


def sampled_row_error(y_rows, ref_rows, scale_rows):
    err = np.abs(np.asarray(y_rows) - np.asarray(ref_rows))
    s = np.asarray(scale_rows)
    zero = s == 0.0
    if np.any(err[zero] != 0.0):
        return float("inf")
    return float(np.max(err[~zero] / s[~zero])) if np.any(~zero) else 0.0
