"""Pins of the oracle's discretisation against facts it does not compute itself.

Each test fails on a plausible mistake in oracle/fem.py or oracle/mesh.py: a wrong
quadrature point or weight, a dropped factor 2 in 2 eta eps:eps, a transposed
grad-transpose term, a wrong sign of B, a misplaced local-node index.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.fem import CellMatrices, System, apply_A_rows, mms_weak_rhs
from oracle.mesh import Mesh
from paper_2305_08986_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    cur = None
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("[") and line.endswith("]"):
            cur = line[1:-1]
            out[cur] = []
        else:
            out[cur].append([float(eval(t)) for t in line.split()])
    return {k: np.array(v) for k, v in out.items()}


def test_dof_counts_closed_form():
    for dim, n in [(2, (16, 16)), (2, (1280, 210)), (3, (64, 64, 64)), (3, (3, 5, 2))]:
        m = Mesh(dim, n, (1.0,) * dim)
        assert m.n_u == dim * int(np.prod([2 * k + 1 for k in n]))
        assert m.Np == int(np.prod([k + 1 for k in n]))
    # the figures quoted for the benchmark meshes
    assert Mesh(2, (16, 16), (1, 1)).n_u == 2178 and Mesh(2, (16, 16), (1, 1)).Np == 289
    assert Mesh(3, (64,) * 3, (1,) * 3).n_u == 6440067
    assert Mesh(2, (1280, 224), (1, 1)).n_u == 2299778


def test_local_numbering():
    m = Mesh(3, (3, 2, 2), (1, 1, 1))
    vn = m.cell_vnodes()
    # cell (1, 1, 0) is cell 1 + 3*1 = 4; its local node (a,b,c) = (2,1,2) is index 2+3+18 = 23
    I = (2 * 1 + 2, 2 * 1 + 1, 2 * 0 + 2)
    assert vn[4, 23] == I[0] + 7 * (I[1] + 5 * I[2])
    pn = m.cell_pnodes()
    assert pn[4, 1 + 2 * 1 + 4 * 1] == (1 + 1) + 4 * ((1 + 1) + 3 * 1)


@pytest.mark.parametrize("h", [1.0, 0.37])
def test_1d_closed_forms(h):
    """Q2 mass h/30 [4 2 -1; 2 16 2; -1 2 4], Q2 stiffness 1/(3h) [7 -8 1; -8 16 -8; 1 -8 7],
    Q1 mass h/6 [2 1; 1 2] (textbook element matrices, tests/golden/element_1d.txt)."""
    g = _read_golden("element_1d.txt")
    cm = CellMatrices(1, (h,))
    np.testing.assert_allclose(cm.mass, h * g["q2_mass_30"] / 30.0, rtol=0, atol=1e-15)
    # in 1D, 2 eps:eps = 2 u' v'
    np.testing.assert_allclose(cm.visc / 2.0, g["q2_stiffness_3"] / (3.0 * h), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(cm.pmass, h * g["q1_mass_6"] / 6.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(cm.div, -g["q1_q2deriv_6"] / 6.0, rtol=1e-14, atol=1e-15)


def _sympy_cell(dim, h, entries):
    """Exact integrals of the definitions over the cell with sympy (independent of Gauss rules)."""
    sym = pytest.importorskip("sympy")
    X = sym.symbols("x0:%d" % dim)
    def lag(nodes, i, t):
        e = sym.Integer(1)
        for j, tj in enumerate(nodes):
            if j != i:
                e *= (t - tj) / (nodes[i] - tj)
        return e
    q2 = [sym.Integer(0), sym.Rational(1, 2), sym.Integer(1)]
    q1 = [sym.Integer(0), sym.Integer(1)]
    hs = [sym.nsimplify(v) for v in h]
    offs3 = Mesh.local_offsets(dim, 3)
    offs2 = Mesh.local_offsets(dim, 2)
    import functools

    @functools.lru_cache(maxsize=None)
    def phi(i):
        return sym.expand(sym.prod([lag(q2, int(offs3[i, a]), X[a] / hs[a]) for a in range(dim)]))

    @functools.lru_cache(maxsize=None)
    def psi(q):
        return sym.expand(sym.prod([lag(q1, int(offs2[q, a]), X[a] / hs[a]) for a in range(dim)]))

    def integ(e):
        poly = sym.Poly(sym.expand(e), *X)
        for a in range(dim):
            poly = sym.Poly(poly.integrate(X[a]).subs(X[a], hs[a]) - poly.integrate(X[a]).subs(X[a], 0), *X)
        return float(poly.as_expr())
    nb = 3 ** dim
    out = {}
    for kind, I, J in entries:
        if kind == "visc":
            a, i = divmod(I, nb)
            b, j = divmod(J, nb)
            # 2 eps(u):eps(v) with u = phi_j e_b, v = phi_i e_a, written as a symmetric-gradient product
            gu = sym.zeros(dim, dim)
            gv = sym.zeros(dim, dim)
            for s in range(dim):
                gu[b, s] = sym.diff(phi(j), X[s])
                gv[a, s] = sym.diff(phi(i), X[s])
            eu = (gu + gu.T) / 2
            ev = (gv + gv.T) / 2
            out[(kind, I, J)] = integ(2 * sum(eu[r, s] * ev[r, s] for r in range(dim) for s in range(dim)))
        elif kind == "mass":
            a, i = divmod(I, nb)
            b, j = divmod(J, nb)
            out[(kind, I, J)] = integ(phi(i) * phi(j)) if a == b else 0.0
        elif kind == "div":
            b, j = divmod(J, nb)
            out[(kind, I, J)] = -integ(psi(I) * sym.diff(phi(j), X[b]))
        elif kind == "pmass":
            out[(kind, I, J)] = integ(psi(I) * psi(J))
    return out


def test_cell_matrices_exact_2d():
    h = (0.5, 0.25)
    cm = CellMatrices(2, h)
    nd = 2 * 9
    entries = [("visc", I, J) for I in range(nd) for J in range(nd)]
    entries += [("mass", I, J) for I in range(0, nd, 3) for J in range(nd)]
    entries += [("div", q, J) for q in range(4) for J in range(nd)]
    entries += [("pmass", q, r) for q in range(4) for r in range(4)]
    ex = _sympy_cell(2, h, entries)
    for (kind, I, J), v in ex.items():
        assert abs(getattr(cm, kind)[I, J] - v) <= 1e-13 * max(1.0, abs(v)), (kind, I, J)


def test_cell_matrices_exact_3d_sample():
    h = (0.5, 0.25, 0.75)
    cm = CellMatrices(3, h)
    rng = np.random.default_rng(3)
    nd = 81
    entries = [("visc", int(I), int(J)) for I, J in rng.integers(0, nd, size=(40, 2))]
    entries += [("visc", 0, 27 + 13), ("visc", 13, 13), ("visc", 54 + 4, 27 + 22)]
    entries += [("div", int(q), int(J)) for q, J in zip(rng.integers(0, 8, 12), rng.integers(0, nd, 12))]
    ex = _sympy_cell(3, h, entries)
    for (kind, I, J), v in ex.items():
        assert abs(getattr(cm, kind)[I, J] - v) <= 1e-13 * max(1.0, abs(v)), (kind, I, J)


@pytest.mark.parametrize("dim", [2, 3])
def test_rigid_body_kernel(dim):
    """With alpha = 0 and no constraints, eps(u_rb) = 0 for rigid motions, so A u_rb = 0."""
    n = (3, 2, 2)[:dim]
    m = Mesh(dim, n, (0.7, 0.4, 0.9)[:dim], dirichlet_faces=0)
    rng = np.random.default_rng(1)
    eta = np.exp(rng.uniform(0, 8, m.Nc))
    s = System(m, eta, 0.0)
    X = m.vnode_tuples() * (np.array(m.h) / 2.0)
    modes = []
    for a in range(dim):
        u = np.zeros(m.n_u)
        u[a * m.Nv:(a + 1) * m.Nv] = 1.0
        modes.append(u)
    for a, b in itertools.combinations(range(dim), 2):
        u = np.zeros(m.n_u)
        u[a * m.Nv:(a + 1) * m.Nv] = -X[:, b]
        u[b * m.Nv:(b + 1) * m.Nv] = X[:, a]
        modes.append(u)
    scale = abs(s.A_raw).sum(axis=1).max()
    for u in modes:
        assert np.abs(s.A_raw @ u).max() <= 1e-12 * scale
    # a non-rigid field is not in the kernel
    u = np.zeros(m.n_u)
    u[:m.Nv] = X[:, 0] ** 2
    assert np.abs(s.A_raw @ u).max() > 1e-6 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_symmetric_positive_definite(dim):
    n = (4, 3, 2)[:dim]
    p = inputs.config_random_field(dim, n, seed=5, contrast=1e6, alpha=3.0)
    m = Mesh(dim, n, p.length, p.void, p.dirichlet_faces)
    s = System(m, p.eta, p.alpha)
    # symmetric up to the summation order of duplicate entries in the assembly
    assert abs(s.A - s.A.T).max() <= 1e-15 * abs(s.A).max()
    assert abs(s.K - s.K.T).max() <= 1e-15 * abs(s.K).max()
    np.linalg.cholesky(s.A.toarray())


@pytest.mark.parametrize("dim", [2, 3])
def test_divergence_invariants(dim):
    n = (4, 3, 2)[:dim]
    m = Mesh(dim, n, (1.0, 0.5, 0.75)[:dim])
    s = System(m, np.ones(m.Nc), 1.0)
    # B^T 1 = 0 on free velocity rows when the whole boundary is Dirichlet
    free_u = ~s.u_constrained
    assert np.abs((s.B_raw.T @ np.ones(m.Np))[free_u]).max() < 1e-14
    # linear u with constant divergence c: (B u)_q = -c int psi_q
    X = m.vnode_tuples() * (np.array(m.h) / 2.0)
    u = np.zeros(m.n_u)
    coef = [1.5, -0.25, 0.5][:dim]
    for a in range(dim):
        u[a * m.Nv:(a + 1) * m.Nv] = coef[a] * X[:, a] + 0.3 * X[:, (a + 1) % dim]
    c = sum(coef)
    np.testing.assert_allclose(s.B_raw @ u, -c * (s.Mp1 @ np.ones(m.Np)), rtol=1e-13, atol=1e-15)


def test_patch_quadratic_weak_form():
    """For quadratic u and linear p (exact in Q2 / Q1), A_raw u_I + B_raw^T p_I equals the weak
    form alpha (u, v) + 2 eta (eps u, eps v) - (p, div v) integrated with a 5-point Gauss rule."""
    m = Mesh(2, (3, 2), (0.9, 0.5), dirichlet_faces=0)
    eta = np.array([1.0, 3.0, 10.0, 0.5, 2.0, 7.0])
    alpha = 2.5
    X = m.vnode_tuples() * (np.array(m.h) / 2.0)
    P = m.pnode_tuples() * np.array(m.h)
    ufn = lambda x, y: (x * x - 0.5 * x * y + 0.2 * y, 0.3 * y * y + x * y - x)
    gfn = lambda x, y: (2 * x - 0.5 * y, -0.5 * x + 0.2, y - 1.0, 0.6 * y + x)
    pfn = lambda x, y: 0.7 * x - 1.1 * y + 0.2
    s = System(m, eta, alpha)
    u = np.concatenate(ufn(X[:, 0], X[:, 1]))
    p = pfn(P[:, 0], P[:, 1])
    lhs = s.A_raw @ u + s.B_raw.T @ p
    rhs = mms_weak_rhs(m, eta, alpha, ufn, gfn, pfn, npts=5)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-13)


def test_apply_rows_matches_assembled():
    p = inputs.config_random_field(3, (3, 2, 3), seed=9, void_fraction=0.2)
    m = Mesh(3, p.n, p.length, p.void, p.dirichlet_faces)
    s = System(m, p.eta, p.alpha, need_pressure=False)
    x = np.random.default_rng(0).standard_normal(m.n_u)
    rows = np.arange(0, m.n_u, 7)
    np.testing.assert_allclose(apply_A_rows(m, p.eta, p.alpha, x, rows), (s.A @ x)[rows],
                               rtol=1e-13, atol=1e-12)


def test_lift_rhs_constrained_values():
    p = inputs.config_random_field(2, (4, 3), seed=2, faces=inputs.FACE_XM | inputs.FACE_YP,
                                   void_fraction=0.15)
    m = Mesh(2, p.n, p.length, p.void, p.dirichlet_faces)
    s = System(m, p.eta, p.alpha)
    b = s.lift_rhs(p.f, p.g)
    np.testing.assert_array_equal(b[s.constrained], p.g[s.constrained])
    # the solution takes the Dirichlet values and satisfies the unconstrained equations
    import scipy.sparse.linalg as spla
    x = spla.spsolve(s.K.tocsc(), b)
    np.testing.assert_allclose(x[s.constrained], p.g[s.constrained], rtol=0, atol=1e-12)
    F = np.concatenate([s.Mu @ p.f[:m.n_u], s.Mp1 @ p.f[m.n_u:]])
    res = (s.K_raw @ x - F)[~s.constrained]
    scale = (abs(s.K_raw) @ np.abs(x) + np.abs(F))[~s.constrained]
    assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(scale)  # normwise backward error


@pytest.mark.slow
def test_mms_convergence_rates():
    """eta = 1: Q2 velocity L2 error O(h^3), Q1 pressure L2 error O(h^2) (Taylor-Hood)."""
    from oracle.fem import Q1_NODES, Q2_NODES, gauss_rule, tensor_basis
    from oracle.krylov import direct_solve, normalize_pressure

    def l2err(m, x):
        uv, _, w = tensor_basis(2, m.h, Q2_NODES, 5)
        pv, _, _ = tensor_basis(2, m.h, Q1_NODES, 5)
        pts, _ = gauss_rule(5)
        qo = Mesh.local_offsets(2, 5)
        cells, vn, pn = m.cell_index_tuples(), m.cell_vnodes(), m.cell_pnodes()
        eu = ep = 0.0
        for c in range(m.Nc):
            x0 = cells[c] * np.array(m.h)
            xq = x0[0] + pts[qo[:, 0]] * m.h[0]
            yq = x0[1] + pts[qo[:, 1]] * m.h[1]
            ux, uy = inputs.mms_velocity(xq, yq)
            p = inputs.mms_pressure(xq, yq)
            eu += np.sum(w * ((ux - uv @ x[vn[c]]) ** 2 + (uy - uv @ x[m.Nv + vn[c]]) ** 2))
            ep += np.sum(w * (p - pv @ x[m.n_u + pn[c]]) ** 2)
        return math.sqrt(eu), math.sqrt(ep)

    errs = []
    for n in (8, 16, 32):
        m = Mesh(2, (n, n), (1.0, 1.0))
        eta = np.ones(m.Nc)
        s = System(m, eta, 1.0)
        F = mms_weak_rhs(m, eta, 1.0, inputs.mms_velocity, inputs.mms_velocity_grad, inputs.mms_pressure)
        b = np.concatenate([F, np.zeros(m.Np)])
        b[s.constrained] = 0.0
        errs.append(l2err(m, normalize_pressure(m, s, direct_solve(s, b))))
    ru = [math.log2(errs[i][0] / errs[i + 1][0]) for i in range(2)]
    rp = [math.log2(errs[i][1] / errs[i + 1][1]) for i in range(2)]
    assert all(2.8 < r < 3.2 for r in ru), ru
    assert all(1.9 < r < 3.6 for r in rp) and rp[-1] < 3.1, rp
