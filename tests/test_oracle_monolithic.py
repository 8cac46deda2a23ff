"""Pins of the oracle's monolithic multigrid (oracle/monolithic.py), the preconditioner of Sec. 4:
saddle-point V-cycle with the block smoother K_j of Eq. "smoother" and ChebMINRES Schur solves.
Each pin checks the oracle against an independent fact (a dense inverse, a closed form, a
textbook property of MINRES, a dense triple product, convergence to the direct solution)."""
import numpy as np
import pytest

from oracle.krylov import StokesOracle, direct_solve, normalize_pressure
from oracle.mesh import Mesh, mesh_from_problem
from oracle.monolithic import MonolithicHierarchy, minres
from paper_2305_08986_gb300 import inputs


def _hier(p, **kw):
    m = mesh_from_problem(p)
    return m, MonolithicHierarchy(m, p.eta, p.alpha, p.levels, **kw)


def _dense_op(f, n):
    return np.column_stack([f(e) for e in np.eye(n)])


def test_minres_one_step_is_the_preconditioned_minimiser():
    """One MINRES step from zero is x = a P b with a minimising (b - a S P b)^T P (b - a S P b):
    a = (u^T S u) / ((S u)^T P (S u)), u = P b.  Scaling P leaves the iterate unchanged."""
    rng = np.random.default_rng(4)
    n = 9
    Q = rng.standard_normal((n, n))
    S = Q @ Q.T + n * np.eye(n)
    d = rng.uniform(0.5, 2.0, n)
    b = rng.standard_normal(n)
    u = d * b
    Su = S @ u
    a = (u @ Su) / (Su @ (d * Su))
    x1 = minres(lambda z: S @ z, lambda r: d * r, b, 1)
    np.testing.assert_allclose(x1, a * u, rtol=1e-13, atol=1e-15)
    x1s = minres(lambda z: S @ z, lambda r: 7.25 * d * r, b, 1)
    np.testing.assert_allclose(x1s, x1, rtol=1e-13, atol=1e-15)
    # the minimiser: perturbing a in either direction increases the P-norm of the residual
    def pnorm(t):
        r = b - t * Su
        return r @ (d * r)
    assert pnorm(a) < pnorm(a * (1 + 1e-3)) and pnorm(a) < pnorm(a * (1 - 1e-3))


def test_minres_n_steps_solve_n_by_n():
    """In exact arithmetic MINRES terminates within n steps; its residual norm never grows."""
    rng = np.random.default_rng(5)
    n = 12
    Q = rng.standard_normal((n, n))
    S = Q @ Q.T + 0.5 * np.eye(n)
    d = rng.uniform(0.2, 3.0, n)
    b = rng.standard_normal(n)
    xs = [minres(lambda z: S @ z, lambda r: d * r, b, k) for k in range(1, n + 1)]
    res = [np.sqrt((b - S @ x) @ (d * (b - S @ x))) for x in xs]
    assert all(res[k + 1] <= res[k] * (1 + 1e-10) for k in range(n - 1))
    np.testing.assert_allclose(xs[-1], np.linalg.solve(S, b), rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_schur_diagonal_is_the_dense_triple_product(dim):
    """diag(B diag(A)^{-1} B^T), computed by the oracle from the sparse matrices, against the
    dense product on a mesh with obstacle cells (constrained pressure rows give zero)."""
    n = (6, 4) if dim == 2 else (4, 2, 2)
    p = inputs.config_random_field(dim, n, levels=2, seed=7, contrast=1e3, alpha=5.0, void_fraction=0.15)
    m, h = _hier(p)
    for lv in h.levels:
        B = lv.B.toarray()
        D = lv.sys.A.diagonal()
        ref = np.diag(B @ np.diag(1.0 / D) @ B.T)
        np.testing.assert_allclose(lv.ds, ref, rtol=1e-13, atol=1e-300)
        pc = lv.sys.p_constrained
        assert np.all(lv.ds[~pc] > 0.0) and np.all(lv.ds[pc] == 0.0)
        assert np.all(lv.dsinv[pc] == 0.0)


def test_block_smoother_inverts_the_matrix_of_the_smoother_equation():
    """With Shat^{-1} an exact inverse of a fixed SPD Shat, K_j r equals the solution of
    [Ahat B^T; B B Ahat^{-1} B^T - Shat] w = r with Ahat = (Cheb(A, diag A, k_A))^{-1} formed
    densely: a sign, order or transposition error in the factorisation fails this."""
    p = inputs.config_random_field(2, (4, 4), levels=2, seed=11, contrast=1e2, alpha=3.0)
    m, h = _hier(p)
    lv = h.levels[1]
    n_u, n_p = lv.n_u, lv.mesh.Np
    Ahat_inv = _dense_op(lambda e: h.ahat_inv(1, e), n_u)
    Ahat = np.linalg.inv(Ahat_inv)
    B = lv.B.toarray()
    rng = np.random.default_rng(2)
    Q = rng.standard_normal((n_p, n_p))
    Shat = Q @ Q.T / n_p + np.eye(n_p)
    Kblk = np.block([[Ahat, B.T], [B, B @ Ahat_inv @ B.T - Shat]])
    r = rng.standard_normal(n_u + n_p)
    w = h.smoother(1, r, schur=lambda v: np.linalg.solve(Shat, v))
    np.testing.assert_allclose(w, np.linalg.solve(Kblk, r), rtol=1e-9, atol=1e-9 * np.abs(w).max())


@pytest.mark.parametrize("faces", [None, inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP])
def test_coarse_solve_satisfies_the_coarse_system(faces):
    p = inputs.config_random_field(2, (8, 8), levels=2, seed=13, contrast=1e4, alpha=10.0, faces=faces)
    m, h = _hier(p)
    c0 = h.levels[0]
    K = c0.K.toarray()
    free = ~c0.sys.constrained
    rng = np.random.default_rng(3)
    b = rng.standard_normal(c0.mesh.N)
    b[~free] = 0.0
    if h.nullspace:
        pf = free[c0.n_u:]
        b[c0.n_u:][pf] -= b[c0.n_u:][pf].mean()   # consistent: orthogonal to the constant pressure
    x = h.coarse_solve(b)
    np.testing.assert_allclose((K @ x)[free], b[free], rtol=0, atol=1e-10 * np.abs(b).max())
    assert np.all(x[~free] == 0.0)
    if h.nullspace:
        assert abs(x[c0.n_u:][free[c0.n_u:]].sum()) <= 1e-10 * np.abs(x).max()


def test_one_level_is_an_exact_preconditioner():
    p = inputs.config_random_field(2, (4, 4), levels=1, seed=17, contrast=1e3, alpha=2.0,
                                   faces=inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP)
    m = mesh_from_problem(p)
    o = StokesOracle(m, p.eta, p.alpha, 1, precond="monolithic")
    b = o.sys.lift_rhs(p.f, p.g)
    x, it, rel, _ = o.solve(b, tol=1e-10)
    assert it == 1 and rel <= 1e-10


@pytest.mark.parametrize("dim,n", [(2, (8, 6)), (3, (4, 4, 2))])
def test_vcycle_without_smoothing_is_the_coarse_grid_correction(dim, n):
    """With m = 0 a two-level cycle is P M_0'^{-1} P^T b, P = diag(P_u, P_p), formed densely."""
    p = inputs.config_random_field(dim, n, levels=2, seed=29, contrast=1e2, alpha=4.0,
                                   faces=inputs.FACE_XM | inputs.FACE_YM)
    m, h = _hier(p, smooth=0)
    fl, c0 = h.levels[1], h.levels[0]
    P = np.block([[fl.Pu.toarray(), np.zeros((fl.n_u, c0.mesh.Np))],
                  [np.zeros((fl.mesh.Np, c0.n_u)), fl.Pp.toarray()]])
    free = ~c0.sys.constrained
    Minv = np.zeros((c0.mesh.N, c0.mesh.N))
    Minv[np.ix_(free, free)] = np.linalg.inv(c0.K.toarray()[np.ix_(free, free)])
    b = np.random.default_rng(6).standard_normal(fl.mesh.N)
    np.testing.assert_allclose(h.vcycle(b), P @ (Minv @ (P.T @ b)), rtol=1e-10, atol=1e-12)


def test_monolithic_beats_block_triangular_on_a_resolved_inclusion():
    """Sec. 4's premise: on an inclusion the coarse mesh resolves (contrast 1e6), the saddle-point
    multigrid needs fewer FGMRES iterations than the block-triangular variant."""
    p = inputs.config_box_inclusion(2, (32, 32), 3, 1e6, 30.0, seed=5, align_coarse=True)
    m = mesh_from_problem(p)
    its = {}
    for kind in ("block", "monolithic"):
        o = StokesOracle(m, p.eta, p.alpha, 3, precond=kind)
        b = o.sys.lift_rhs(p.f, p.g)
        free = ~o.sys.p_constrained
        b[m.n_u:][free] -= b[m.n_u:][free].mean()
        _, its[kind], rel, _ = o.solve(b, tol=1e-9)
        assert rel <= 1e-9
    assert its["monolithic"] < its["block"], its


def _problem(case):
    kind, dim, n, levels, contrast, faces = case
    if kind == "box":
        return inputs.config_box_inclusion(dim, n, levels, contrast, 30.0, seed=5, faces=faces, align_coarse=True)
    return inputs.config_random_field(dim, n, levels=levels, seed=23, contrast=contrast, alpha=30.0, faces=faces,
                                      void_fraction=0.05)


F3 = inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP


@pytest.mark.parametrize("case,tol", [
    (("box", 2, (32, 16), 3, 1e6, F3), 1e-10), (("rf", 2, (8, 8), 2, 1e3, F3), 1e-11),
    (("rf", 2, (8, 8), 2, 1e3, None), 1e-11), (("box", 3, (8, 8, 8), 2, 1e6, None), 1e-10)])
def test_fgmres_with_the_monolithic_preconditioner_reaches_the_direct_solution(case, tol):
    p = _problem(case)
    m = mesh_from_problem(p)
    o = StokesOracle(m, p.eta, p.alpha, p.levels, precond="monolithic")
    b = o.sys.lift_rhs(p.f, p.g)
    if m.has_pressure_nullspace():
        free = ~o.sys.p_constrained
        b[m.n_u:][free] -= b[m.n_u:][free].mean()   # consistent right-hand side
    x, it, rel, _ = o.solve(b, tol=tol, max_iter=200)
    assert rel <= tol and it < 60
    xd = normalize_pressure(m, o.sys, direct_solve(o.sys, b))
    x = normalize_pressure(m, o.sys, x)
    n_u = m.n_u
    assert np.linalg.norm(x[:n_u] - xd[:n_u]) <= 1e-6 * np.linalg.norm(xd[:n_u])
    # the pressure inside an eta = 1e6 inclusion is a Schur-complement mode of eigenvalue ~1/eta:
    # a residual of 1e-10 pins it only to ~1e-3 (the direct solve has the same sensitivity)
    ptol = 1e-2 if case[4] >= 1e5 else 1e-6
    assert np.linalg.norm(x[n_u:] - xd[n_u:]) <= ptol * np.linalg.norm(xd[n_u:])
