"""Pins of the oracle's corrector-mode momentum block (oracle/corrector.py): convection
rho ((v° . grad) v, w) and the streamline diffusion of Eq. "a_stab", checked against the
predictor system, the Kronecker closed form of the 1D Q2 matrices, skew-symmetry for a
divergence-free field, the Brooks-Hughes parameter, and the sparse direct solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.corrector import CorrectorOracle, CorrectorSystem, cell_parameters, convection_matrices, xi
from oracle.fem import System
from oracle.mesh import Mesh, mesh_from_problem
from paper_2305_08986_gb300 import inputs

# 1D Q2 matrices on [0, 1] (exact rationals): Mi / 30 = int phi_i phi_j, Ei / 6 = int phi_i' phi_j
MI = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0
EI = np.array([[-3, -4, 1], [4, 0, -4], [-1, 4, 3]]) / 6.0


def _field(m, fx, fy):
    X = m.vnode_tuples() * (np.array(m.h) / 2.0)
    return np.concatenate([fx(X[:, 0], X[:, 1]), fy(X[:, 0], X[:, 1])])


def test_zero_field_gives_the_predictor_system():
    p = inputs.config_random_field(2, (6, 4), seed=3, contrast=1e2, alpha=5.0, void_fraction=0.1)
    m = mesh_from_problem(p)
    cs = CorrectorSystem(m, p.eta, p.alpha, np.zeros(m.n_u), rho=1e3)
    assert abs(cs.K - System(m, p.eta, p.alpha).K).max() == 0.0


def test_constant_field_cell_matrix_is_the_kronecker_closed_form():
    """For v° = (a, b) constant: int_K phi_i (a d_x + b d_y) phi_j = a (Mi hy/30 (x) Ei^T/6) + b
    (Ei^T/6 (x) Mi hx/30) (x fastest: the y factor is the outer Kronecker factor)."""
    m = Mesh(2, (1, 1), (0.7, 0.3), dirichlet_faces=0)
    a, b, rho = 0.8, -1.3, 2.5
    v = np.concatenate([np.full(m.Nv, a), np.full(m.Nv, b)])
    C, S = convection_matrices(m, v, np.ones(1), rho)
    hx, hy = m.h
    ref = rho * (a * np.kron(hy * MI, EI.T) + b * np.kron(EI.T, hx * MI))
    np.testing.assert_allclose(C.toarray()[:9, :9], ref, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(C.toarray()[9:, 9:], ref, rtol=1e-13, atol=1e-15)
    assert abs(C.toarray()[:9, 9:]).max() == 0.0      # componentwise: no coupling of components


def test_divergence_free_field_gives_a_skew_symmetric_free_block():
    """div v° = 0 and every face Dirichlet: int phi_i v°.grad phi_j + int phi_j v°.grad phi_i =
    int v°.grad(phi_i phi_j) = 0 for free i, j (exact 3-point quadrature for a linear v°)."""
    m = Mesh(2, (6, 5), (1.0, 0.8))
    v = _field(m, lambda x, y: x - 0.4, lambda x, y: -(y - 0.3))
    C, _ = convection_matrices(m, v, np.ones(30), 1.0)
    free = np.tile(~m.vnode_constrained(), 2)
    Cf = C.toarray()[np.ix_(free, free)]
    assert np.abs(Cf + Cf.T).max() <= 1e-14 * np.abs(Cf).max()
    assert np.abs(Cf).max() > 0.0


def test_streamline_term_and_parameter():
    assert xi(1.0) == pytest.approx(1.0 / np.tanh(1.0) - 1.0)
    assert xi(50.0) == pytest.approx(1.0 - 1.0 / 50.0, rel=1e-12)
    assert np.all(np.diff(xi(np.linspace(0.5, 20, 40))) > 0)
    m = Mesh(2, (8, 4), (2.0, 1.0))
    eta = np.full(32, 1e-2)
    v = _field(m, lambda x, y: 1.0 + 0.5 * y, lambda x, y: 0.2 * x)
    rho = 10.0
    vn, pe, r = cell_parameters(m, v, eta, rho)
    hK = np.hypot(*m.h)
    big = pe >= 1.0
    assert big.all()
    np.testing.assert_allclose(r, hK / (2 * vn * 2) * (1 / np.tanh(pe) - 1 / pe), rtol=1e-14)
    _, S = convection_matrices(m, v, eta, rho)
    Sd = S.toarray()
    assert np.abs(Sd - Sd.T).max() <= 1e-14 * np.abs(Sd).max()
    assert np.linalg.eigvalsh(Sd).min() >= -1e-12 * np.abs(Sd).max()
    # below Pe = 1 the streamline term vanishes
    _, S0 = convection_matrices(m, 1e-6 * v, eta, rho)
    assert abs(S0).max() == 0.0


def test_corrector_solve_reaches_the_direct_solution():
    """Channel with the predictor solution as v° (rho = 1e3 on alpha = 1e3): non-symmetric K_c."""
    from oracle.krylov import StokesOracle
    p = inputs.config_channel(nx=160, ny=28, levels=3)
    m = mesh_from_problem(p)
    pred = StokesOracle(m, p.eta, p.alpha, 3)
    b0 = pred.sys.lift_rhs(p.f, p.g)
    x0, _, _, _ = pred.solve(b0, tol=1e-10)
    vcirc = x0[:m.n_u]
    o = CorrectorOracle(m, p.eta, p.alpha, vcirc, rho=1.0, levels=3)
    K = o.sys.K
    assert abs(K - K.T).max() > 0.0                     # convection makes the block non-symmetric
    b = o.sys.lift_rhs(p.f, p.g)
    x, it, rel, _ = o.solve(b, tol=1e-10)
    xd = spla.spsolve(K.tocsc(), b)
    assert rel <= 1e-10 and it < 80, (it, rel)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)


def test_bicgstab_facts():
    """S = c I is solved in one step; n_S steps converge on a non-symmetric, diagonally dominant
    system; a positive scaling of the preconditioner leaves every iterate unchanged."""
    from oracle.monolithic import bicgstab
    rng = np.random.default_rng(8)
    n = 10
    b = rng.standard_normal(n)
    np.testing.assert_allclose(bicgstab(lambda z: 3.5 * z, lambda r: r, b, 1), b / 3.5, rtol=1e-14)
    S = rng.standard_normal((n, n)) + 6.0 * np.eye(n)
    d = rng.uniform(0.5, 2.0, n)
    x = bicgstab(lambda z: S @ z, lambda r: d * r, b, 3 * n)
    np.testing.assert_allclose(S @ x, b, rtol=0, atol=1e-10 * np.abs(b).max())
    for k in (1, 2, 4):
        np.testing.assert_allclose(bicgstab(lambda z: S @ z, lambda r: 9.0 * d * r, b, k),
                                   bicgstab(lambda z: S @ z, lambda r: d * r, b, k), rtol=1e-12, atol=1e-14)


def test_corrector_with_the_monolithic_preconditioner():
    """Sec. 4's saddle-point multigrid on the corrector block (ChebBiCGStab Schur solves): FGMRES
    reaches the sparse direct solution of the non-symmetric system."""
    from oracle.krylov import StokesOracle, fgmres
    from oracle.monolithic import MonolithicHierarchy
    p = inputs.config_box_inclusion(2, (32, 16), 3, 1e4, 30.0, seed=7,
                                    faces=inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP, align_coarse=True)
    m = mesh_from_problem(p)
    pred = StokesOracle(m, p.eta, p.alpha, 3)
    x0, _, _, _ = pred.solve(pred.sys.lift_rhs(p.f, p.g), tol=1e-8)
    vcirc = 5.0 * x0[:m.n_u] / np.abs(x0[:m.n_u]).max()       # a field of size 5
    rho = 40.0                                                 # Pe_K up to ~4: streamline term on ~120 cells
    _, pe, _ = cell_parameters(m, vcirc, p.eta, rho)
    assert (pe >= 1.0).any()                                   # the streamline term is active somewhere
    cs = CorrectorSystem(m, p.eta, p.alpha, vcirc, rho)
    mono = MonolithicHierarchy(m, p.eta, p.alpha, 3, corrector=(vcirc, rho))

    def precond(r):
        z = mono.apply(r)
        z[cs.constrained] = r[cs.constrained]
        return z

    b = cs.lift_rhs(p.f, p.g)
    x, it, rel, _ = fgmres(lambda v: cs.K @ v, precond, b, tol=1e-10, max_iter=300)
    xd = spla.spsolve(cs.K.tocsc(), b)
    assert rel <= 1e-10 and it < 40, (it, rel)
    n_u = m.n_u
    assert np.linalg.norm(x[:n_u] - xd[:n_u]) <= 1e-6 * np.linalg.norm(xd[:n_u])


def test_constant_field_cell_matrix_3d():
    """3D: int_K phi_i (v° . grad) phi_j = sum_a v°_a (Ei^T/6 in direction a, h Mi/30 elsewhere),
    Kronecker factors ordered z (outer), y, x (inner)."""
    m = Mesh(3, (1, 1, 1), (0.7, 0.3, 0.5), dirichlet_faces=0)
    vv = (0.8, -1.3, 0.4)
    v = np.concatenate([np.full(m.Nv, c) for c in vv])
    C, _ = convection_matrices(m, v, np.ones(1), 1.0)
    h = m.h
    fac = lambda a, ax: EI.T if a == ax else h[ax] * MI
    ref = sum(vv[a] * np.kron(fac(a, 2), np.kron(fac(a, 1), fac(a, 0))) for a in range(3))
    for comp in range(3):
        blk = C.toarray()[27 * comp:27 * (comp + 1), 27 * comp:27 * (comp + 1)]
        np.testing.assert_allclose(blk, ref, rtol=1e-13, atol=1e-15)
