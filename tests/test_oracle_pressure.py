"""Pins of the oracle's pressure-Laplacian multigrid (oracle/pressure.py)."""
import numpy as np
import pytest

from oracle.krylov import StokesOracle
from oracle.mesh import Mesh, mesh_from_problem
from oracle.pressure import (PressureHierarchy, pressure_laplacian, q1_prolongation, q1_stiffness_cell)
from paper_2305_08986_gb300 import inputs
from tests.test_oracle_fem import _read_golden


@pytest.mark.parametrize("h", [1.0, 0.3])
def test_q1_stiffness_1d_closed_form(h):
    g = _read_golden("element_1d.txt")
    np.testing.assert_allclose(q1_stiffness_cell(1, (h,)), g["q1_stiffness_1"] / h, rtol=1e-14)


def test_q1_stiffness_2d_exact():
    """int grad psi_q . grad psi_r on [0,hx] x [0,hy], exact (sympy), against the quadrature."""
    sym = pytest.importorskip("sympy")
    hx, hy = sym.Rational(1, 2), sym.Rational(1, 5)
    x, y = sym.symbols("x y")
    psi = [(1 - x / hx) * (1 - y / hy), x / hx * (1 - y / hy), (1 - x / hx) * y / hy, x / hx * y / hy]
    K = q1_stiffness_cell(2, (0.5, 0.2))
    for i in range(4):
        for j in range(4):
            e = sym.diff(psi[i], x) * sym.diff(psi[j], x) + sym.diff(psi[i], y) * sym.diff(psi[j], y)
            v = float(sym.integrate(sym.integrate(sym.expand(e), (x, 0, hx)), (y, 0, hy)))
            assert abs(K[i, j] - v) <= 1e-14 * max(1.0, abs(v))


def test_pure_neumann_kernel_and_mixed_spd():
    m = Mesh(2, (5, 4), (1.0, 0.8))                       # every velocity face Dirichlet
    K, c = pressure_laplacian(m)
    assert not c.any()
    assert np.abs(K @ np.ones(m.Np)).max() < 1e-13
    m2 = Mesh(2, (5, 4), (1.0, 0.8), dirichlet_faces=inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP)
    K2, c2 = pressure_laplacian(m2)
    assert c2.sum() == 5                                  # the outflow column x = L
    np.linalg.cholesky(K2.toarray())


@pytest.mark.parametrize("dim", [2, 3])
def test_q1_prolongation_reproduces_bilinear(dim):
    cm = Mesh(dim, (2, 3, 2)[:dim], (1.0, 0.6, 0.8)[:dim])
    fm = Mesh(dim, tuple(2 * k for k in cm.n), cm.length)
    P = q1_prolongation(cm, fm, np.zeros(cm.Np, bool), np.zeros(fm.Np, bool))
    def field(m):
        X = m.pnode_tuples() * np.array(m.h)
        f = 1.0 + 2.0 * X[:, 0] - 0.5 * X[:, 1] + 3.0 * X[:, 0] * X[:, 1]
        if dim == 3:
            f = f + X[:, 2] * (1.0 - X[:, 0])
        return f
    np.testing.assert_allclose(P @ field(cm), field(fm), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("faces", [None, inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP])
def test_pressure_vcycle_symmetric_contracting(faces):
    m = Mesh(2, (16, 8), (1.0, 0.5), dirichlet_faces=faces)
    H = PressureHierarchy(m, 3)
    K = H.levels[-1]["K"].toarray()
    c = H.levels[-1]["c"]
    idx = np.nonzero(~c)[0]
    V = np.stack([H.vcycle(np.eye(m.Np)[i]) for i in idx], axis=1)[idx]
    assert np.abs(V - V.T).max() <= 1e-10 * np.abs(V).max()
    E = np.eye(len(idx)) - V @ K[np.ix_(idx, idx)]
    ev = np.abs(np.linalg.eigvals(E))
    if faces is None:   # the constant is in the kernel of K: E keeps it (eigenvalue 1)
        ev = np.sort(ev)[:-1]
    assert ev.max() < 0.2


def test_cahouet_chabard_is_robust_in_alpha():
    """alpha = 1e3 channel: the Cahouet-Chabard term keeps FGMRES in the tens of iterations
    (the pressure mass alone needs several hundred on the same problem)."""
    p = inputs.config_channel(nx=160, ny=28, levels=3)
    m = mesh_from_problem(p)
    o = StokesOracle(m, p.eta, p.alpha, p.levels, schur="cc")
    b = o.sys.lift_rhs(p.f, p.g)
    x, it, rel, _ = o.solve(b, tol=1e-8)
    assert rel <= 1e-8 and it < 50, it
