"""Pins of the oracle's FGMRES and full solve (oracle/krylov.py) by brute force and closed forms."""
import numpy as np
import pytest

from oracle.fem import System
from oracle.krylov import StokesOracle, direct_solve, fgmres, normalize_pressure
from oracle.mesh import Mesh
from paper_2305_08986_gb300 import inputs


def _dense_solution(s, b):
    """Dense least-squares solution of K x = b with the free pressure mean fixed by bordering."""
    K = s.K.toarray()
    m = s.mesh
    if m.has_pressure_nullspace():
        e = np.zeros(m.N)
        e[m.n_u:][~s.p_constrained] = 1.0
        Kb = np.block([[K, e[:, None]], [e[None, :], np.zeros((1, 1))]])
        return np.linalg.solve(Kb, np.concatenate([b, [0.0]]))[:-1]
    return np.linalg.solve(K, b)


@pytest.mark.parametrize("dim,n,levels,faces", [
    (2, (4, 4), 2, None), (2, (4, 2), 2, inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP),
    (3, (2, 2, 2), 2, None)])
def test_fgmres_matches_dense_solve(dim, n, levels, faces):
    p = inputs.config_random_field(dim, n, levels=levels, seed=3, contrast=1e4, alpha=10.0, faces=faces)
    m = Mesh(dim, p.n, p.length, p.void, p.dirichlet_faces)
    o = StokesOracle(m, p.eta, p.alpha, levels)
    b = o.sys.lift_rhs(p.f, p.g)
    if m.has_pressure_nullspace():
        free = ~o.sys.p_constrained
        b[m.n_u:][free] -= b[m.n_u:][free].mean()   # consistent right-hand side
    x, it, rel, _ = o.solve(b, tol=1e-13)
    xd = _dense_solution(o.sys, b)
    x = normalize_pressure(m, o.sys, x)
    xd = normalize_pressure(m, o.sys, xd)
    assert rel <= 1e-13
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_exact_preconditioner_one_iteration():
    p = inputs.config_random_field(2, (3, 3), seed=1, faces=inputs.FACE_XM | inputs.FACE_YM)
    m = Mesh(2, p.n, p.length, p.void, p.dirichlet_faces)
    s = System(m, p.eta, p.alpha)
    K = s.K.toarray()
    Kinv = np.linalg.inv(K)
    b = s.lift_rhs(p.f, p.g)
    x, it, rel, _ = fgmres(lambda v: K @ v, lambda v: Kinv @ v, b, tol=1e-10)
    assert it == 1 and rel <= 1e-10


def test_unpreconditioned_converges_within_dimension():
    p = inputs.config_random_field(2, (2, 2), seed=2, contrast=10.0,
                                   faces=inputs.FACE_XM | inputs.FACE_YM)
    m = Mesh(2, p.n, p.length, p.void, p.dirichlet_faces)
    s = System(m, p.eta, p.alpha)
    b = s.lift_rhs(p.f, p.g)
    nfree = int((~s.constrained).sum())
    x, it, rel, _ = fgmres(lambda v: s.K @ v, lambda v: v, b, tol=1e-10, restart=m.N, max_iter=m.N)
    # K is block diagonal [K_free, I]: the Krylov space has at most nfree + 1 dimensions
    # (one more step of slack for rounding)
    assert rel <= 1e-10 and it <= nfree + 2


def test_gmres_residual_history_monotone():
    p = inputs.config_disc(n=8, levels=2)
    m = Mesh(p.dim, p.n, p.length, p.void, p.dirichlet_faces)
    o = StokesOracle(m, p.eta, p.alpha, p.levels)
    b = o.sys.lift_rhs(p.f, p.g)
    x, it, rel, hist = o.solve(b, tol=1e-10)
    assert rel <= 1e-10
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))


def test_config1_solution_matches_direct():
    p = inputs.config_disc()
    m = Mesh(p.dim, p.n, p.length, p.void, p.dirichlet_faces)
    o = StokesOracle(m, p.eta, p.alpha, p.levels)
    b = o.sys.lift_rhs(p.f, p.g)
    x, it, rel, _ = o.solve(b, tol=1e-11)   # the attainable residual floor is about 3e-12 here
    xd = normalize_pressure(m, o.sys, direct_solve(o.sys, b))
    assert rel <= 1e-11
    assert np.linalg.norm(normalize_pressure(m, o.sys, x) - xd) <= 1e-8 * np.linalg.norm(xd)
    assert it < 60
