"""Pins of the oracle's mesh-extension solve (oracle/extension.py): CG preconditioned by the velocity
multigrid for Eq. "extenstion", checked against textbook CG facts, the sparse direct solution and
the exact reproduction of rigid motions."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.extension import ExtensionOracle, pcg
from oracle.mesh import mesh_from_problem
from paper_2305_08986_gb300 import inputs


def test_pcg_exact_preconditioner_one_step():
    rng = np.random.default_rng(1)
    n = 10
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = rng.standard_normal(n)
    Ainv = np.linalg.inv(A)
    x, it, rel = pcg(lambda v: A @ v, lambda v: Ainv @ v, b, tol=1e-12)
    assert it == 1 and rel <= 1e-12


def test_pcg_unpreconditioned_terminates_within_n():
    rng = np.random.default_rng(2)
    n = 14
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + 0.3 * np.eye(n)
    b = rng.standard_normal(n)
    x, it, rel = pcg(lambda v: A @ v, lambda v: v, b, tol=1e-10, max_iter=4 * n)
    assert it <= n + 2 and rel <= 1e-10
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-7, atol=1e-9)


def _ext(nx, ny, levels):
    p = inputs.config_extension(nx=nx, ny=ny, levels=levels)
    m = mesh_from_problem(p)
    return p, m, ExtensionOracle(m, p.eta, levels)


def test_extension_matches_direct_solution():
    p, m, o = _ext(160, 28, 3)
    b = o.lift_rhs(p.g[:m.n_u])
    x, it, rel = o.solve(b, tol=1e-10)
    xd = spla.spsolve(o.sys.A.tocsc(), b)
    assert rel <= 1e-10 and it < 60
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    # Dirichlet data reproduced: the bar's tip moved, the obstacle and the outer walls did not
    con = o.con
    np.testing.assert_array_equal(x[con], p.g[:m.n_u][con])
    assert np.abs(x).max() <= 0.02 * (1 + 1e-9)


def test_extension_reproduces_rigid_motions():
    """eps(u) = 0 for u = c + w (-(y - y0), x - x0): with that field as boundary data on the solid
    and the outer faces, the discrete extension is the field itself, whatever mu_A."""
    p, m, o = _ext(160, 28, 3)
    X = inputs.vnode_coords(2, p.n, p.length)
    u = np.concatenate([0.3 - 0.7 * (X[:, 1] - 0.2), -0.1 + 0.7 * (X[:, 0] - 0.3)])
    b = o.lift_rhs(u)
    x, it, rel = o.solve(b, tol=1e-12)
    assert np.linalg.norm(x - u) <= 1e-10 * np.linalg.norm(u)


def test_extension_iterations_stay_bounded_under_refinement():
    """Three refinements of the same coarse mesh: a few more iterations per level at most (the thin
    bar is an obstacle only on the fine levels; coarse levels see it as averaged cells)."""
    its = []
    for nx, ny, lev in [(80, 14, 2), (160, 28, 3), (320, 56, 4)]:
        p, m, o = _ext(nx, ny, lev)
        _, it, rel = o.solve(o.lift_rhs(p.g[:m.n_u]), tol=1e-6)
        assert rel <= 1e-6
        its.append(it)
    assert all(b - a <= 4 for a, b in zip(its, its[1:])) and max(its) <= 20, its
