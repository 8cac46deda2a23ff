"""Pins of the oracle's per-cell alpha (rho_s != rho_f, alpha = rho / (gamma tau) per cell): the
assembled mass term against a loop over cells, the reduction to the scalar case, the weighted
pressure Laplacian of the Cahouet-Chabard term, and a solve against the direct solution."""
import numpy as np
import pytest

from oracle.fem import CellMatrices, System
from oracle.krylov import StokesOracle, direct_solve, normalize_pressure
from oracle.mesh import Mesh, mesh_from_problem
from oracle.pressure import pressure_laplacian
from paper_2305_08986_gb300 import inputs


@pytest.mark.parametrize("dim,n", [(2, (3, 2)), (3, (2, 2, 1))])
def test_mass_term_is_the_sum_of_weighted_cell_masses(dim, n):
    """A_raw(alpha_K) - A_raw(0) = sum_K alpha_K M_K, the right side assembled by a plain loop."""
    m = Mesh(dim, n, (1.0, 0.7, 0.4)[:dim], dirichlet_faces=0)
    rng = np.random.default_rng(1)
    nc = int(np.prod(n))
    eta = rng.uniform(1.0, 5.0, nc)
    al = rng.uniform(0.5, 20.0, nc)
    d = (System(m, eta, al, need_pressure=False).A_raw - System(m, eta, 0.0, need_pressure=False).A_raw).toarray()
    cm = CellMatrices(dim, m.h)
    ref = np.zeros((m.n_u, m.n_u))
    ud = m.cell_udofs()
    for k in range(nc):
        for i, gi in enumerate(ud[k]):
            for j, gj in enumerate(ud[k]):
                ref[gi, gj] += al[k] * cm.mass[i, j]
    np.testing.assert_allclose(d, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_uniform_alpha_array_is_the_scalar_case():
    p = inputs.config_box_inclusion(2, (16, 16), 2, 1e3, 25.0, seed=3, align_coarse=True)
    m = mesh_from_problem(p)
    o1 = StokesOracle(m, p.eta, 25.0, 2)
    o2 = StokesOracle(m, p.eta, np.full(int(np.prod(p.n)), 25.0), 2)
    assert abs(o1.sys.K - o2.sys.K).max() == 0.0
    b = o1.sys.lift_rhs(p.f, p.g)
    x1, it1, r1, _ = o1.solve(b, tol=1e-10)
    x2, it2, r2, _ = o2.solve(b, tol=1e-10)
    assert it1 == it2 and np.array_equal(x1, x2)


def test_weighted_pressure_laplacian():
    """Constant weight c scales K_p by c; any weights keep the constant in the kernel of the
    pure-Neumann Laplacian (every velocity face Dirichlet) and keep it positive semidefinite."""
    m = Mesh(2, (6, 5), (1.0, 0.8))
    K1, c = pressure_laplacian(m)
    K3, _ = pressure_laplacian(m, np.full(30, 3.0))
    free = ~c
    np.testing.assert_allclose(K3.toarray()[np.ix_(free, free)], 3.0 * K1.toarray()[np.ix_(free, free)],
                               rtol=1e-14, atol=1e-14)
    w = np.random.default_rng(2).uniform(0.1, 10.0, 30)
    Kw = pressure_laplacian(m, w)[0].toarray()[np.ix_(free, free)]
    assert np.abs(Kw @ np.ones(free.sum())).max() <= 1e-12 * np.abs(Kw).max()
    ev = np.linalg.eigvalsh(Kw)
    assert ev[0] >= -1e-12 * ev[-1] and ev[1] > 0


def test_solve_with_solid_density_ten_times_the_fluid():
    """FSI2i density ratio rho_s / rho_f = 10 (alpha 10x larger on the bar)."""
    p = inputs.config_channel(nx=160, ny=28, levels=3, rho_ratio=10.0)
    m = mesh_from_problem(p)
    o = StokesOracle(m, p.eta, p.alpha, 3)
    assert o.schur == "cc" and o.pmg.abar == 1e4
    b = o.sys.lift_rhs(p.f, p.g)
    x, it, rel, _ = o.solve(b, tol=1e-10)
    assert rel <= 1e-10 and it < 80
    xd = direct_solve(o.sys, b)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    # the scalar-alpha system differs: the mass term of the bar carries alpha_s
    o1 = StokesOracle(m, p.eta, 1e3, 3)
    assert abs(o1.sys.A - o.sys.A).max() > 0.0
