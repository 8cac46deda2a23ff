"""Pins of the oracle's rigid-body deflation of stiff inclusions (oracle/deflation.py)."""
import numpy as np
import scipy.ndimage as ndi

from oracle.deflation import Deflation, inclusion_labels, stiff_cells
from oracle.fem import System
from oracle.krylov import StokesOracle
from oracle.mesh import Mesh, mesh_from_problem
from paper_2305_08986_gb300 import inputs


def _partition(labels):
    return sorted(tuple(np.nonzero(labels == k)[0]) for k in range(1, labels.max() + 1))


def test_inclusion_labels_match_a_flood_fill():
    """Components of node-sharing cells against scipy's labelling with full connectivity."""
    rng = np.random.default_rng(3)
    for dim, n in ((2, (13, 9)), (3, (5, 4, 6))):
        m = Mesh(dim, n, (1.0,) * dim)
        stiff = rng.uniform(size=m.Nc) < 0.3
        lab = inclusion_labels(m, stiff)
        grid = stiff.reshape(n[::-1])  # (z, y, x) with x fastest
        ref, nref = ndi.label(grid, structure=np.ones((3,) * dim))
        assert lab.max() == nref
        assert _partition(lab) == _partition(ref.ravel())
        # labels follow the first cell of each inclusion
        firsts = [np.nonzero(lab == k)[0][0] for k in range(1, lab.max() + 1)]
        assert firsts == sorted(firsts)


def test_stiff_cells_threshold():
    m = Mesh(2, (4, 4), (1.0, 1.0))
    eta = np.ones(16)
    assert not stiff_cells(m, eta).any()
    eta[5] = 999.0  # contrast below 1e3: no inclusion
    assert not stiff_cells(m, eta).any()
    eta[5] = 1e4
    assert np.nonzero(stiff_cells(m, eta))[0].tolist() == [5]


def _disc_problem(eta_in=1e6, alpha=100.0):
    return inputs.config_discs(n=32, levels=3, n_discs=4, eta_in=eta_in, alpha=alpha, seed=2, rmin=0.05, rmax=0.1)


def test_galerkin_projection():
    """After x += Z E^-1 Z^T r the new residual is orthogonal to the deflation space."""
    p = _disc_problem()
    m = mesh_from_problem(p)
    A = System(m, p.eta, p.alpha).A
    d = Deflation(m, p.eta, A)
    assert d.m >= 6 and d.m % 3 == 0
    r = np.random.default_rng(0).standard_normal(m.n_u)
    r_new = r - A @ d.correction(r)
    assert np.linalg.norm(d.Z.T @ r_new) <= 1e-9 * np.linalg.norm(d.Z.T @ r)


def _floating_discs(dim, eta_in, n):
    """Two stiff inclusions away from the (Dirichlet) boundary."""
    m = Mesh(dim, (n,) * dim, (1.0,) * dim)
    c = inputs.cell_centroids(dim, m.n, m.length)
    centres = [(0.3, 0.35, 0.4)[:dim], (0.68, 0.6, 0.55)[:dim]]
    inside = np.zeros(m.Nc, dtype=bool)
    for ctr, r in zip(centres, (0.12, 0.15)):
        inside |= ((c - np.array(ctr)) ** 2).sum(axis=1) <= r * r
    return m, np.where(inside, eta_in, 1.0)


def test_rigid_modes_carry_no_strain_inside():
    """A rigid motion is linear, so its viscous energy inside a floating inclusion is zero: E does
    not change when the inclusions' eta changes (a wrong rotation sign or centre, or a missing
    node, would leave strain inside and scale E with eta)."""
    for dim, n in ((2, 24), (3, 10)):
        Es = []
        for eta_in in (1e4, 1e7):
            m, eta = _floating_discs(dim, eta_in, n)
            d = Deflation(m, eta, System(m, eta, 30.0).A)
            assert d.m == (6 if dim == 2 else 12)
            Es.append(d.E)
        assert np.abs(Es[0] - Es[1]).max() <= 1e-6 * np.abs(Es[0]).max()
    # and E is symmetric positive definite
    assert np.allclose(Es[0], Es[0].T, rtol=1e-12, atol=1e-12 * np.abs(Es[0]).max())
    assert np.linalg.eigvalsh(0.5 * (Es[0] + Es[0].T)).min() > 0


def test_deflation_restores_convergence():
    """Stiff discs below the coarse-cell size: the plain V-cycle stalls, the deflated one converges."""
    p = inputs.config_discs(n=64, levels=4, n_discs=10, seed=5)
    m = mesh_from_problem(p)
    plain = StokesOracle(m, p.eta, p.alpha, p.levels)
    defl = StokesOracle(m, p.eta, p.alpha, p.levels, deflate=True)
    b = plain.sys.lift_rhs(p.f, p.g)
    _, it_p, rel_p, _ = plain.solve(b, tol=1e-8, max_iter=150)
    _, it_d, rel_d, _ = defl.solve(b, tol=1e-8, max_iter=150)
    assert rel_d <= 1e-8 and it_d < 150
    assert rel_p > 1e-8 or it_p > 2 * it_d
