"""Pins of the oracle's multigrid pieces (oracle/mg.py) against closed forms and invariants."""
import math

import numpy as np
import pytest

from oracle.fem import System
from oracle.mesh import Mesh
from oracle.mg import (Hierarchy, chebyshev, lanczos_max, lanczos_start, prolongation,
                       prolongation_1d, splitmix64)
from paper_2305_08986_gb300 import inputs


def test_splitmix64_published_value():
    """First output of SplitMix64 seeded with 0 (the generator's published reference code)."""
    assert splitmix64(0) == 0xE220A8397B1DCDAF
    v = lanczos_start(4, 0, 0)
    assert np.all(np.abs(v) < 1.0)
    assert v[0] == 2.0 * ((0xE220A8397B1DCDAF >> 11) * 2.0 ** -53) - 1.0


def test_prolongation_1d_stencil():
    """Q2 embedding: fine vertices copy coarse nodes, fine quarter points get (3/8, 3/4, -1/8)."""
    P = prolongation_1d(2).toarray()
    assert P.shape == (9, 5)
    exp = np.zeros((9, 5))
    exp[0, 0] = exp[2, 1] = exp[4, 2] = exp[6, 3] = exp[8, 4] = 1.0
    exp[1, 0:3] = [3 / 8, 3 / 4, -1 / 8]
    exp[3, 0:3] = [-1 / 8, 3 / 4, 3 / 8]
    exp[5, 2:5] = [3 / 8, 3 / 4, -1 / 8]
    exp[7, 2:5] = [-1 / 8, 3 / 4, 3 / 8]
    np.testing.assert_allclose(P, exp, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_prolongation_reproduces_quadratics(dim):
    cm = Mesh(dim, (2, 3, 2)[:dim], (1.0, 0.6, 0.8)[:dim], dirichlet_faces=0)
    fm = Mesh(dim, tuple(2 * k for k in cm.n), cm.length, dirichlet_faces=0)
    P = prolongation(cm, fm)
    def field(m):
        X = m.vnode_tuples() * (np.array(m.h) / 2.0)
        comps = []
        for a in range(dim):
            x = X[:, a]
            y = X[:, (a + 1) % dim]
            comps.append(1.0 + 2 * x - 3 * x * x + x * y + 0.5 * y * y)
        return np.concatenate(comps)
    np.testing.assert_allclose(P @ field(cm), field(fm), rtol=1e-13, atol=1e-13)


def test_prolongation_constraints():
    cm = Mesh(2, (2, 2), (1.0, 1.0))
    fm = Mesh(2, (4, 4), (1.0, 1.0))
    P = prolongation(cm, fm)
    fc = np.tile(fm.vnode_constrained(), 2)
    cc = np.tile(cm.vnode_constrained(), 2)
    assert abs(P[fc]).sum() == 0.0 and abs(P[:, cc]).sum() == 0.0


@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_chebyshev_closed_form(k):
    """On A = diag(lam), D = I the Chebyshev error after k steps is T_k((theta-lam)/delta) /
    T_k(theta/delta) times the initial error, componentwise (Saad, Sec. 12.3)."""
    lam = np.linspace(0.05, 2.0, 17)
    import scipy.sparse as sp
    A = sp.diags(lam).tocsr()
    lo, hi = 0.1, 2.1
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    xs = np.random.default_rng(0).standard_normal(17)
    b = lam * xs
    x0 = np.random.default_rng(1).standard_normal(17)
    x = chebyshev(A, np.ones(17), b, x0, k, lo, hi)
    Tk = lambda t: np.cosh(k * np.arccosh(t)) if np.all(np.abs(t) >= 1) else np.cos(k * np.arccos(np.clip(t, -1, 1)))
    def T(t):
        t = np.asarray(t, dtype=float)
        out = np.empty_like(t)
        inside = np.abs(t) <= 1
        out[inside] = np.cos(k * np.arccos(t[inside]))
        out[~inside] = np.sign(t[~inside]) ** k * np.cosh(k * np.arccosh(np.abs(t[~inside])))
        return out
    ratio = T((theta - lam) / delta) / T(np.array([theta / delta]))[0]
    np.testing.assert_allclose(x - xs, ratio * (x0 - xs), rtol=1e-10, atol=1e-12)
    # zero initial guess: the error starts at -xs
    x = chebyshev(A, np.ones(17), b, None, k, lo, hi)
    np.testing.assert_allclose(x - xs, ratio * (-xs), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_lanczos_brackets_spectrum(dim):
    p = inputs.config_random_field(dim, (6, 4, 4)[:dim], seed=4, contrast=1e4, alpha=5.0)
    m = Mesh(dim, p.n, p.length, p.void, p.dirichlet_faces)
    s = System(m, p.eta, p.alpha, need_pressure=False)
    D = s.A.diagonal()
    S = s.A.toarray() / np.sqrt(np.outer(D, D))
    ev = np.linalg.eigvalsh(S[np.ix_(~s.u_constrained, ~s.u_constrained)])
    v0 = lanczos_start(m.n_u, 0, 1)
    v0[s.u_constrained] = 0.0
    lam = lanczos_max(s.A, D, v0, 12)
    assert lam <= ev[-1] * (1 + 1e-12)       # Ritz values interlace
    assert lam >= 0.8 * ev[-1]                # the extreme one converges fast


@pytest.mark.parametrize("dim,n,levels,kind", [
    (2, (16, 16), 3, "one"), (3, (4, 4, 4), 2, "one"), (2, (8, 4), 3, "rand"), (3, (4, 4, 4), 2, "rand")])
def test_vcycle_symmetric_and_contracting(dim, n, levels, kind):
    """The V-cycle is a symmetric operator (Chebyshev pre/post smoothing with the same
    polynomial); its error propagation I - V A contracts strongly for eta = 1 and stays
    below 1 for rough random coefficients."""
    p = inputs.config_random_field(dim, n, seed=11, contrast=1e3, alpha=2.0)
    if kind == "one":
        p.eta[:] = 1.0
    m = Mesh(dim, p.n, p.length, p.void, p.dirichlet_faces)
    H = Hierarchy(m, p.eta, p.alpha, levels)
    A = H.levels[-1].A.toarray()
    nu = A.shape[0]
    free = ~H.levels[-1].sys.u_constrained
    idx = np.nonzero(free)[0]
    Vm = np.zeros((nu, len(idx)))
    for c, i in enumerate(idx):
        e = np.zeros(nu)
        e[i] = 1.0
        Vm[:, c] = H.vcycle(e)
    Vf = Vm[idx]
    assert np.abs(Vf - Vf.T).max() <= 1e-9 * np.abs(Vf).max()
    E = np.eye(len(idx)) - Vf @ A[np.ix_(idx, idx)]
    rho = np.abs(np.linalg.eigvals(E)).max()
    assert rho < (0.2 if kind == "one" else 0.95), rho


@pytest.mark.parametrize("dim", [2, 3])
def test_wathen_bounds(dim):
    """eig(D^{-1} M_p(1/eta)) lies in [2^-d, (3/2)^d] for any positive cell weights."""
    p = inputs.config_random_field(dim, (5, 4, 3)[:dim], seed=6, contrast=1e6, void_fraction=0.1)
    m = Mesh(dim, p.n, p.length, p.void, p.dirichlet_faces)
    s = System(m, p.eta, p.alpha)
    M = s.Mpw.toarray()
    d = np.diag(M)
    ev = np.linalg.eigvalsh(M / np.sqrt(np.outer(d, d)))
    assert ev.min() >= 0.5 ** dim * (1 - 1e-12)
    assert ev.max() <= 1.5 ** dim * (1 + 1e-12)
