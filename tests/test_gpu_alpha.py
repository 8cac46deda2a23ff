"""GPU parity of per-cell alpha (gs_create_ex; solid density different from the fluid's) against
the FP64 oracle, through the C ABI.

Operators, row by row as for the scalar case (tests/rowcheck.py: error over the cellwise
absolute sum of the row, FP64 1e-12, FP32 1e-6): A x, the full saddle operator; diag(A) per
level entry by entry; the dense coarse solve with the coarsened alpha, the weighted
pressure Laplacian of the Cahouet-Chabard term and its V-cycle.  Solves: FP64-multigrid
iteration counts within max(2, 5 %) of the oracle's, solutions against the sparse direct solve.
A uniform alpha array reproduces the scalar solve to rounding.
"""
import numpy as np
import pytest

from oracle.fem import System
from oracle.krylov import StokesOracle, direct_solve
from oracle.mesh import mesh_from_problem
from oracle.mg import Hierarchy
from oracle.pressure import PressureHierarchy, pressure_laplacian
from paper_2305_08986_gb300 import inputs
from tests.rowcheck import AbsOperators, row_error

pytestmark = pytest.mark.gpu

CASES = [
    dict(dim=2, n=(40, 24), levels=2, void=0.05, faces=None),
    dict(dim=3, n=(10, 8, 12), levels=2, void=0.0, faces=inputs.FACE_ZM | inputs.FACE_XP),
]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _problem(case, seed=0, contrast=1e4):
    p = inputs.config_random_field(case["dim"], case["n"], levels=case["levels"], seed=seed, contrast=contrast,
                                   alpha=1.0, faces=case["faces"], void_fraction=case["void"])
    rng = np.random.default_rng(seed + 100)
    p.alpha = np.exp(rng.uniform(0.0, np.log(1e3), len(p.eta)))  # log-uniform alpha in [1, 1e3]
    return p


@pytest.mark.parametrize("case", CASES)
def test_operators_with_alpha_per_cell(case):
    import torch
    from paper_2305_08986_gb300 import gs
    # operators on a contrast-1e6 field (rows of the fluid cells checked at their own magnitude)
    p = _problem(case, contrast=1e6)
    m = mesh_from_problem(p)
    sysm = System(m, p.eta, p.alpha)
    s = gs.Solver.from_problem(p, mg_precision=64)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(m.N)
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    ab = AbsOperators(m, p.eta, p.alpha)
    s.vmult(xt, yt)
    assert row_error(yt.cpu().numpy(), sysm.K @ x, ab.K, x) <= 1e-12
    xu = torch.tensor(x[:m.n_u], device="cuda")
    yu = torch.empty_like(xu)
    s.vmult_A(xu, yu)
    assert row_error(yu.cpu().numpy(), sysm.A @ x[:m.n_u], ab.A, x[:m.n_u]) <= 1e-12
    y32 = torch.empty(m.n_u, dtype=torch.float32, device="cuda")
    s.vmult_A(xu.float(), y32)
    xr = xu.float().double().cpu().numpy()
    assert row_error(y32.double().cpu().numpy(), sysm.A @ xr, ab.A, xr) <= 1e-6
    # diagonals and the dense coarse solve on a contrast-1e4 field (the coarse solve's error grows
    # with the condition number of A_0)
    p = _problem(case)
    m = mesh_from_problem(p)
    s = gs.Solver.from_problem(p, mg_precision=64)
    H = Hierarchy(m, p.eta, p.alpha, p.levels)
    for l, lv in enumerate(H.levels):
        d = torch.empty(lv.mesh.n_u, dtype=torch.float64, device="cuda")
        s.apply_level(l, 2, None, d)                                  # diag(A_l)
        assert np.max(np.abs(d.cpu().numpy() - lv.D) / np.abs(lv.D)) <= 1e-13
    c0 = H.levels[0]
    free = ~c0.sys.u_constrained
    b0 = rng.standard_normal(c0.mesh.n_u)
    b0[~free] = 0.0
    y0 = torch.empty_like(torch.tensor(b0, device="cuda"))
    s.apply_level(0, 10, torch.tensor(b0, device="cuda"), y0)       # A_0^{-1}
    ref = np.zeros_like(b0)
    ref[free] = np.linalg.solve(c0.A.toarray()[np.ix_(free, free)], b0[free])
    assert rel(y0.cpu().numpy(), ref) <= 1e-9


@pytest.mark.parametrize("case", CASES)
def test_weighted_pressure_laplacian_and_vcycle(case):
    import torch
    from paper_2305_08986_gb300 import gs
    p = _problem(case, seed=2)
    m = mesh_from_problem(p)
    s = gs.Solver.from_problem(p, mg_precision=64)
    assert s.info().schur_cc == 1
    ph = PressureHierarchy(m, p.levels, degree=2, alpha=p.alpha)
    K, c = pressure_laplacian(m, ph.abar / p.alpha)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(m.Np)
    y = torch.empty(m.Np, dtype=torch.float64, device="cuda")
    s.apply_level(p.levels - 1, 13, torch.tensor(x, device="cuda"), y)  # K_p^w x
    assert row_error(y.cpu().numpy(), K @ x, abs(K).tocsr(), x) <= 1e-12
    r = rng.standard_normal(m.Np)
    s.apply_level(p.levels - 1, 14, torch.tensor(r, device="cuda"), y)  # V_p(r)
    assert rel(y.cpu().numpy(), ph.apply_inverse(r)) <= 1e-10
    inf = s.info()
    for l in range(1, p.levels):
        assert abs(inf.plambda_max[l] - ph.levels[l]["lam_hi"]) <= 1e-10 * ph.levels[l]["lam_hi"]


def test_channel_solve_with_solid_density_ten_times_the_fluid():
    import torch
    from paper_2305_08986_gb300 import gs
    p = inputs.config_channel(nx=160, ny=28, levels=3, rho_ratio=10.0)
    m = mesh_from_problem(p)
    o = StokesOracle(m, p.eta, p.alpha, 3)
    b = o.sys.lift_rhs(p.f, p.g)
    _, it_o, rel_o, _ = o.solve(b, tol=1e-10)
    xd = direct_solve(o.sys, b)
    bt = torch.tensor(b, device="cuda")
    for prec in (64, 32):
        s = gs.Solver.from_problem(p, mg_precision=prec)
        f = torch.tensor(p.f, device="cuda")
        g = torch.tensor(p.g, device="cuda")
        bl = torch.empty_like(f)
        s.lift_rhs(f, g, bl)
        assert rel(bl.cpu().numpy(), b) <= 1e-13
        x = torch.zeros_like(bt)
        it, rr, st = s.solve(bt, x, tol=1e-10)
        assert st == 0 and rr <= 1e-10
        if prec == 64:
            assert abs(it - it_o) <= max(2, 0.05 * it_o), (it, it_o)
        else:
            assert it <= it_o + max(3, 0.1 * it_o), (it, it_o)
        assert rel(x.cpu().numpy(), xd) <= 1e-7


def test_uniform_alpha_array_matches_the_scalar_solve():
    import torch
    from paper_2305_08986_gb300 import gs
    p = inputs.config_channel(nx=160, ny=28, levels=3)
    f = torch.tensor(p.f, device="cuda")
    g = torch.tensor(p.g, device="cuda")
    out = []
    for al in (p.alpha, np.full(len(p.eta), p.alpha)):
        p.alpha = al
        s = gs.Solver.from_problem(p, mg_precision=64)
        b = torch.empty_like(f)
        s.lift_rhs(f, g, b)
        x = torch.zeros_like(b)
        it, rr, st = s.solve(b, x, tol=1e-10)
        out.append((it, x.cpu().numpy()))
    # the coefficients round differently (alpha h^2 / 900 against (h^2 / 900) alpha_K)
    assert abs(out[0][0] - out[1][0]) <= 1
    assert rel(out[1][1], out[0][1]) <= 1e-9
