"""GPU parity of the individual operators (called through the C ABI) against the FP64 oracle.

Sizes span several CTA tiles and ragged tile edges; obstacle cells, do-nothing faces and
high-contrast random viscosity are included.  Tolerances: FP64 operators 1e-12 (norm-wise
relative, from the arithmetic: a few dozen rounded FMAs per entry), FP32 operators 2e-6.
"""
import numpy as np
import pytest

from oracle.fem import CellMatrices, System, apply_A_rows
from oracle.mesh import Mesh, mesh_from_problem
from oracle.mg import Hierarchy, prolongation, schur_apply_inv
from paper_2305_08986_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [
    dict(dim=2, n=(40, 24), levels=2, void=0.0, faces=None),        # 2 x 2 tiles, ragged
    dict(dim=2, n=(70, 18), levels=2, void=0.08, faces=inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP),
    dict(dim=3, n=(10, 8, 12), levels=2, void=0.0, faces=None),     # ragged 3D tiles
    dict(dim=3, n=(8, 6, 6), levels=2, void=0.1, faces=inputs.FACE_ZM | inputs.FACE_XP),
]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _setup(case, seed=0, mg_precision=64):
    import torch
    from paper_2305_08986_gb300 import gs
    p = inputs.config_random_field(case["dim"], case["n"], levels=case["levels"], seed=seed,
                                   contrast=1e6, alpha=7.0, faces=case["faces"], void_fraction=case["void"])
    s = gs.Solver.from_problem(p, mg_precision=mg_precision)
    return p, s, torch


@pytest.mark.parametrize("case", CASES)
def test_apply_A_fp64_and_fp32(case):
    p, s, torch = _setup(case)
    m = mesh_from_problem(p)
    sysm = System(m, p.eta, p.alpha, need_pressure=False)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(m.n_u)
    y_ref = sysm.A @ x
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    s.vmult_A(xt, yt)
    assert rel(yt.cpu().numpy(), y_ref) <= 1e-12
    x32 = xt.float()
    y32 = torch.empty_like(x32)
    s.vmult_A(x32, y32)
    ref32 = sysm.A @ x32.double().cpu().numpy()
    assert rel(y32.double().cpu().numpy(), ref32) <= 2e-6
    # unconstrained operator
    s.apply_level(p.levels - 1, 12, xt, yt)
    assert rel(yt.cpu().numpy(), sysm.A_raw @ x) <= 1e-12


@pytest.mark.parametrize("case", CASES)
def test_saddle_B_BT(case):
    p, s, torch = _setup(case)
    m = mesh_from_problem(p)
    sysm = System(m, p.eta, p.alpha)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(m.N)
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    s.vmult(xt, yt)
    assert rel(yt.cpu().numpy(), sysm.K @ x) <= 1e-12
    L = p.levels - 1
    yp = torch.empty(m.Np, dtype=torch.float64, device="cuda")
    s.apply_level(L, 6, xt[:m.n_u].contiguous(), yp)
    assert rel(yp.cpu().numpy(), sysm.B @ x[:m.n_u]) <= 1e-12
    yu = torch.empty(m.n_u, dtype=torch.float64, device="cuda")
    s.apply_level(L, 7, xt[m.n_u:].contiguous(), yu)
    assert rel(yu.cpu().numpy(), sysm.B.T @ x[m.n_u:]) <= 1e-12


@pytest.mark.parametrize("case", CASES)
def test_diag_and_transfers(case):
    p, s, torch = _setup(case)
    m = mesh_from_problem(p)
    H = Hierarchy(m, p.eta, p.alpha, p.levels)
    L = p.levels - 1
    d = torch.empty(m.n_u, dtype=torch.float64, device="cuda")
    s.apply_level(L, 2, None, d)
    assert rel(d.cpu().numpy(), H.levels[L].D) <= 1e-13
    P = H.levels[L].P
    rng = np.random.default_rng(3)
    rf = rng.standard_normal(P.shape[0])
    rc = torch.empty(P.shape[1], dtype=torch.float64, device="cuda")
    s.apply_level(L, 4, torch.tensor(rf, device="cuda"), rc)
    assert rel(rc.cpu().numpy(), P.T @ rf) <= 1e-14
    xc = rng.standard_normal(P.shape[1])
    xf0 = rng.standard_normal(P.shape[0])
    xf = torch.tensor(xf0, device="cuda")
    s.apply_level(L, 5, torch.tensor(xc, device="cuda"), xf)
    assert rel(xf.cpu().numpy(), xf0 + P @ xc) <= 1e-14


@pytest.mark.parametrize("case", CASES)
def test_schur_mass_and_inverse(case):
    p, s, torch = _setup(case)
    m = mesh_from_problem(p)
    sysm = System(m, p.eta, p.alpha)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(m.Np)
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    L = p.levels - 1
    s.apply_level(L, 8, xt, yt)
    assert rel(yt.cpu().numpy(), sysm.Mpw @ x) <= 1e-12
    s.apply_level(L, 9, xt, yt)
    assert rel(yt.cpu().numpy(), schur_apply_inv(sysm.Mpw, x, m.dim)) <= 1e-11


@pytest.mark.parametrize("case", CASES)
def test_lift_rhs(case):
    p, s, torch = _setup(case)
    m = mesh_from_problem(p)
    sysm = System(m, p.eta, p.alpha)
    f = torch.tensor(p.f, device="cuda")
    g = torch.tensor(p.g, device="cuda")
    b = torch.empty_like(f)
    s.lift_rhs(f, g, b)
    ref = sysm.lift_rhs(p.f, p.g)
    assert rel(b.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("case", CASES)
def test_lanczos_bounds_and_smoother(case):
    p, s, torch = _setup(case, mg_precision=64)
    m = mesh_from_problem(p)
    H = Hierarchy(m, p.eta, p.alpha, p.levels)
    inf = s.info()
    for l in range(1, p.levels):
        assert abs(inf.lambda_max[l] - H.levels[l].lam_hi) <= 1e-10 * H.levels[l].lam_hi
    L = p.levels - 1
    lv = H.levels[L]
    rng = np.random.default_rng(5)
    b = rng.standard_normal(m.n_u)
    x0 = rng.standard_normal(m.n_u)
    from oracle.mg import chebyshev
    y = torch.empty(m.n_u, dtype=torch.float64, device="cuda")
    s.apply_level(L, 3, torch.tensor(b, device="cuda"), y)
    ref = chebyshev(lv.A, 1.0 / lv.D, b, None, 4, lv.lam_hi / 15, lv.lam_hi)
    assert rel(y.cpu().numpy(), ref) <= 1e-10
    s.apply_level(L, 3, torch.tensor(b, device="cuda"), y, aux=torch.tensor(x0, device="cuda"))
    ref = chebyshev(lv.A, 1.0 / lv.D, b, x0, 4, lv.lam_hi / 15, lv.lam_hi)
    assert rel(y.cpu().numpy(), ref) <= 1e-10


def test_fullsize_channel_apply_sampled():
    """Configuration 2 mesh as stated (1280 x 210, FP64 and FP32 apply) at sampled rows."""
    import torch
    from paper_2305_08986_gb300 import gs
    p = inputs.config_channel(nx=1280, ny=210, levels=1)
    s = gs.Solver.from_problem(p, coarse_mode=1)
    m = mesh_from_problem(p)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(m.n_u)
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    s.vmult_A(xt, yt)
    rows = rng.choice(m.n_u, 400, replace=False)
    ref = apply_A_rows(m, p.eta, p.alpha, x, rows)
    y = yt.cpu().numpy()[rows]
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
    y32 = torch.empty(m.n_u, dtype=torch.float32, device="cuda")
    s.vmult_A(xt.float(), y32)
    ref32 = apply_A_rows(m, p.eta, p.alpha, xt.float().double().cpu().numpy(), rows)
    assert np.linalg.norm(y32.double().cpu().numpy()[rows] - ref32) <= 2e-6 * np.linalg.norm(ref32)


def test_fullsize_spheres_apply_sampled():
    """Configuration 3 mesh (64^3) FP64 apply at sampled rows."""
    import torch
    from paper_2305_08986_gb300 import gs
    p = inputs.config_spheres(n=64, levels=5)
    s = gs.Solver.from_problem(p)
    m = mesh_from_problem(p)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(m.n_u)
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    s.vmult_A(xt, yt)
    rows = rng.choice(m.n_u, 200, replace=False)
    ref = apply_A_rows(m, p.eta, p.alpha, x, rows)
    assert np.linalg.norm(yt.cpu().numpy()[rows] - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("case", CASES)
def test_pressure_laplacian_transfers_vcycle(case):
    """Cahouet-Chabard pieces: K_p apply, Q1 transfers, Lanczos bounds and the pressure V-cycle
    (FP64 multigrid) against oracle/pressure.py."""
    from oracle.pressure import PressureHierarchy
    p, s, torch = _setup(case, mg_precision=64)
    m = mesh_from_problem(p)
    H = PressureHierarchy(m, p.levels, degree=2)
    inf = s.info()
    assert inf.schur_cc == 1
    L = p.levels - 1
    rng = np.random.default_rng(12)
    x = rng.standard_normal(m.Np)
    y = torch.empty(m.Np, dtype=torch.float64, device="cuda")
    s.apply_level(L, 13, torch.tensor(x, device="cuda"), y)
    assert rel(y.cpu().numpy(), H.levels[L]["K"] @ x) <= 1e-12
    for l in range(1, p.levels):
        assert abs(inf.plambda_max[l] - H.levels[l]["lam_hi"]) <= 1e-10 * H.levels[l]["lam_hi"]
    P = H.levels[L]["P"]
    rc = torch.empty(P.shape[1], dtype=torch.float64, device="cuda")
    s.apply_level(L, 15, torch.tensor(x, device="cuda"), rc)
    assert rel(rc.cpu().numpy(), P.T @ x) <= 1e-14
    xc = rng.standard_normal(P.shape[1])
    xf = torch.tensor(x, device="cuda")
    s.apply_level(L, 16, torch.tensor(xc, device="cuda"), xf)
    assert rel(xf.cpu().numpy(), x + P @ xc) <= 1e-14
    s.apply_level(L, 14, torch.tensor(x, device="cuda"), y)
    assert rel(y.cpu().numpy(), H.apply_inverse(x)) <= 1e-10


TILE_HEIGHT_CASES = {
    "channel_small": lambda: inputs.config_channel(nx=160, ny=28, levels=3),
    "box_ragged": lambda: inputs.config_box_inclusion(2, (100, 52), 3, 1e4, 30.0, seed=4, align_coarse=True),
}


@pytest.mark.parametrize("name", sorted(TILE_HEIGHT_CASES))
def test_tile_heights_give_identical_solves(name):
    """The 2D cell kernel's tile height (32 x 16, 32 x 17, 32 x 8 evaluated cells, forced or
    autotuned) changes only the launch shape: every node sums its cell contributions in a fixed
    order, so the solve is bitwise the same."""
    import torch
    from paper_2305_08986_gb300 import gs
    p = TILE_HEIGHT_CASES[name]()
    outs = []
    for mode in (1, 2, 3, 0):
        s = gs.Solver.from_problem(p, tile_autotune=mode)
        inf = s.info()
        rows = [inf.tile_rows[l] for l in range(p.levels)]
        assert all(r in (8, 16, 17) for r in rows) and inf.saddle_tile_rows in (8, 16, 17)
        if mode:
            assert rows == [(16, 17, 8)[mode - 1]] * p.levels
        f = torch.tensor(p.f, device="cuda")
        g = torch.tensor(p.g, device="cuda")
        b = torch.empty_like(f)
        s.lift_rhs(f, g, b)
        x = torch.zeros_like(b)
        it, rr, _ = s.solve(b, x, tol=1e-9)
        outs.append((x.cpu(), it, rr))
    for x, it, rr in outs[1:]:
        assert (it, rr) == outs[0][1:] and torch.equal(x, outs[0][0])
