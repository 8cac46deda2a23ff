"""GPU parity of the individual operators (called through the C ABI) against the FP64 oracle.

Sizes span several CTA tiles and ragged tile edges; obstacle cells, do-nothing faces and
random viscosity of contrast 1e6 are included.  Operator outputs are checked row by row
(tests/rowcheck.py): max_i |y_i - y_ref,i| / (sum_K |A_K| |x_K|)_i <= 1e-12 in FP64 and
<= FP32_ROW_TOL in FP32, so the rows of the fluid cells (~1e-6 of the stiff rows) are held to
their own magnitude.  The bound: a row is a sum of cell contributions, each the result of a
chain of at most ~10 rounded sweeps (3 x 3 integer line operators, coefficient scalings, the
gather over <= 2^d cells), so its error is a few tens of unit roundoffs of s_i: ~1e-15 in FP64
(1e-12 leaves three orders of margin) and a few 1e-7 in FP32 (u = 6e-8; measured at most 2.2e-7
on these cases, gate 1e-6).  Iterative outputs
(Chebyshev smoothers, the Schur inverse) are compared norm-wise.
"""
import numpy as np
import pytest

from oracle.fem import CellMatrices, System, apply_A_rows
from oracle.mesh import Mesh, mesh_from_problem
from oracle.mg import Hierarchy, prolongation, schur_apply_inv
from paper_2305_08986_gb300 import inputs
from tests.rowcheck import AbsOperators, abs_rows, row_error, sampled_row_error

pytestmark = pytest.mark.gpu

FP64_ROW_TOL = 1e-12
FP32_ROW_TOL = 1e-6

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
    ab = AbsOperators(m, p.eta, p.alpha)
    y_ref = sysm.A @ x
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    s.vmult_A(xt, yt)
    assert row_error(yt.cpu().numpy(), y_ref, ab.A, x) <= FP64_ROW_TOL
    x32 = xt.float()
    y32 = torch.empty_like(x32)
    s.vmult_A(x32, y32)
    xr = x32.double().cpu().numpy()
    assert row_error(y32.double().cpu().numpy(), sysm.A @ xr, ab.A, xr) <= FP32_ROW_TOL
    # unconstrained operator
    s.apply_level(p.levels - 1, 12, xt, yt)
    assert row_error(yt.cpu().numpy(), sysm.A_raw @ x, ab.A_raw, x) <= FP64_ROW_TOL


@pytest.mark.parametrize("case", CASES)
def test_saddle_B_BT(case):
    p, s, torch = _setup(case)
    m = mesh_from_problem(p)
    sysm = System(m, p.eta, p.alpha)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(m.N)
    xt = torch.tensor(x, device="cuda")
    yt = torch.empty_like(xt)
    ab = AbsOperators(m, p.eta, p.alpha)
    s.vmult(xt, yt)
    assert row_error(yt.cpu().numpy(), sysm.K @ x, ab.K, x) <= FP64_ROW_TOL
    L = p.levels - 1
    yp = torch.empty(m.Np, dtype=torch.float64, device="cuda")
    s.apply_level(L, 6, xt[:m.n_u].contiguous(), yp)
    assert row_error(yp.cpu().numpy(), sysm.B @ x[:m.n_u], ab.B, x[:m.n_u]) <= FP64_ROW_TOL
    yu = torch.empty(m.n_u, dtype=torch.float64, device="cuda")
    s.apply_level(L, 7, xt[m.n_u:].contiguous(), yu)
    assert row_error(yu.cpu().numpy(), sysm.B.T @ x[m.n_u:], ab.B.T.tocsr(), x[m.n_u:]) <= FP64_ROW_TOL


@pytest.mark.parametrize("case", CASES)
def test_diag_and_transfers(case):
    p, s, torch = _setup(case)
    m = mesh_from_problem(p)
    H = Hierarchy(m, p.eta, p.alpha, p.levels)
    L = p.levels - 1
    d = torch.empty(m.n_u, dtype=torch.float64, device="cuda")
    s.apply_level(L, 2, None, d)
    assert np.max(np.abs(d.cpu().numpy() - H.levels[L].D) / np.abs(H.levels[L].D)) <= 1e-13
    P = H.levels[L].P
    rng = np.random.default_rng(3)
    rf = rng.standard_normal(P.shape[0])
    rc = torch.empty(P.shape[1], dtype=torch.float64, device="cuda")
    s.apply_level(L, 4, torch.tensor(rf, device="cuda"), rc)
    assert row_error(rc.cpu().numpy(), P.T @ rf, abs(P.T).tocsr(), rf) <= 1e-14
    xc = rng.standard_normal(P.shape[1])
    xf0 = rng.standard_normal(P.shape[0])
    xf = torch.tensor(xf0, device="cuda")
    s.apply_level(L, 5, torch.tensor(xc, device="cuda"), xf)
    import scipy.sparse as sps
    PI = sps.hstack([sps.identity(P.shape[0]), abs(P)]).tocsr()   # scale |xf0| + |P| |xc|
    assert row_error(xf.cpu().numpy(), xf0 + P @ xc, PI, np.concatenate([xf0, xc])) <= 1e-14


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
    assert sysm.Mpw.min() >= 0.0   # the Q1 mass has positive entries: |M_p| = M_p
    assert row_error(yt.cpu().numpy(), sysm.Mpw @ x, sysm.Mpw, x) <= FP64_ROW_TOL
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
    # per row: b = F - K_raw g on free rows, scale |M| |f| + |K_raw| |g_c|
    import scipy.sparse as sps
    ab = AbsOperators(m, p.eta, p.alpha)
    gc = np.where(sysm.constrained, p.g, 0.0)
    Kraw_abs = sps.bmat([[ab.A_raw, abs(sysm.B_raw).T], [abs(sysm.B_raw), None]]).tocsr()
    Mabs = sps.block_diag([abs(sysm.Mu), sysm.Mp1]).tocsr()
    scale = Mabs @ np.abs(p.f) + Kraw_abs @ np.abs(gc)
    free = ~sysm.constrained
    err = np.abs(b.cpu().numpy() - ref)
    assert np.all(err[~free] == 0.0)
    assert np.max(err[free] / np.maximum(scale[free], 1e-300)) <= FP64_ROW_TOL


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
    assert sampled_row_error(y, ref, abs_rows(m, p.eta, p.alpha, x, rows)) <= FP64_ROW_TOL
    y32 = torch.empty(m.n_u, dtype=torch.float32, device="cuda")
    s.vmult_A(xt.float(), y32)
    xr = xt.float().double().cpu().numpy()
    ref32 = apply_A_rows(m, p.eta, p.alpha, xr, rows)
    assert sampled_row_error(y32.double().cpu().numpy()[rows], ref32,
                             abs_rows(m, p.eta, p.alpha, xr, rows)) <= FP32_ROW_TOL


def test_fullsize_spheres_apply_sampled():
    """Configuration 3 mesh (64^3, spheres of eta 1e6 in 1) FP64 and FP32 apply at sampled rows."""
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
    assert sampled_row_error(yt.cpu().numpy()[rows], ref, abs_rows(m, p.eta, p.alpha, x, rows)) <= FP64_ROW_TOL
    y32 = torch.empty(m.n_u, dtype=torch.float32, device="cuda")
    s.vmult_A(xt.float(), y32)
    xr = xt.float().double().cpu().numpy()
    ref32 = apply_A_rows(m, p.eta, p.alpha, xr, rows)
    assert sampled_row_error(y32.double().cpu().numpy()[rows], ref32,
                             abs_rows(m, p.eta, p.alpha, xr, rows)) <= FP32_ROW_TOL


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
    Kp = H.levels[L]["K"]
    assert row_error(y.cpu().numpy(), Kp @ x, abs(Kp).tocsr(), x) <= FP64_ROW_TOL
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
    """The 2D velocity-block kernel variant (cell tiles of 32 x 16, 32 x 17, 32 x 8 evaluated cells,
    or the strip kernel; forced or autotuned) changes only the launch shape: every variant sums a
    node's cell contributions in the same order, so the solve is bitwise the same."""
    import torch
    from paper_2305_08986_gb300 import gs
    p = TILE_HEIGHT_CASES[name]()
    outs = []
    for mode in (1, 2, 3, 4, 5, 0):
        s = gs.Solver.from_problem(p, tile_autotune=mode)
        inf = s.info()
        rows = [inf.tile_rows[l] for l in range(p.levels)]
        assert all(r in (0, 8, 16, 17) for r in rows) and inf.saddle_tile_rows in (8, 16, 17)
        if mode:
            if mode <= 4:
                assert rows == [(16, 17, 8, 0)[mode - 1]] * p.levels
        f = torch.tensor(p.f, device="cuda")
        g = torch.tensor(p.g, device="cuda")
        b = torch.empty_like(f)
        s.lift_rhs(f, g, b)
        x = torch.zeros_like(b)
        it, rr, _ = s.solve(b, x, tol=1e-9)
        outs.append((x.cpu(), it, rr))
    for x, it, rr in outs[1:]:
        assert (it, rr) == outs[0][1:] and torch.equal(x, outs[0][0])


TILE_DEPTH_CASES_3D = {
    "box_3d": lambda: inputs.config_box_inclusion(3, (24, 16, 20), 3, 1e5, 20.0, seed=6, align_coarse=True),
    "ragged_void_3d": lambda: inputs.config_random_field(3, (13, 9, 11), levels=1, seed=8, contrast=1e6, alpha=3.0,
                                                         faces=inputs.FACE_XM | inputs.FACE_ZP, void_fraction=0.1),
}


@pytest.mark.parametrize("name", sorted(TILE_DEPTH_CASES_3D))
def test_3d_tile_depths_give_identical_results(name):
    """The 3D cell tile of 8 x 8 x 8 or 8 x 8 x 4 evaluated cells (forced or autotuned): every node
    sums its cells' contributions in the order of their global parity class, so A x, the saddle
    operator and the whole solve are bitwise the same."""
    import torch
    from paper_2305_08986_gb300 import gs
    p = TILE_DEPTH_CASES_3D[name]()
    rng = np.random.default_rng(5)
    outs = []
    for mode in (1, 2, 0):
        s = gs.Solver.from_problem(p, tile_autotune=mode, coarse_mode=1 if p.levels == 1 else 0)
        inf = s.info()
        depths = [inf.tile_rows[l] for l in range(p.levels)]
        if mode:
            assert depths == [(8, 4)[mode - 1]] * p.levels and inf.saddle_tile_rows == (8, 4)[mode - 1]
        else:
            assert all(dd in (8, 4) for dd in depths) and inf.saddle_tile_rows in (8, 4)
        xk = torch.tensor(rng.standard_normal(s.n_total) if not outs else outs[0][0], device="cuda")
        yk = torch.empty_like(xk)
        s.vmult(xk, yk)
        xa32 = xk[:s.n_u].float().contiguous()
        ya32 = torch.empty_like(xa32)
        s32 = gs.Solver.from_problem(p, tile_autotune=mode, mg_precision=32, coarse_mode=1 if p.levels == 1 else 0)
        s32.vmult_A(xa32, ya32)
        if p.levels > 1:
            f = torch.tensor(p.f, device="cuda")
            g = torch.tensor(p.g, device="cuda")
            b = torch.empty_like(f)
            s.lift_rhs(f, g, b)
            x = torch.zeros_like(b)
            it, rr, _ = s.solve(b, x, tol=1e-9)
            sol = (x.cpu(), it, rr)
        else:
            sol = None
        outs.append((xk.cpu().numpy(), yk.cpu(), ya32.cpu(), sol))
    for _, y, y32, sol in outs[1:]:
        assert torch.equal(y, outs[0][1]) and torch.equal(y32, outs[0][2])
        if sol is not None:
            assert sol[1:] == outs[0][3][1:] and torch.equal(sol[0], outs[0][3][0])


@pytest.mark.parametrize("case", CASES[:2] + [dict(dim=2, n=(20, 6), levels=1, void=0.1, faces=inputs.FACE_YM)])
@pytest.mark.parametrize("variant", [1, 4])
def test_velocity_kernel_variants_bitwise(case, variant):
    """A x, b - A x and the Chebyshev step of the strip kernel and of the 32 x 16 tile kernel give
    the same bits (FP64 and FP32, with obstacles and do-nothing faces) and match the oracle row by
    row; the strip kernel is also checked on a mesh with a single strip and a single segment."""
    import torch
    from paper_2305_08986_gb300 import gs
    p = inputs.config_random_field(case["dim"], case["n"], levels=case["levels"], seed=3, contrast=1e6, alpha=7.0,
                                   faces=case["faces"], void_fraction=case["void"])
    m = mesh_from_problem(p)
    sysm = System(m, p.eta, p.alpha, need_pressure=False)
    ab = AbsOperators(m, p.eta, p.alpha)
    rng = np.random.default_rng(31)
    x, b, d = (rng.standard_normal(m.n_u) for _ in range(3))
    for prec, dt, tol in ((64, torch.float64, FP64_ROW_TOL), (32, torch.float32, FP32_ROW_TOL)):
        outs = []
        for v in (variant, 2):
            s = gs.Solver.from_problem(p, mg_precision=prec, tile_autotune=v, coarse_mode=1 if p.levels == 1 else 0)
            L = p.levels - 1
            xt = torch.tensor(x, device="cuda", dtype=dt)
            bt = torch.tensor(b, device="cuda", dtype=dt)
            ya, yr = torch.empty_like(xt), torch.empty_like(xt)
            s.apply_level(L, gs.OP_A, xt, ya)
            s.apply_level(L, gs.OP_RESIDUAL_A, xt, yr, aux=bt)
            aux = torch.tensor(np.concatenate([b, d, 1.0 / sysm.A.diagonal()]), device="cuda", dtype=dt)
            yc = torch.empty_like(xt)
            s.apply_level(L, gs.OP_CHEB_STEP, xt, yc, aux=aux)
            outs.append((ya.cpu(), yr.cpu(), yc.cpu(), aux.cpu()))
            xr = xt.double().cpu().numpy()
            assert row_error(ya.double().cpu().numpy(), sysm.A @ xr, ab.A, xr) <= tol
        for a0, a1 in zip(outs[0], outs[1]):
            assert torch.equal(a0, a1)


@pytest.mark.parametrize("case", CASES)
def test_single_chebyshev_step(case):
    """GS_OP_CHEB_STEP (the fused step the smoother launches): r = b - A x, d <- c1 d + c2 D^-1 r,
    y = x + d with the level's second-step coefficients, FP64 and FP32, row by row."""
    import torch
    from paper_2305_08986_gb300 import gs
    p, s, _ = _setup(case, mg_precision=64)
    m = mesh_from_problem(p)
    H = Hierarchy(m, p.eta, p.alpha, p.levels)
    L = p.levels - 1
    lv = H.levels[L]
    hi = lv.lam_hi
    lo = hi / 15.0
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    rn = 1.0 / (2.0 * sigma - rho)
    c1, c2 = rn * rho, 2.0 * rn / delta
    ab = AbsOperators(m, p.eta, p.alpha)
    rng = np.random.default_rng(21)
    x, b, d = (rng.standard_normal(m.n_u) for _ in range(3))
    dinv = 1.0 / lv.D
    scale_d = abs(c1) * np.abs(d) + abs(c2) * dinv * (np.abs(b) + ab.A @ np.abs(x))
    for dt, tol in ((torch.float64, FP64_ROW_TOL), (torch.float32, FP32_ROW_TOL)):
        if dt == torch.float32:
            s = gs.Solver.from_problem(p, mg_precision=32)
        xt = torch.tensor(x, device="cuda", dtype=dt)
        aux = torch.tensor(np.concatenate([b, d, dinv]), device="cuda", dtype=dt)
        yt = torch.empty_like(xt)
        # inputs as the kernel sees them (rounded to dt), taken before d is updated in place
        xr, br, dr, dir_ = [v.double().cpu().numpy() for v in (xt, aux[:m.n_u], aux[m.n_u:2 * m.n_u],
                                                               aux[2 * m.n_u:])]
        s.apply_level(L, gs.OP_CHEB_STEP, xt, yt, aux=aux)
        dref = c1 * dr + c2 * dir_ * (br - lv.A @ xr)
        err_d = np.abs(aux[m.n_u:2 * m.n_u].double().cpu().numpy() - dref)
        err_y = np.abs(yt.double().cpu().numpy() - (xr + dref))
        assert np.max(err_d / scale_d) <= tol
        assert np.max(err_y / (np.abs(x) + scale_d)) <= tol
