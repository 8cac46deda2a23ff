"""GPU parity of the corrector stage (gs_set_corrector; Sec. 3.1.2, Eq. "v_star" and Eq. "a_stab")
against the FP64 oracle (oracle/corrector.py), through the C ABI.

The velocity block gains rho (C + S): convection by the given field v° and the streamline
diffusion, both at the 3 x 3 Gauss points.  Checked: A_c x and the saddle operator K_c row by row
(FP64 1e-12, FP32 1e-6 of the row's absolute sum), diag(A_c) per level, the Chebyshev bounds from
the symmetric part per level, one V-cycle (FP64 multigrid, 1e-10), the solve against the sparse
direct solution of the non-symmetric system (1e-8) with the oracle's iteration count (FP64
multigrid, within max(2, 5 %)), and the return to the predictor stage (bitwise).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.corrector import CorrectorOracle, CorrectorSystem, convection_matrices
from oracle.krylov import StokesOracle
from oracle.mesh import mesh_from_problem
from paper_2305_08986_gb300 import inputs
from tests.rowcheck import AbsOperators

pytestmark = pytest.mark.gpu

F3 = inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _random_case(seed=0, dim=2):
    if dim == 2:
        p = inputs.config_random_field(2, (40, 24), levels=2, seed=seed, contrast=1e3, alpha=20.0, faces=F3,
                                       void_fraction=0.05)
    else:  # ragged 3D tiles (8 x 8 x 4 cells), obstacle cells, a do-nothing face
        p = inputs.config_random_field(3, (10, 8, 12), levels=2, seed=seed, contrast=1e3, alpha=20.0,
                                       faces=inputs.all_faces(3) & ~inputs.FACE_XP, void_fraction=0.05)
    m = mesh_from_problem(p)
    rng = np.random.default_rng(seed + 50)
    vcirc = 5.0 * rng.standard_normal(m.n_u)
    return p, m, vcirc, 50.0


def _scale(m, p, vcirc, rho, x_u):
    """Row scale of the corrector block: cellwise |A| |x| plus (|C| + |S|) |x| on free rows and columns."""
    ab = AbsOperators(m, p.eta, p.alpha)
    C, S = convection_matrices(m, vcirc, p.eta, rho)
    keep = sp.diags((~ab.u_constrained).astype(float))
    CS = keep @ (abs(C) + abs(S)) @ keep
    return ab.A @ np.abs(x_u) + CS @ np.abs(x_u), ab


def _rowerr(y, ref, scale):
    err = np.abs(np.asarray(y) - ref)
    z = scale == 0
    assert np.all(err[z] == 0.0)
    return float(np.max(err[~z] / scale[~z]))


@pytest.mark.parametrize("dim", [2, 3])
def test_corrector_operators_diag_and_bounds(dim):
    import torch
    from paper_2305_08986_gb300 import gs
    p, m, vcirc, rho = _random_case(dim=dim)
    cs = CorrectorSystem(m, p.eta, p.alpha, vcirc, rho)
    o = CorrectorOracle(m, p.eta, p.alpha, vcirc, rho, levels=p.levels)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(m.N)
    xu = x[:m.n_u]
    for prec in (64, 32):
        s = gs.Solver.from_problem(p, mg_precision=prec, corrector=1)
        s.set_corrector(vcirc, rho)
        xt = torch.tensor(xu, device="cuda")
        y = torch.empty_like(xt)
        s.vmult_A(xt, y)
        scale, ab = _scale(m, p, vcirc, rho, xu)
        assert _rowerr(y.cpu().numpy(), cs.A @ xu, scale) <= 1e-12
        x32 = xt.float()
        y32 = torch.empty_like(x32)
        s.vmult_A(x32, y32)
        xr = x32.double().cpu().numpy()
        scale32, _ = _scale(m, p, vcirc, rho, xr)
        assert _rowerr(y32.double().cpu().numpy(), cs.A @ xr, scale32) <= 1e-6
        # saddle operator K_c (FP64): velocity rows with the corrector block, B and B^T unchanged
        xk = torch.tensor(x, device="cuda")
        yk = torch.empty_like(xk)
        s.vmult(xk, yk)
        sK = np.concatenate([scale + abs(cs.B.T) @ np.abs(x[m.n_u:]), abs(cs.B) @ np.abs(xu)])
        sK[m.n_u:][cs.p_constrained] = np.abs(x[m.n_u:][cs.p_constrained])
        assert _rowerr(yk.cpu().numpy(), cs.K @ x, sK) <= 1e-12
        # per level: diag(A_c) and the Chebyshev bound of the symmetric part
        inf = s.info()
        for l, lv in enumerate(o.levels):
            d = torch.empty(lv["mesh"].n_u, dtype=torch.float64, device="cuda")
            s.apply_level(l, gs.OP_DIAG_A, None, d)
            assert np.max(np.abs(d.cpu().numpy() - lv["D"]) / np.abs(lv["D"])) <= 1e-13
            if l > 0 and prec == 64:  # FP64 Lanczos matches the oracle's; FP32 only to its precision
                assert abs(inf.lambda_max[l] - lv["lam"]) <= 1e-10 * lv["lam"], (prec, l)
        s.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_corrector_vcycle_fp64(dim):
    import torch
    from paper_2305_08986_gb300 import gs
    p, m, vcirc, rho = _random_case(seed=1, dim=dim)
    o = CorrectorOracle(m, p.eta, p.alpha, vcirc, rho, levels=p.levels)
    s = gs.Solver.from_problem(p, mg_precision=64, corrector=1)
    s.set_corrector(vcirc, rho)
    b = np.random.default_rng(4).standard_normal(m.n_u)
    z = torch.empty(m.n_u, dtype=torch.float64, device="cuda")
    s.vcycle(torch.tensor(b, device="cuda"), z)
    assert rel(z.cpu().numpy(), o.vcycle(b)) <= 1e-10


def _channel_case():
    p = inputs.config_channel(nx=160, ny=28, levels=3)
    m = mesh_from_problem(p)
    pred = StokesOracle(m, p.eta, p.alpha, 3)
    x0, _, _, _ = pred.solve(pred.sys.lift_rhs(p.f, p.g), tol=1e-10)
    return p, m, x0[:m.n_u], 1.0


@pytest.mark.parametrize("prec", [64, 32])
def test_corrector_solve_matches_the_direct_solution(prec):
    """Channel with the predictor solution as v° (rho = 1, alpha = 1e3): the non-symmetric system
    K_c x = b solved by FGMRES with the block-triangular preconditioner built on A_c."""
    import torch
    from paper_2305_08986_gb300 import gs
    p, m, vcirc, rho = _channel_case()
    o = CorrectorOracle(m, p.eta, p.alpha, vcirc, rho=rho, levels=p.levels)
    b = o.sys.lift_rhs(p.f, p.g)
    _, it_o, _, _ = o.solve(b, tol=1e-10)
    xd = spla.spsolve(o.sys.K.tocsc(), b)
    s = gs.Solver.from_problem(p, mg_precision=prec, corrector=1)
    s.set_corrector(vcirc, rho)
    f = torch.tensor(p.f, device="cuda")
    g = torch.tensor(p.g, device="cuda")
    bt = torch.empty_like(f)
    s.lift_rhs(f, g, bt)
    assert rel(bt.cpu().numpy(), b) <= 1e-12
    x = torch.zeros_like(bt)
    it, rr, st = s.solve(bt, x, tol=1e-10)
    assert st == 0 and rr <= 1e-10
    xg = x.cpu().numpy()
    assert np.linalg.norm(b - o.sys.K @ xg) <= 2e-10 * np.linalg.norm(b)
    assert rel(xg, xd) <= 1e-8, rel(xg, xd)
    if prec == 64:
        assert abs(it - it_o) <= max(2, 0.05 * it_o), (it, it_o)
    else:
        assert it <= it_o + max(3, 0.1 * it_o), (it, it_o)


def test_return_to_the_predictor_stage_is_bitwise():
    import torch
    from paper_2305_08986_gb300 import gs
    p, m, vcirc, rho = _channel_case()
    f = torch.tensor(p.f, device="cuda")
    g = torch.tensor(p.g, device="cuda")
    out = []
    for switch in (False, True):
        s = gs.Solver.from_problem(p, corrector=1)
        if switch:
            s.set_corrector(vcirc, rho)
            b = torch.empty_like(f)
            s.lift_rhs(f, g, b)
            x = torch.zeros_like(b)
            s.solve(b, x, tol=1e-8)
            s.set_corrector(None)
        b = torch.empty_like(f)
        s.lift_rhs(f, g, b)
        x = torch.zeros_like(b)
        it, rr, _ = s.solve(b, x, tol=1e-9)
        out.append((it, x.cpu()))
        s.close()
    assert out[0][0] == out[1][0] and torch.equal(out[0][1], out[1][1])


def test_corrector_rejects_unsupported_contexts():
    from paper_2305_08986_gb300 import gs
    p, m, vcirc, rho = _random_case()
    s = gs.Solver.from_problem(p)                       # created without the corrector fields
    with pytest.raises(gs.GsError):
        s.set_corrector(vcirc, rho)
    p3 = inputs.config_box_inclusion(3, (8, 8, 8), 2, 1e3, 5.0, seed=1)
    with pytest.raises(gs.GsError):
        gs.Solver.from_problem(p3, corrector=1, deflate=1)  # with deflation: not built
    s2 = gs.Solver.from_problem(p, corrector=1)
    bad = vcirc.copy()
    bad[3] = np.nan
    with pytest.raises(gs.GsError):
        s2.set_corrector(bad, rho)


def test_saddle_point_multigrid_in_the_corrector_stage_3d():
    """The block smoother K_j with ChebBiCGStab(1, 1) and one V-cycle of the saddle-point multigrid on
    a 3D corrector block (FP64) against MonolithicHierarchy(corrector=(v°, rho))."""
    import torch
    from oracle.monolithic import MonolithicHierarchy
    from paper_2305_08986_gb300 import gs
    p = inputs.config_box_inclusion(3, (8, 8, 8), 2, 1e3, 20.0, seed=2, faces=inputs.all_faces(3) & ~inputs.FACE_XP,
                                    align_coarse=True)
    m = mesh_from_problem(p)
    rng = np.random.default_rng(8)
    vcirc = 2.0 * rng.standard_normal(m.n_u)
    rho = 20.0
    h = MonolithicHierarchy(m, p.eta, p.alpha, p.levels, corrector=(vcirc, rho))
    s = gs.Solver.from_problem(p, precond_kind=1, mg_precision=64, corrector=1)
    s.set_corrector(vcirc, rho)
    L = p.levels - 1
    fl = h.levels[L]
    r = rng.standard_normal(fl.mesh.N)
    r[fl.sys.constrained] = 0.0
    rt = torch.tensor(r, device="cuda")
    y = torch.empty_like(rt)
    s.apply_level(L, gs.OP_SADDLE_SMOOTH, rt, y)
    assert rel(y.cpu().numpy(), h.smoother(L, r)) <= 1e-9
    s.apply_level(L, gs.OP_SADDLE_VCYCLE, rt, y)
    assert rel(y.cpu().numpy(), h.vcycle(r)) <= 1e-9


def test_saddle_point_multigrid_in_the_corrector_stage():
    """Sec. 4's own preconditioner with the corrector block: the block smoother K_j with
    Shat^{-1} = ChebBiCGStab(1, 1) and one V-cycle (FP64 multigrid) against
    MonolithicHierarchy(corrector=(v°, rho)); the preconditioned solve reaches the sparse direct
    solution of the non-symmetric system."""
    import torch
    from oracle.monolithic import MonolithicHierarchy
    from paper_2305_08986_gb300 import gs
    p = inputs.config_box_inclusion(2, (32, 16), 2, 1e3, 20.0, seed=2, faces=F3, align_coarse=True)
    m = mesh_from_problem(p)
    rng = np.random.default_rng(8)
    vcirc = 4.0 * rng.standard_normal(m.n_u)
    rho = 20.0
    h = MonolithicHierarchy(m, p.eta, p.alpha, p.levels, corrector=(vcirc, rho))
    s = gs.Solver.from_problem(p, precond_kind=1, mg_precision=64, corrector=1)
    s.set_corrector(vcirc, rho)
    L = p.levels - 1
    fl = h.levels[L]
    r = rng.standard_normal(fl.mesh.N)
    r[fl.sys.constrained] = 0.0
    rt = torch.tensor(r, device="cuda")
    y = torch.empty_like(rt)
    s.apply_level(L, gs.OP_SADDLE_SMOOTH, rt, y)
    assert rel(y.cpu().numpy(), h.smoother(L, r)) <= 1e-9
    s.apply_level(L, gs.OP_SADDLE_VCYCLE, rt, y)
    assert rel(y.cpu().numpy(), h.vcycle(r)) <= 1e-9
    cs = CorrectorSystem(m, p.eta, p.alpha, vcirc, rho)
    b = cs.lift_rhs(p.f, p.g)
    xd = spla.spsolve(cs.K.tocsc(), b)
    x = torch.zeros(m.N, dtype=torch.float64, device="cuda")
    it, rr, st = s.solve(torch.tensor(b, device="cuda"), x, tol=1e-10)
    assert st == 0 and rr <= 1e-10 and it < 60, it
    assert rel(x.cpu().numpy(), xd) <= 1e-8


@pytest.mark.parametrize("prec", [64, 32])
def test_corrector_solve_3d_matches_the_direct_solution(prec):
    """3D box inclusion with a random v° (rho = 20: the streamline term is active in most cells):
    FGMRES with the block-triangular preconditioner on the 3D corrector block reaches the sparse
    direct solution of the non-symmetric system; FP64 multigrid within the oracle's iteration count.
    This system is far from symmetric (contrast 1e3, rho |v°| h / eta up to ~10): at rel-res 1e-10 even
    the oracle's FGMRES stays 5e-8 from the direct solution, so the solves run to rel-res 1e-12."""
    import torch
    from paper_2305_08986_gb300 import gs
    p = inputs.config_box_inclusion(3, (8, 8, 8), 2, 1e3, 20.0, seed=4, faces=inputs.all_faces(3) & ~inputs.FACE_ZP,
                                    align_coarse=True)
    m = mesh_from_problem(p)
    vcirc = 3.0 * np.random.default_rng(9).standard_normal(m.n_u)
    rho = 20.0
    o = CorrectorOracle(m, p.eta, p.alpha, vcirc, rho=rho, levels=p.levels)
    b = o.sys.lift_rhs(p.f, p.g)
    _, it_o, _, _ = o.solve(b, tol=1e-12)
    xd = spla.spsolve(o.sys.K.tocsc(), b)
    s = gs.Solver.from_problem(p, mg_precision=prec, corrector=1)
    s.set_corrector(vcirc, rho)
    x = torch.zeros(m.N, dtype=torch.float64, device="cuda")
    it, rr, st = s.solve(torch.tensor(b, device="cuda"), x, tol=1e-12)
    assert st == 0 and rr <= 1e-12
    xg = x.cpu().numpy()
    assert np.linalg.norm(b - o.sys.K @ xg) <= 2e-12 * np.linalg.norm(b)
    assert rel(xg, xd) <= 1e-8, rel(xg, xd)
    if prec == 64:
        assert abs(it - it_o) <= max(2, 0.05 * it_o), (it, it_o)
    else:
        assert it <= it_o + max(3, 0.1 * it_o), (it, it_o)
