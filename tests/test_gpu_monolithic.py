"""GPU parity of the saddle-point multigrid of Sec. 4 (precond_kind = 1) against the FP64 oracle
(oracle/monolithic.py), through the C ABI.

Operators (FP64 multigrid): the Schur diagonal diag(B diag(A)^{-1} B^T) per level (1e-12 entry by
entry, a sum of a few hundred non-negative products), the block smoother K_j, the dense coarse saddle solve and one
V-cycle (1e-9 norm-wise: Chebyshev recurrences and one MINRES step, whose step length a is a
ratio of two inner products and so carries their rounding).  Solves: FP64-multigrid iteration
counts within max(2, 5 %) of the oracle's (the same algorithm; counts drift only through
rounding order), solutions against the sparse direct solution; FP32 multigrid converges to the
same tolerance.  The batching engine runs monolithic solves bitwise as it runs them alone.
"""
import numpy as np
import pytest

from oracle.krylov import StokesOracle, direct_solve, normalize_pressure
from oracle.mesh import mesh_from_problem
from oracle.monolithic import MonolithicHierarchy
from paper_2305_08986_gb300 import inputs

pytestmark = pytest.mark.gpu

F3 = inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP
OP_CASES = [
    dict(dim=2, n=(40, 24), levels=3, void=0.0, faces=None),       # several 2D tiles, ragged
    dict(dim=2, n=(72, 20), levels=2, void=0.08, faces=F3),        # obstacle cells, do-nothing face
    dict(dim=3, n=(12, 8, 8), levels=2, void=0.0, faces=None),     # ragged 3D tiles
    dict(dim=3, n=(8, 8, 4), levels=2, void=0.1, faces=inputs.FACE_ZM | inputs.FACE_XP),
]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _problem(case, seed=0):
    return inputs.config_random_field(case["dim"], case["n"], levels=case["levels"], seed=seed, contrast=1e3,
                                      alpha=7.0, faces=case["faces"], void_fraction=case["void"])


def _solver(p, **opts):
    from paper_2305_08986_gb300 import gs
    return gs.Solver.from_problem(p, precond_kind=1, **opts)


@pytest.mark.parametrize("case", OP_CASES)
def test_schur_diagonal_per_level(case):
    import torch
    p = _problem(case)
    s = _solver(p, mg_precision=64)
    h = MonolithicHierarchy(mesh_from_problem(p), p.eta, p.alpha, p.levels)
    assert s.info().precond_kind == 1
    for l, lv in enumerate(h.levels):
        y = torch.empty(lv.mesh.Np, dtype=torch.float64, device="cuda")
        s.apply_level(l, 17, torch.zeros(1, dtype=torch.float64, device="cuda"), y)
        # entry by entry (a sum of non-negative products: no cancellation)
        nz = lv.ds != 0.0
        assert np.max(np.abs(y.cpu().numpy()[nz] - lv.ds[nz]) / lv.ds[nz]) <= 1e-12
        assert np.all(y.cpu().numpy()[lv.sys.p_constrained] == 0.0)


@pytest.mark.parametrize("case", OP_CASES)
def test_block_smoother_coarse_solve_and_vcycle(case):
    import torch
    p = _problem(case, seed=1)
    s = _solver(p, mg_precision=64)
    m = mesh_from_problem(p)
    h = MonolithicHierarchy(m, p.eta, p.alpha, p.levels)
    rng = np.random.default_rng(2)
    L = p.levels - 1
    fl = h.levels[L]
    r = rng.standard_normal(fl.mesh.N)
    r[fl.sys.constrained] = 0.0
    rt = torch.tensor(r, device="cuda")
    y = torch.empty_like(rt)
    s.apply_level(L, 18, rt, y)                      # K_j r
    assert rel(y.cpu().numpy(), h.smoother(L, r)) <= 1e-9
    s.apply_level(L, 19, rt, y)                      # V_L(r)
    assert rel(y.cpu().numpy(), h.vcycle(r)) <= 1e-9
    c0 = h.levels[0]
    free = ~c0.sys.constrained
    b0 = rng.standard_normal(c0.mesh.N)
    b0[~free] = 0.0
    if h.nullspace:  # consistent right-hand side (orthogonal to the constant pressure)
        pf = free[c0.n_u:]
        b0[c0.n_u:][pf] -= b0[c0.n_u:][pf].mean()
    y0 = torch.empty(c0.mesh.N, dtype=torch.float64, device="cuda")
    s.apply_level(0, 20, torch.tensor(b0, device="cuda"), y0)
    y0 = y0.cpu().numpy()
    # Gauss-Jordan without pivoting (device) against pivoted LU (oracle): both to ~cond(M_0) eps
    assert rel(y0, h.coarse_solve(b0)) <= 1e-9
    assert np.linalg.norm((c0.K @ y0)[free] - b0[free]) <= 1e-9 * np.linalg.norm(b0)
    assert s.info().saddle_coarse_free == int((~c0.sys.constrained).sum())


def _solve_cases():
    return [
        ("box2d", inputs.config_box_inclusion(2, (32, 32), 3, 1e6, 30.0, seed=5, align_coarse=True), 1e-9),
        ("box2d_open", inputs.config_box_inclusion(2, (64, 32), 3, 1e6, 30.0, seed=7, faces=F3, align_coarse=True),
         1e-9),
        ("rf2d", inputs.config_random_field(2, (48, 40), levels=3, seed=9, contrast=1e3, alpha=30.0, faces=F3,
                                            void_fraction=0.04), 1e-10),
        ("box3d", inputs.config_box_inclusion(3, (8, 8, 8), 2, 1e6, 30.0, seed=5, align_coarse=True), 1e-9),
    ]


def _fluid_pressure_nodes(m, p):
    """Pressure nodes touched by no stiff cell (eta >= sqrt(eta_min eta_max) when the contrast is
    at least 1e3)."""
    eta = np.asarray(p.eta)
    touch = np.zeros(m.Np, bool)
    if eta.max() >= 1e3 * eta.min():
        stiff = eta >= np.sqrt(eta.max() * eta.min())
        stiff[np.setdiff1d(np.arange(len(eta)), m.active_cells())] = False
        touch[m.cell_pnodes()[stiff].ravel()] = True
    return ~touch


def _consistent_rhs(m, sysm, p):
    b = sysm.lift_rhs(p.f, p.g)
    if m.has_pressure_nullspace():
        free = ~sysm.p_constrained
        b[m.n_u:][free] -= b[m.n_u:][free].mean()
    return b


@pytest.mark.parametrize("k", range(4))
def test_monolithic_solve_matches_oracle(k):
    import torch
    name, p, tol = _solve_cases()[k]
    m = mesh_from_problem(p)
    o = StokesOracle(m, p.eta, p.alpha, p.levels, precond="monolithic")
    b = _consistent_rhs(m, o.sys, p)
    _, it_o, rel_o, _ = o.solve(b, tol=tol, max_iter=300)
    assert rel_o <= tol
    xd = normalize_pressure(m, o.sys, direct_solve(o.sys, b))
    n_u = m.n_u
    bt = torch.tensor(b, device="cuda")
    for prec in (64, 32):
        s = _solver(p, mg_precision=prec)
        x = torch.zeros_like(bt)
        it, rr, st = s.solve(bt, x, tol=tol)
        assert st == 0 and rr <= tol, (name, prec, it, rr)
        if prec == 64:
            assert abs(it - it_o) <= max(2, 0.05 * it_o), (name, it, it_o)
        else:
            assert it <= it_o + max(3, 0.1 * it_o), (name, it, it_o)
        xg = normalize_pressure(m, o.sys, x.cpu().numpy())
        assert rel(xg[:n_u], xd[:n_u]) <= 1e-6, (name, prec)
        # the pressure inside an eta = 1e6 inclusion is a Schur-complement mode of eigenvalue
        # ~1/eta: a residual of 1e-9 pins it only to a few 1e-2 (the direct solve has the same
        # sensitivity); the pressure on nodes outside the stiff cells is pinned tightly
        fm = _fluid_pressure_nodes(m, p) & ~o.sys.p_constrained
        pg, pd = xg[n_u:][fm], xd[n_u:][fm]
        assert rel(pg - pg.mean(), pd - pd.mean()) <= 1e-5, (name, prec)
        assert rel(xg[n_u:], xd[n_u:]) <= (1e-1 if name.startswith("box") else 1e-6), (name, prec)


def test_monolithic_options_cycles_and_chebyshev_coarse():
    import torch
    _, p, tol = _solve_cases()[1]
    m = mesh_from_problem(p)
    from oracle.fem import System
    sysm = System(m, p.eta, p.alpha)
    bt = torch.tensor(_consistent_rhs(m, sysm, p), device="cuda")
    its = {}
    for key, opts in {"n1": {}, "n2": dict(mono_cycles=2), "m1": dict(mono_smooth=1),
                      "cheb0": dict(coarse_mode=1)}.items():
        s = _solver(p, mg_precision=64, **opts)
        x = torch.zeros_like(bt)
        it, rr, st = s.solve(bt, x, tol=tol, allow_noconv=True)
        assert st == 0 and rr <= tol, (key, it, rr)
        its[key] = it
    assert its["n2"] <= its["n1"], its


def test_monolithic_in_the_engine():
    """Monolithic and block-triangular solves in one engine: each bitwise as it runs alone."""
    import torch
    from oracle.fem import System
    from paper_2305_08986_gb300 import gs
    cases = _solve_cases()
    runs = [(cases[1][1], 1), (cases[2][1], 1), (cases[1][1], 0)]

    def setup(p, kind):
        s = gs.Solver.from_problem(p, precond_kind=kind)
        m = mesh_from_problem(p)
        b = torch.tensor(_consistent_rhs(m, System(m, p.eta, p.alpha), p), device="cuda")
        return s, b, torch.zeros_like(b), m.n_u

    alone = []
    for p, kd in runs:
        s, b, x, n_u = setup(p, kd)
        eng = gs.Engine(1)
        assert eng.add(s, b, x, 1e-9)
        r = eng.run()[0]
        assert r["status"] == 0, r
        alone.append((x.cpu(), r["iterations"], r["rel_residual"], r["status"]))
        xs = torch.zeros_like(b)
        it, rr, st = s.solve(b, xs, tol=1e-9)
        assert abs(it - r["iterations"]) <= max(2, 0.05 * it)
        xs, xe = xs.cpu()[:n_u], x.cpu()[:n_u]
        assert torch.linalg.norm(xs - xe) <= 1e-6 * torch.linalg.norm(xs)
    setups = [setup(p, kd) for p, kd in runs]
    eng = gs.Engine(len(runs))
    for i, (s, b, x, _) in enumerate(setups):
        assert eng.add(s, b, x, 1e-9, tag=i)
    res = {r["tag"]: r for r in eng.run()}
    for i, (s, b, x, _) in enumerate(setups):
        xr, itr, rrr, st = alone[i]
        assert res[i]["status"] == st == 0
        assert res[i]["iterations"] == itr and res[i]["rel_residual"] == rrr
        assert torch.equal(x.cpu(), xr)


def test_monolithic_rejects_deflation_and_block_contexts_reject_saddle_ops():
    import torch
    from paper_2305_08986_gb300 import gs
    p = _problem(OP_CASES[0])
    with pytest.raises(gs.GsError):
        gs.Solver.from_problem(p, precond_kind=1, deflate=1)
    s = gs.Solver.from_problem(p)
    y = torch.empty(10, dtype=torch.float32, device="cuda")
    with pytest.raises(gs.GsError):
        s.apply_level(p.levels - 1, 18, y, y)
