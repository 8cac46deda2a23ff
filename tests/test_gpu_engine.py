"""Batching engine on the GPU (gs_engine_*, gs_batch_solve).

Each solve in the engine runs the launches gs_solve issues for it, merged with the other solves'
launches through the batched kernel entry points.  Alone in the engine or in a mix (2D and 3D,
different sizes, levels and options, joining at any step) its iterate, iteration count and
residual are bitwise the same.  Against gs_solve -- the same kernel bodies compiled into the
single-instance entry points, where the compiler may contract multiply-adds differently -- the
solutions agree to the solver tolerance and the iteration counts within max(2, 5 %).  One batched
solve is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

from paper_2305_08986_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _problems():
    return [
        inputs.config_disc(n=16, levels=3),
        inputs.config_channel(nx=160, ny=28, levels=3),
        inputs.config_box_inclusion(3, (8, 8, 8), 2, 1e4, 50.0, seed=3),
        inputs.config_box_inclusion(2, (32, 32), inputs.levels_for(32, 2), 1e5, 300.0, seed=5),
        inputs.config_box_inclusion(3, (16, 16, 16), inputs.levels_for(16, 3), 1e3, 10.0, seed=6),
        inputs.config_random_field(2, (48, 32), levels=3, seed=8, contrast=1e3, alpha=20.0,
                                   faces=inputs.FACE_XM | inputs.FACE_YM | inputs.FACE_YP, void_fraction=0.03),
    ]


def _setup(p, **opts):
    import torch
    from paper_2305_08986_gb300 import gs
    s = gs.Solver.from_problem(p, **opts)
    f = torch.tensor(p.f, device="cuda")
    g = torch.tensor(p.g, device="cuda")
    b = torch.empty_like(f)
    s.lift_rhs(f, g, b)
    x = torch.zeros_like(b)
    return s, b, x


def _alone(p, **opts):
    s, b, x = _setup(p, **opts)
    it, rr, st = s.solve(b, x, tol=TOL, allow_noconv=True)
    return x.cpu(), it, rr, st


def _engine_alone(p, **opts):
    from paper_2305_08986_gb300 import gs
    s, b, x = _setup(p, **opts)
    eng = gs.Engine(1)
    assert eng.add(s, b, x, TOL)
    r = eng.run()[0]
    return x.cpu(), r["iterations"], r["rel_residual"], r["status"]


def _same(ref, x, it, rr, st):
    import torch
    xr, itr, rrr, str_ = ref
    assert st == str_ and it == itr and rr == rrr, ((st, it, rr), (str_, itr, rrr))
    assert torch.equal(x.cpu(), xr)


def _close(ref, x, it, rr, st):
    import torch
    xr, itr, rrr, str_ = ref
    assert st == str_ == 0 and rr <= TOL and rrr <= TOL
    assert abs(it - itr) <= max(2, 0.05 * itr), (it, itr)
    xc = x.cpu()
    # both stop at rel-res <= TOL; the difference of the iterates is bounded by the conditioning
    assert torch.linalg.norm(xc - xr) <= 1e-6 * torch.linalg.norm(xr)


@pytest.mark.parametrize("k", [0, 2])
def test_engine_single_solve_matches_gs_solve(k):
    from paper_2305_08986_gb300 import gs
    p = _problems()[k]
    ref = _alone(p)
    s, b, x = _setup(p)
    eng = gs.Engine(1)
    assert eng.add(s, b, x, TOL, tag=7)
    res = eng.run()
    assert len(res) == 1 and res[0]["tag"] == 7
    r = res[0]
    _close(ref, x, r["iterations"], r["rel_residual"], r["status"])
    assert r["t_done"] >= r["t_added"]
    # deterministic: the same solve again gives the same bits
    _same(_engine_alone(p), x, r["iterations"], r["rel_residual"], r["status"])
    st = eng.stats()
    assert st["steps"] >= r["iterations"] and st["plan_builds"] >= 1 and st["plan_kernels"] > 0


def test_engine_mix_alone_vs_in_the_mix():
    """2D and 3D solves of different sizes and level counts, all in one engine."""
    from paper_2305_08986_gb300 import gs
    probs = _problems()
    refs = [_engine_alone(p) for p in probs]
    solo = [_alone(p) for p in probs]
    setups = [_setup(p) for p in probs]
    eng = gs.Engine(len(probs))
    for i, (s, b, x) in enumerate(setups):
        assert eng.add(s, b, x, TOL, tag=i)
    res = {r["tag"]: r for r in eng.run()}
    assert sorted(res) == list(range(len(probs)))
    for i, (s, b, x) in enumerate(setups):
        r = res[i]
        _same(refs[i], x, r["iterations"], r["rel_residual"], r["status"])
        assert r["status"] == gs.GS_OK
        _close(solo[i], x, r["iterations"], r["rel_residual"], r["status"])


def test_engine_continuous_joining():
    """Three slots for six solves: the others join as slots free up (plan rebuilt on joins)."""
    from paper_2305_08986_gb300 import gs
    probs = _problems()
    refs = [_engine_alone(p) for p in probs]
    setups = [_setup(p) for p in probs]
    eng = gs.Engine(3)
    pending = list(range(len(probs)))
    done = {}
    while pending and eng.add(*setups[pending[0]], TOL, tag=pending[0]):
        pending.pop(0)
    assert len(pending) == 3
    s, b, x = setups[pending[0]]
    assert not eng.add(s, b, x, TOL, tag=99)  # full: GS_EBUSY
    steps = 0
    while eng.active() > 0 or pending:
        eng.step()
        steps += 1
        for r in eng.poll():
            done[r["tag"]] = r
        while pending and eng.add(*setups[pending[0]], TOL, tag=pending[0]):
            pending.pop(0)
        assert steps < 5000
    assert sorted(done) == list(range(len(probs)))
    for i, (s, b, x) in enumerate(setups):
        r = done[i]
        _same(refs[i], x, r["iterations"], r["rel_residual"], r["status"])
    assert eng.stats()["plan_builds"] >= 2


def test_engine_options_in_one_batch():
    """FP64 multigrid, the FP64 Krylov basis and the mass-only Schur term next to the defaults."""
    from paper_2305_08986_gb300 import gs
    probs = _problems()[:3]
    opts = [dict(mg_precision=64), dict(krylov_fp64=2), dict(schur_kind=1, max_iter=3000)]
    refs = [_engine_alone(p, **o) for p, o in zip(probs, opts)]
    setups = [_setup(p, **o) for p, o in zip(probs, opts)]
    eng = gs.Engine(4)
    for i, (s, b, x) in enumerate(setups):
        assert eng.add(s, b, x, TOL, tag=i)
    res = {r["tag"]: r for r in eng.run()}
    for i, (s, b, x) in enumerate(setups):
        _same(refs[i], x, res[i]["iterations"], res[i]["rel_residual"], res[i]["status"])


@pytest.mark.parametrize("orth", [3, 2])
def test_engine_gram_schmidt_forms(orth):
    """The explicit CGS2 (orth = 3) and the Gram-matrix form (orth = 2, the default) in the engine:
    a 2D and a 3D solve, alone and together, give the same bits, and agree with gs_solve to the
    solver tolerance."""
    from paper_2305_08986_gb300 import gs
    probs = [_problems()[1], _problems()[2]]
    refs = [_engine_alone(p, orth=orth) for p in probs]
    setups = [_setup(p, orth=orth) for p in probs]
    eng = gs.Engine(2)
    for i, (s, b, x) in enumerate(setups):
        assert eng.add(s, b, x, TOL, tag=i)
    res = {r["tag"]: r for r in eng.run()}
    for i, (s, b, x) in enumerate(setups):
        _same(refs[i], x, res[i]["iterations"], res[i]["rel_residual"], res[i]["status"])
        xa, ita, rra, sta = _alone(probs[i], orth=orth)
        _close((xa, ita, rra, sta), x, res[i]["iterations"], res[i]["rel_residual"], res[i]["status"])


def test_engine_rejects_selective_reorthogonalisation():
    from paper_2305_08986_gb300 import gs
    s, b, x = _setup(_problems()[0], orth=1)
    eng = gs.Engine(2)
    with pytest.raises(gs.GsError):
        eng.add(s, b, x, TOL)


def test_batch_solve_matches_engine_and_oracle():
    from oracle.krylov import StokesOracle, normalize_pressure
    from oracle.mesh import mesh_from_problem
    from paper_2305_08986_gb300 import gs
    probs = _problems()[:4]
    refs = [_engine_alone(p) for p in probs]
    setups = [_setup(p) for p in probs]
    st, its, rels = gs.batch_solve([s for s, _, _ in setups], [b for _, b, _ in setups], [x for _, _, x in setups],
                                   tol=TOL)
    assert st == gs.GS_OK
    for i, (s, b, x) in enumerate(setups):
        _same(refs[i], x, its[i], rels[i], gs.GS_OK)
    p = probs[0]
    m = mesh_from_problem(p)
    o = StokesOracle(m, p.eta, p.alpha, p.levels)
    b_ref = o.sys.lift_rhs(p.f, p.g)
    xo, _, _, _ = o.solve(b_ref, tol=1e-11)
    xg = normalize_pressure(m, o.sys, setups[0][2].cpu().numpy())
    xo = normalize_pressure(m, o.sys, xo)
    assert np.linalg.norm(xg - xo) <= 1e-7 * np.linalg.norm(xo)


def test_engine_recycled_contexts():
    """Short solves come and go through one slot while a long one keeps the plan alive; a new
    context may live at a destroyed one's address and must never run the old one's launches."""
    from paper_2305_08986_gb300 import gs
    probs = _problems()
    long_p, short_p = probs[1], probs[0]
    ref_short = _engine_alone(short_p)
    sl, bl, xl = _setup(long_p)
    eng = gs.Engine(2)
    assert eng.add(sl, bl, xl, 1e-13, tag=100)  # runs past the short ones (stops at max_iter or 1e-13)
    for k in range(4):
        s, b, x = _setup(short_p)
        assert eng.add(s, b, x, TOL, tag=k)
        res = []
        while not res:
            eng.step()
            res = [r for r in eng.poll() if r["tag"] == k]
        _same(ref_short, x, res[0]["iterations"], res[0]["rel_residual"], res[0]["status"])
        s.close()
        del s, b, x
    eng.run()
