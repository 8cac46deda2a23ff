"""The allocation-free coarse solve (gs_coarse_solve_noalloc) against the regular coarse solve.

Callers that cannot allocate device memory where they call the coarse solve (inside a graph
capture or a latency-critical loop) use the entry point whose scratch is a static device
array; it must return what gs_apply_level(..., GS_OP_COARSE, ...) returns.  Two calls in a
row with different right-hand sides check that the shared array's leftover contents from
the previous call never leak into the next result.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2305_08986_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [lambda: inputs.config_disc(n=16, levels=3),
                                  lambda: inputs.config_box_inclusion(3, (8, 8, 8), 2, 1e4, 50.0, seed=3)])
def test_noalloc_coarse_solve_matches_regular(make):
    import torch
    from paper_2305_08986_gb300 import build
    build.build(verbose=False)
    from paper_2305_08986_gb300 import gs

    p = make()
    s = gs.Solver.from_problem(p)
    inf = s.info()
    n0 = inf.level_n_u[0]
    assert 0 < inf.coarse_free <= 16384
    rng = np.random.default_rng(11)
    for call in range(2):
        b = torch.tensor(rng.standard_normal(n0), device="cuda")
        y_ref = torch.full((n0,), np.nan, dtype=torch.float64, device="cuda")
        y_new = torch.full((n0,), np.nan, dtype=torch.float64, device="cuda")
        s.apply_level(0, gs.OP_COARSE, b, y_ref, prec=64)
        st = gs._lib.gs_coarse_solve_noalloc(s.ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(y_new.data_ptr()))
        assert st == gs.GS_OK, gs._lib.gs_last_error()
        torch.cuda.synchronize()
        a, r = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - r) <= 1e-12 * np.linalg.norm(r), call
    s.close()


def test_noalloc_coarse_solve_rejects_bad_contexts():
    import torch
    from paper_2305_08986_gb300 import gs

    p = inputs.config_channel(nx=160, ny=28, levels=1)
    s = gs.Solver.from_problem(p, coarse_mode=1)   # no dense coarse solve in this context
    b = torch.zeros(s.n_u, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(b)
    st = gs._lib.gs_coarse_solve_noalloc(s.ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(y.data_ptr()))
    assert st == gs.GS_EINVAL
    assert gs._lib.gs_coarse_solve_noalloc(s.ctx, None, ctypes.c_void_p(y.data_ptr())) == gs.GS_EINVAL
    s.close()


def test_noalloc_coarse_solve_rejects_a_coarse_level_above_the_limit():
    """46 x 46 cells, every face Dirichlet, one level: 2 x 91^2 = 16,562 free coarse unknowns, just
    above the 16,384 entries of the static array; the call must refuse instead of overrunning it."""
    import torch
    from paper_2305_08986_gb300 import gs

    p = inputs.config_random_field(2, (46, 46), levels=1, seed=2, contrast=10.0, alpha=1.0)
    s = gs.Solver.from_problem(p)
    inf = s.info()
    assert inf.coarse_free == 2 * 91 * 91 > 16384
    b = torch.zeros(s.n_u, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(b)
    st = gs._lib.gs_coarse_solve_noalloc(s.ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(y.data_ptr()))
    assert st == gs.GS_EINVAL
    assert b"at most 16384" in gs._lib.gs_last_error()
    s.close()
