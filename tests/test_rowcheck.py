"""The per-row parity measure (tests/rowcheck.py) on the CPU: it sees what a norm-wise check misses.

A mistake is planted in the oracle: the viscosity of the low-eta (fluid) cells is perturbed by
a relative 1e-7, as an FP32 rounding of eta leaking into an FP64 path would do.  On a random
field of contrast 1e6 the norm-wise relative difference stays below 1e-12 (the stiff rows set
the norm) while the per-row measure reports ~1e-7, so the GPU operator tests, which gate on the
per-row measure at 1e-12 (FP64), would fail on such a kernel.
"""
import numpy as np
import pytest

from oracle.fem import System
from oracle.mesh import mesh_from_problem
from paper_2305_08986_gb300 import inputs
from tests.rowcheck import AbsOperators, abs_rows, row_error, sampled_row_error


def _case(dim, n, seed=0, void=0.05):
    p = inputs.config_random_field(dim, n, levels=1, seed=seed, contrast=1e6, alpha=7.0, void_fraction=void,
                                   faces=inputs.FACE_XM | inputs.FACE_YM)
    return p, mesh_from_problem(p)


@pytest.mark.parametrize("dim,n", [(2, (12, 10)), (3, (4, 3, 5))])
def test_planted_low_eta_error_is_caught_per_row_not_norm_wise(dim, n):
    p, m = _case(dim, n)
    ref = System(m, p.eta, p.alpha)
    low = p.eta < 10.0
    assert low.any() and (~low).any() and p.eta.max() / p.eta.min() > 1e5
    bad = System(m, np.where(low, p.eta * (1.0 + 1e-7), p.eta), p.alpha)
    ab = AbsOperators(m, p.eta, p.alpha)
    x = np.random.default_rng(3).standard_normal(m.N)
    # velocity block
    y_ref, y_bad = ref.A @ x[:m.n_u], bad.A @ x[:m.n_u]
    assert np.linalg.norm(y_bad - y_ref) / np.linalg.norm(y_ref) < 1e-12      # norm-wise: blind
    assert row_error(y_bad, y_ref, ab.A, x[:m.n_u]) > 1e-8                      # per row: caught
    assert row_error(y_ref, y_ref, ab.A, x[:m.n_u]) == 0.0
    # full saddle operator
    assert np.linalg.norm(bad.K @ x - ref.K @ x) / np.linalg.norm(ref.K @ x) < 1e-12
    assert row_error(bad.K @ x, ref.K @ x, ab.K, x) > 1e-8


def test_scale_dominates_assembled_absolute_and_sampled_rows_agree():
    p, m = _case(2, (9, 7), seed=1)
    ref = System(m, p.eta, p.alpha)
    ab = AbsOperators(m, p.eta, p.alpha)
    x = np.random.default_rng(4).standard_normal(m.n_u)
    s = ab.A @ np.abs(x)
    A_abs = abs(ref.A)
    assert np.all(s >= A_abs @ np.abs(x) * (1 - 1e-14))   # cellwise sum >= assembled |A| |x|
    rows = np.random.default_rng(5).choice(m.n_u, 60, replace=False)
    assert np.allclose(abs_rows(m, p.eta, p.alpha, x, rows), s[rows], rtol=1e-13, atol=0)
    y = ref.A @ x
    assert sampled_row_error(y[rows], y[rows], s[rows]) == 0.0
    # an error of one unit roundoff of the scale in one row reads as ~1e-16
    yb = y.copy()
    yb[rows[0]] += 1e-16 * s[rows[0]]
    assert 5e-17 < row_error(yb, y, ab.A, x) < 2e-16
