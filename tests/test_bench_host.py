"""Host-side pieces of bench.py: the algorithmic byte / FMA model of the Gram-Schmidt kernels and
the level-weighted roofline of the tile kernels."""
import pytest


def test_krylov_bytes_closed_form():
    import bench
    n, K = 1000, 7
    dots, axpy, fd, fa = bench.krylov_bytes(n, K, restart=50, form="explicit")
    # iteration k orthogonalises against k + 1 rows: the first pass reads them and w once
    assert dots == sum((k + 2) * n * 8 for k in range(K)) == n * 8 * (K * (K + 1) // 2 + K)
    # two update passes (rows + w read + w written) and the new basis vector (w read, v written)
    assert axpy == sum(2 * (k + 3) * n * 8 + 2 * n * 8 for k in range(K))
    # FMAs: one per row entry for the dots, two for the fused update + dots, one (+ the norm) last
    assert fd == sum((k + 1) * n for k in range(K))
    assert fa == sum((3 * (k + 1) + 1) * n for k in range(K))


def test_krylov_bytes_gram_form():
    import bench
    n, K = 1000, 7
    dots, axpy, fd, fa = bench.krylov_bytes(n, K, restart=50)
    # one dot pass (rows + w) with two dots per row entry, one update pass (rows + w read + w written)
    assert dots == sum((k + 2) * n * 8 for k in range(K))
    assert axpy == sum((k + 3) * n * 8 + 2 * n * 8 for k in range(K))
    assert fd == sum(2 * (k + 1) * n for k in range(K))
    assert fa == sum((k + 2) * n for k in range(K))
    # 3 instead of 4 FMAs per basis entry (plus the norm)
    e = bench.krylov_bytes(n, K, restart=50, form="explicit")
    assert fd + fa - K * n == pytest.approx(0.75 * (e[2] + e[3] - K * n))


def test_krylov_bytes_restart_resets_the_row_count():
    import bench
    a = bench.krylov_bytes(100, 10, restart=5)
    b = bench.krylov_bytes(100, 5, restart=5)
    assert a == tuple(2 * v for v in b)


def test_krylov_rooflines_skip_missing_classes():
    import bench
    out = bench.krylov_rooflines({"gram_schmidt_dots": (10, 2.0)}, 1000, 3, 50, 1000.0, 1.0)
    assert set(out) == {"gram_schmidt_dots"}
    r = out["gram_schmidt_dots"]
    assert r["achieved_gbs"] == pytest.approx(r["algorithmic_bytes"] / 2e-3 / 1e9)
    assert r["frac_hbm"] == pytest.approx(r["achieved_gbs"] / 1000.0)
    assert r["achieved_fp64_tflops"] == pytest.approx(2 * r["fp64_fma"] / 2e-3 / 1e12)


def test_level_weighted_roofline_by_hand():
    """sum_l bytes_l x launches_l / sum_l time_l, with the byte model of the fused Chebyshev step
    (six vectors of d N_v FP32 entries plus eta per cell) on the levels of a 2-level 2D mesh."""
    import bench
    sizes = bench.level_sizes(2, (8, 4), 2)
    assert sizes == [(2 * 9 * 5, 8), (2 * 17 * 9, 32)]
    per_level = {-1: {}, 0: {"cheb_step": (3, 0.003)}, 1: {"cheb_step": (3, 0.006)}}
    r = bench.level_weighted_roofline(per_level, sizes, "cheb_step", 4, 100.0)
    b0 = 6 * 90 * 4 + 8 * 4
    b1 = 6 * 306 * 4 + 32 * 4
    assert r["launches"] == 6
    assert r["achieved"] == pytest.approx((3 * b0 + 3 * b1) / 0.009e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 100.0)
    assert [x["level"] for x in r["per_level"]] == [0, 1]
