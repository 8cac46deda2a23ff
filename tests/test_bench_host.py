"""Host-side pieces of bench.py: the algorithmic byte model of the Gram-Schmidt kernels."""
import pytest


def test_krylov_bytes_closed_form():
    import bench
    n, K = 1000, 7
    dots, axpy = bench.krylov_bytes(n, K, restart=50)
    # iteration k orthogonalises against k + 1 rows: the first pass reads them and w once
    assert dots == sum((k + 2) * n * 8 for k in range(K)) == n * 8 * (K * (K + 1) // 2 + K)
    # two update passes (rows + w read + w written) and the new basis vector (w read, two writes)
    assert axpy == sum(2 * (k + 3) * n * 8 + 3 * n * 8 for k in range(K))


def test_krylov_bytes_restart_resets_the_row_count():
    import bench
    a = bench.krylov_bytes(100, 10, restart=5)
    b = bench.krylov_bytes(100, 5, restart=5)
    assert a == (2 * b[0], 2 * b[1])


def test_krylov_rooflines_skip_missing_classes():
    import bench
    out = bench.krylov_rooflines({"gram_schmidt_dots": (10, 2.0)}, 1000, 3, 50, 1000.0)
    assert set(out) == {"gram_schmidt_dots"}
    r = out["gram_schmidt_dots"]
    assert r["achieved_gbs"] == pytest.approx(r["algorithmic_bytes"] / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved_gbs"] / 1000.0)
