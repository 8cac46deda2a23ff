"""Host logic of the serving loop (no GPU): footprint accounting and latency statistics."""
from paper_2305_08986_gb300 import inputs


def test_request_footprint_grows_with_the_mesh():
    from paper_2305_08986_gb300 import serving
    a = serving.request_footprint(inputs.config_box_inclusion(2, (32, 32), 3, 1e3, 1.0, seed=0))
    b = serving.request_footprint(inputs.config_box_inclusion(2, (64, 64), 4, 1e3, 1.0, seed=0))
    c = serving.request_footprint(inputs.config_box_inclusion(3, (16, 16, 16), 3, 1e3, 1.0, seed=0))
    assert 0 < a < b and a < c
    # the Krylov basis alone (2 m + 1 full vectors of doubles) is a lower bound
    p = inputs.config_box_inclusion(2, (64, 64), 4, 1e3, 1.0, seed=0)
    assert b > 101 * 8 * len(p.f)


def test_summarize_percentiles():
    from paper_2305_08986_gb300 import serving
    rs = [serving.Result(i, 0, 10, 1e-9, 0.0, 0.0, 0.0, (i + 1) * 0.01) for i in range(100)]
    rs.append(serving.Result(100, 4, 1000, 1e-3, 0.0, 0.0, 0.0, 5.0))  # failed: not in the latencies
    s = serving.summarize(rs, 0.0)
    assert s["requests"] == 101 and s["ok"] == 100
    assert abs(s["p50_ms"] - 500.0) <= 10.0 and abs(s["p99_ms"] - 990.0) <= 10.0
    assert abs(s["solves_per_s"] - 100 / 5.0) < 1e-9
