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


def test_problem_spec_matches_the_built_problem():
    """The serving workload's request descriptions carry the mesh fields the admission needs and
    build the same instance config_box_inclusion draws."""
    import numpy as np
    from paper_2305_08986_gb300 import serving
    sp = inputs.serving_specs(6, seed=3)
    for s in sp:
        p = s.build()
        assert (p.dim, tuple(p.n), p.levels, p.alpha) == (s.dim, tuple(s.n), s.levels, s.alpha)
        assert p.n_total == s.n_total == len(p.f)
        assert serving.request_footprint(p) == serving.request_footprint(s)
        q = inputs.config_box_inclusion(s.dim, s.n, s.levels, s.contrast, s.alpha, seed=s.seed, align_coarse=True)
        assert np.array_equal(p.eta, q.eta) and np.array_equal(p.f, q.f)


def test_serving_mix_binds_a_150_gb_cap():
    """The default request mix: mean footprint of a few GB and a tail near 20 GB, so that a few
    dozen concurrent solves fill a 150 GB cap."""
    from paper_2305_08986_gb300 import serving
    fps = [serving.request_footprint(s) for s in inputs.serving_specs(400, seed=1)]
    mean = sum(fps) / len(fps)
    assert 1e9 < mean < 6e9 and max(fps) < 150e9 / 4
