"""Serving loop on the GPU: requests that arrive while others run are admitted as slots and the
HBM cap allow, their solves overlap on the device, and each result is the same alone and in the
mix (bitwise: the batched kernels give every solve the same arithmetic whatever runs beside it)."""
import pytest

from paper_2305_08986_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-9


def _requests():
    P = [
        inputs.config_box_inclusion(2, (32, 32), inputs.levels_for(32, 2), 1e4, 100.0, seed=11),
        inputs.config_box_inclusion(3, (8, 8, 8), inputs.levels_for(8, 3), 1e6, 3.0, seed=12),
        inputs.config_box_inclusion(2, (48, 48), inputs.levels_for(48, 2), 3e2, 900.0, seed=13),
        inputs.config_box_inclusion(3, (16, 16, 16), inputs.levels_for(16, 3), 1e5, 40.0, seed=14),
        inputs.config_box_inclusion(2, (64, 64), inputs.levels_for(64, 2), 1e6, 1.0, seed=15),
        inputs.config_box_inclusion(2, (24, 24), inputs.levels_for(24, 2), 1e3, 500.0, seed=16),
        inputs.config_box_inclusion(3, (12, 12, 12), inputs.levels_for(12, 3), 2e4, 7.0, seed=17),
        inputs.config_box_inclusion(2, (40, 40), inputs.levels_for(40, 2), 5e5, 60.0, seed=18),
    ]
    return P


def _alone(p):
    import torch
    from paper_2305_08986_gb300 import gs
    s = gs.Solver.from_problem(p)
    f = torch.tensor(p.f, device="cuda")
    g = torch.tensor(p.g, device="cuda")
    b = torch.empty_like(f)
    s.lift_rhs(f, g, b)
    x = torch.zeros_like(b)
    eng = gs.Engine(1)
    assert eng.add(s, b, x, TOL)
    r = eng.run()[0]
    return x.cpu(), r["iterations"], r["rel_residual"]


def test_serving_alone_vs_in_the_mix():
    import torch
    from paper_2305_08986_gb300 import serving
    probs = _requests()
    alone = [_alone(p) for p in probs]
    fps = [serving.request_footprint(p) for p in probs]
    cap = 1.2 * max(fps)  # the largest request cannot join the first three: queueing on the footprint
    srv = serving.StokesServer(hbm_cap_bytes=cap, max_slots=3, setup_workers=2, keep_solutions=True)
    # all arrive at once, then two more bursts while the first ones run
    stream = [(0.0 if i < 4 else 0.05 * (i - 3), serving.Request(i, p, tol=TOL)) for i, p in enumerate(probs)]
    t0 = serving.run_stream(srv, stream, timeout_s=300)
    assert len(srv.results) == len(probs)
    assert srv.peak_used <= cap and srv.peak_running <= 3
    assert srv.cap_waits > 0  # the cap, not only the slot count, held requests back
    for r in srv.results:
        xa, ita, rra = alone[r.rid]
        assert r.status == 0 and r.rel_residual <= TOL
        assert (r.iterations, r.rel_residual) == (ita, rra)
        assert torch.equal(r.x, xa)
        assert r.t_arrival <= r.t_admitted <= r.t_ready <= r.t_done
    summ = serving.summarize(srv.results, t0)
    assert summ["ok"] == len(probs) and summ["p99_ms"] >= summ["p50_ms"] > 0
    srv.close()


def test_serving_rejects_requests_above_the_cap():
    from paper_2305_08986_gb300 import gs, serving
    p = _requests()[0]
    srv = serving.StokesServer(hbm_cap_bytes=serving.request_footprint(p) // 2, max_slots=2)
    serving.run_stream(srv, [(0.0, serving.Request(0, p))], timeout_s=60)
    assert [r.status for r in srv.results] == [gs.GS_ENOMEM]
    srv.close()


def test_described_requests_build_on_the_setup_thread():
    """A request given as a description (inputs.ProblemSpec) is built by the setup worker and
    solves to the same bits as the same request given with its arrays."""
    import torch
    from paper_2305_08986_gb300 import serving
    sp = inputs.serving_specs(3, seed=4, n2=(24, 48), n3=(8, 12))
    srv = serving.StokesServer(hbm_cap_bytes=64e9, max_slots=4, setup_workers=2, keep_solutions=True)
    stream = [(0.01 * i, serving.Request(i, s, tol=TOL)) for i, s in enumerate(sp)]
    serving.run_stream(srv, stream, timeout_s=300)
    assert sorted(r.rid for r in srv.results) == [0, 1, 2]
    for r in srv.results:
        xa, ita, rra = _alone(sp[r.rid].build())
        assert r.status == 0 and (r.iterations, r.rel_residual) == (ita, rra)
        assert torch.equal(r.x, xa)
    srv.close()
