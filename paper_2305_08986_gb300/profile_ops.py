"""Operator microbenchmark / profiling driver (one operator, repeated launches, CUDA events).

    python -m paper_2305_08986_gb300.profile_ops --op cheb32 --mesh 1280x224 --reps 20

Ops: a64, a32 (gs_vmult_A), saddle64 (gs_vmult), cheb32 / cheb64 (one Chebyshev smoothing call
of the finest level: k_A - 1 fused steps), vcycle (one V-cycle in the context precision).
The mesh is the channel workload geometry at the given size; --levels sets the hierarchy
(1 with --coarse-mode 1 builds only the finest level).  Prints one JSON line per op with the
median device time per launch and the operator throughput.
"""
from __future__ import annotations

import argparse
import json
import statistics


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="cheb32,a32,a64")
    ap.add_argument("--mesh", default="1280x224")
    ap.add_argument("--dim3", type=int, default=0, help="use the 3D sphere workload with n^3 cells")
    ap.add_argument("--levels", type=int, default=1)
    ap.add_argument("--coarse-mode", type=int, default=1)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--flush", type=int, default=1)
    ap.add_argument("--tile-autotune", type=int, default=0,
                    help="2D tile height: 0 autotuned, 1 / 2 / 3 forced 32 x 16 / 17 / 8 (gs_options.tile_autotune)")
    args = ap.parse_args()

    import torch
    from paper_2305_08986_gb300 import build
    build.build(verbose=False)
    from paper_2305_08986_gb300 import gs, inputs

    if args.dim3:
        p = inputs.config_spheres(n=args.dim3, levels=args.levels)
    else:
        nx, ny = (int(v) for v in args.mesh.split("x"))
        p = inputs.config_channel(nx=nx, ny=ny, levels=args.levels)
    dev = torch.device("cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for op in args.op.split(","):
        prec = 64 if op.endswith("64") else 32
        s = gs.Solver.from_problem(p, levels=args.levels, coarse_mode=args.coarse_mode, mg_precision=prec,
                                   tile_autotune=args.tile_autotune,
                                   restart=2)
        dt = torch.float64 if prec == 64 else torch.float32
        nu = s.n_u
        L = args.levels - 1
        if op.startswith("saddle"):
            x = torch.randn(s.n_total, dtype=torch.float64, device=dev)
            y = torch.empty_like(x)
            run = lambda: s.vmult(x, y)
            n_out = s.n_total
        elif op.startswith("cheb"):
            b = torch.randn(nu, dtype=dt, device=dev)
            y = torch.empty_like(b)
            run = lambda: s.apply_level(L, gs.OP_SMOOTH, b, y)
            n_out = nu
        elif op == "vcycle":
            r = torch.randn(nu, dtype=torch.float64, device=dev)
            z = torch.empty_like(r)
            run = lambda: s.vcycle(r, z)
            n_out = nu
        else:
            x = torch.randn(nu, dtype=dt, device=dev)
            y = torch.empty_like(x)
            run = lambda: s.vmult_A(x, y)
            n_out = nu
        for _ in range(3):
            run()
        ts = []
        st = torch.cuda.current_stream()
        for _ in range(args.reps):
            if args.flush:
                flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(st)
            run()
            e.record(st)
            e.synchronize()
            ts.append(a.elapsed_time(e))
        t = statistics.median(ts)
        print(json.dumps({"op": op, "mesh": args.mesh if not args.dim3 else f"{args.dim3}^3", "unknowns": n_out,
                          "median_ms": t, "min_ms": min(ts), "gdofs_per_s": n_out / (t * 1e-3) / 1e9}), flush=True)
        s.close()


if __name__ == "__main__":
    main()
