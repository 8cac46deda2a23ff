"""Benchmark of the generalized Stokes solve on GB300 (one JSON line on stdout).

Step = one full solve of the 2D channel workload (FSI2i-like geometry: 2.5 x 0.41 channel,
square obstacle, stiff bar with eta contrast 1e4, alpha = rho / dt = 1e3, parabolic inflow,
do-nothing outflow) on a 1280 x 224 Q2-Q1 mesh with 6 multigrid levels: FGMRES in FP64 with the
FP32 multigrid V-cycle + Schur step inside, to relative residual 1e-8.  Inputs are resident in
HBM before the timed region; L2 is flushed (256 MiB write) between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gs|reference]

N > 1 (torchrun, one process per GPU): every rank solves its own replica (the path has no
exchange step); value = unknowns solved by all ranks / max-over-ranks time.
--impl reference times the FP64 CPU oracle (the plain assembled-matrix reference of the same
method) on a bounded sample of the workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A·x GDoF/s; time-to-solve rel-res 1e-8, FP32-MG vs FP64 on GB300; p50/p99"
WORKLOAD = dict(nx=1280, ny=224, levels=6)
TOL = 1e-8


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# --------------------------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# --------------------------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample
# --------------------------------------------------------------------------------------------
ORACLE_SAMPLE = dict(nx=320, ny=56, levels=4)  # ~5 s of host work per solve and core


def oracle_sample_run(steps: int, warmup: int):
    """Time the oracle on the channel workload at a reduced mesh (same geometry and coefficients):
    full setup + FGMRES solve to rel-res 1e-8, and one CSR SpMV of the assembled velocity block A
    (median of 20).  Returns a dict of per-solve seconds, unknowns, iterations and SpMV seconds."""
    import numpy as np
    from oracle.krylov import StokesOracle
    from oracle.mesh import mesh_from_problem
    from paper_2305_08986_gb300 import inputs
    p = inputs.config_channel(**ORACLE_SAMPLE)
    m = mesh_from_problem(p)
    times, its, spmv = [], [], []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        o = StokesOracle(m, p.eta, p.alpha, p.levels)
        b = o.sys.lift_rhs(p.f, p.g)
        x, it, rel, _ = o.solve(b, tol=TOL, max_iter=2000)
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
            its.append(it)
    A = o.sys.A
    xv = np.random.default_rng(0).standard_normal(A.shape[0])
    for _ in range(22):
        t0 = time.perf_counter()
        A @ xv
        spmv.append(time.perf_counter() - t0)
    return {"t": times, "n": m.N, "n_u": m.n_u, "it": its, "spmv_s": statistics.median(spmv[2:]),
            "csr_nnz": int(A.nnz)}


def _oracle_worker(args):
    steps, warmup = args
    return oracle_sample_run(steps, warmup)


def host_cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_all_cores(steps: int, warmup: int, cores: int = 0):
    """The oracle as it stands (single-threaded NumPy / SciPy code) on every host core at once: one
    independent solve per core in spawned worker processes (BLAS pinned to one thread each), so
    the throughput is whole-machine.  Returns the per-worker results and the wall time."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(steps, warmup)] * cores)
    return res, time.perf_counter() - t0, cores


def cpu_baseline_entry(res, cores):
    """GDoF/s of the whole host: unknowns solved by all workers / the slowest worker's time."""
    t = max(sum(r["t"]) for r in res)
    n = res[0]["n"]
    solves = sum(len(r["t"]) for r in res)
    spmv = statistics.median(r["spmv_s"] for r in res)
    return {"value": n * solves / t / 1e9, "unit": "GDoF/s", "cores": cores, "kind": "oracle",
            "cpu_model": host_cpu_model(),
            "csr_spmv_gdofs": res[0]["n_u"] * cores / spmv / 1e9,
            "csr_spmv_gdofs_per_core": res[0]["n_u"] / spmv / 1e9,
            "csr_bytes_per_dof": (res[0]["csr_nnz"] * 12 + 8 * res[0]["n_u"]) / res[0]["n_u"],
            "sample": (f"channel geometry at {ORACLE_SAMPLE['nx']}x{ORACLE_SAMPLE['ny']} cells, "
                       f"{ORACLE_SAMPLE['levels']} levels ({n} unknowns): full setup + FGMRES solve to rel-res "
                       f"1e-8 ({statistics.median(res[0]['it'])} iterations), {len(res[0]['t'])} per core on "
                       f"{cores} cores at once (one process per core); CSR SpMV of the assembled A "
                       f"({res[0]['n_u']} rows, {res[0]['csr_nnz']} nonzeros), median of 20 per core")}


def krylov_bytes(n: int, iterations: int, restart: int, form: str = "gram"):
    """Algorithmic HBM bytes and FP64 fused multiply-adds of the Gram-Schmidt kernels over one solve
    (8 B per basis entry; iteration k uses the j + 1 = (k mod restart) + 1 basis rows of its cycle).
    form "gram" (the default, orth = 0 / 2):
      dot pass: the j + 1 rows and w read once; 2 (j + 1) FMAs per entry (V^T w and the newest
      column of V^T V);
      update pass (+ norm): the rows read, w read and written; j + 2 FMAs per entry;
    form "explicit" (orth = 3):
      first pass (strip dots): the j + 1 rows and w read once; j + 1 FMAs per entry;
      second pass (update + dots): the rows read once from HBM (again from L1/L2 for the dots), w read
      and written; 2 (j + 1) FMAs per entry;
      third pass (update + norm): the rows read, w read and written; j + 2 FMAs per entry;
    both: the new basis vector, w read and v written."""
    dots = axpy = 0
    fma_dots = fma_axpy = 0
    for k in range(iterations):
        rows = (k % restart) + 1
        dots += (rows + 1) * n * 8
        if form == "gram":
            axpy += (rows + 2) * n * 8 + 2 * n * 8
            fma_dots += 2 * rows * n
            fma_axpy += (rows + 1) * n
        else:
            axpy += 2 * (rows + 2) * n * 8 + 2 * n * 8
            fma_dots += rows * n
            fma_axpy += (3 * rows + 1) * n
    return dots, axpy, fma_dots, fma_axpy


def krylov_rooflines(prof: dict, n: int, iterations: int, restart: int, peak_gbs: float, fp64_tflops: float,
                     form: str = "gram"):
    """Achieved GB/s (fraction of the measured HBM peak) and FP64 TFLOP/s (fraction of the measured
    FP64 peak) of the Gram-Schmidt classes, from the live per-class device time of one solve (CUDA
    events, one pair per launch: slightly long).  With the FP64 basis the FMA count binds: one FP64
    FMA per 8-byte entry read needs 0.85 T FMA/s at the HBM rate, above the ~0.5 T FMA/s of GB300."""
    dots_b, axpy_b, dots_f, axpy_f = krylov_bytes(n, iterations, restart, form)
    out = {}
    for cls, b, f in (("gram_schmidt_dots", dots_b, dots_f), ("krylov_axpy", axpy_b, axpy_f)):
        if cls in prof and prof[cls][1] > 0:
            t = prof[cls][1] * 1e-3
            gbs = b / t / 1e9
            tf = 2 * f / t / 1e12
            out[cls] = {"algorithmic_bytes": b, "fp64_fma": f, "ms": prof[cls][1], "achieved_gbs": gbs,
                        "frac_hbm": gbs / peak_gbs, "achieved_fp64_tflops": tf, "frac_fp64": tf / fp64_tflops}
    return out


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Largest value of x over the ranks of the default process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(unknowns_per_rank: int, steps: int, world: int, max_total_ms: float) -> float:
    """GDoF/s of the whole job: unknowns solved by all ranks / the max-over-ranks timed region."""
    return unknowns_per_rank * steps * world / (max_total_ms * 1e-3) / 1e9


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = max(1, min(args.steps, 2))
    res, wall, cores = oracle_all_cores(steps, 0)
    cb = cpu_baseline_entry(res, cores)
    t = max(sum(r["t"]) for r in res) / steps
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "GDoF/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": 0, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"channel {WORKLOAD['nx']}x{WORKLOAD['ny']} (sampled at "
                                   f"{ORACLE_SAMPLE['nx']}x{ORACLE_SAMPLE['ny']}, one solve per host core)", "tol": TOL},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------------
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch, from one ncu --set full
# capture of each kernel as built now: the finest-level fused Chebyshev step at the 1280 x 224
# workload (strip kernel; its writes d, x' stay in L2 within the capture, so the figure is the read
# traffic) and the FP64 saddle operator (x and eta read once; y and spilled registers written).
NCU_TRAFFIC_BYTES = {"cheb_step": 38.5664e6 + 7.936e3, "saddle_fp64": 25.351168e6 + 7.776256e6}


def tile_step_bytes(n_u: int, n_cells: int, elem: int, kind: str) -> int:
    """Algorithmic HBM bytes of one launch of a velocity tile kernel on one level.
    cheb_step: x, b, d, D^-1 read, d and x' written (6 vectors of d N_v entries) plus eta per cell;
    residual_A: x, b read, r written (3 vectors) plus eta; apply: x read, y written plus eta."""
    nvec = {"cheb_step": 6, "residual_A": 3, "apply": 2}[kind]
    return nvec * n_u * elem + n_cells * elem


def level_sizes(dim: int, n_fine, levels: int):
    """(n_u, n_cells) per level, coarsest first (n_l = n_fine / 2^(L-1-l) per axis)."""
    out = []
    for l in range(levels):
        n = [k >> (levels - 1 - l) for k in n_fine]
        nv = 1
        nc = 1
        for k in n:
            nv *= 2 * k + 1
            nc *= k
        out.append((dim * nv, nc))
    return out


def level_weighted_roofline(per_level: dict, sizes, cls: str, elem: int, peak_gbs: float):
    """Roofline of a tile-kernel class over all levels from the live per-level profile:
    achieved = sum_l bytes_l x launches_l / sum_l device time_l."""
    tot_b = tot_ms = 0.0
    n = 0
    rows = []
    for l, st in per_level.items():
        if l < 0 or cls not in st or st[cls][0] == 0:
            continue
        nl, ms = st[cls]
        bl = tile_step_bytes(sizes[l][0], sizes[l][1], elem, cls)
        tot_b += bl * nl
        tot_ms += ms
        n += nl
        rows.append({"level": l, "launches": nl, "bytes_per_launch": bl, "us_per_launch": 1e3 * ms / nl,
                     "frac": bl / (ms / nl * 1e-3) / 1e9 / peak_gbs})
    if n == 0:
        return None
    ach = tot_b / (tot_ms * 1e-3) / 1e9
    return {"achieved": ach, "frac": ach / peak_gbs, "launches": n, "ms": tot_ms,
            "bytes_per_launch": tot_b / n, "per_level": rows}


def time_apply_rotating(solver, n_u, n_cells, dtype, dev, stream, peak_gbs, reps=40):
    """A x through gs_vmult_A: `reps` back-to-back launches inside one CUDA event pair, cycling through
    copies of (x, y) that together exceed three times L2, so no launch finds its operands in L2 and
    none pays for another's dirty lines.  Algorithmic bytes: x read and y written (2 words per DoF)
    and eta read (one word per cell)."""
    import torch
    elem = 8 if dtype == torch.float64 else 4
    nsets = max(2, int(math.ceil(3 * 129e6 / (2 * n_u * elem))) + 1)
    sets = [(torch.randn(n_u, dtype=dtype, device=dev), torch.empty(n_u, dtype=dtype, device=dev))
            for _ in range(nsets)]
    for xx, yy in sets:
        solver.vmult_A(xx, yy)
    reps = max(reps, nsets)
    ts = []
    for _ in range(3):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(reps):
            xx, yy = sets[i % nsets]
            solver.vmult_A(xx, yy)
        e.record(stream)
        e.synchronize()
        ts.append(a.elapsed_time(e) / reps)
    t = min(ts) * 1e-3
    nbytes = 2 * elem * n_u + elem * n_cells
    del sets
    return {"gdofs": n_u / t / 1e9, "us": t * 1e6, "bytes": nbytes, "achieved_gbs": nbytes / t / 1e9,
            "frac_hbm": nbytes / t / 1e9 / peak_gbs, "launches": reps, "buffer_sets": nsets}


def run_gpu(args, rank, world):
    import numpy as np
    import torch
    from paper_2305_08986_gb300 import build as gsbuild
    gsbuild.build(verbose=False)
    from paper_2305_08986_gb300 import gs, inputs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    p = inputs.config_channel(**WORKLOAD)
    stream = torch.cuda.current_stream(dev)
    solver = gs.Solver.from_problem(p, device=dev, restart=args.restart, max_iter=4000,
                                    tile_autotune=args.tile_autotune)
    N = solver.n_total
    f = torch.tensor(p.f, device=dev)
    g = torch.tensor(p.g, device=dev)
    rhs = torch.empty_like(f)
    solver.lift_rhs(f, g, rhs)
    x = torch.zeros_like(f)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        x.zero_()
        solver.solve(rhs, x, tol=TOL, allow_noconv=True)
    launches0 = solver.info().kernel_launches
    times, its, rels = [], [], []
    clocks = Clocks(local)
    barrier()
    clocks.start()
    for _ in range(args.steps):
        x.zero_()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        it, rel, st = solver.solve(rhs, x, tol=TOL, allow_noconv=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        its.append(it)
        rels.append(rel)
    barrier()
    clk = clocks.stop()
    launches = solver.info().kernel_launches - launches0 - 0
    total_ms = max_over_ranks(sum(times), dist, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_value(N, args.steps, world, total_ms)

    # ---- per-kernel profile of one solve: per class and per multigrid level ----
    solver.profile(True)
    x.zero_()
    solver.solve(rhs, x, tol=TOL, allow_noconv=True)
    solver.profile(False)
    prof = solver.profile_read()
    per_level = {l: solver.profile_read(level=l) for l in range(-1, p.levels)}
    peaks = _peaks()
    peak_gbs = peaks.get("hbm_gbs", 6800.0)
    n_cells = p.n_cells
    n_u, n_p = solver.n_u, solver.n_p
    sizes = level_sizes(2, (WORKLOAD["nx"], WORKLOAD["ny"]), p.levels)

    # the finest-level fused Chebyshev step alone: 60 back-to-back launches (one event pair around
    # all of them) cycling through enough copies of its vectors that no launch finds its inputs in L2
    finest = None
    try:
        set_bytes = 5 * n_u * 4
        nsets = max(2, int(math.ceil(3 * 129e6 / set_bytes)) + 1)
        sets = []
        for k in range(nsets):
            xs_ = torch.randn(n_u, dtype=torch.float32, device=dev)
            aux = torch.randn(3 * n_u, dtype=torch.float32, device=dev)
            aux[2 * n_u:].abs_().mul_(1e-3)
            sets.append((xs_, aux, torch.empty_like(xs_)))
        L = p.levels - 1
        for xs_, aux, ys_ in sets:
            solver.apply_level(L, gs.OP_CHEB_STEP, xs_, ys_, aux=aux)
        reps = 60
        ts = []
        for _ in range(3):
            flush.fill_(3.0)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            for r_ in range(reps):
                xs_, aux, ys_ = sets[r_ % nsets]
                solver.apply_level(L, gs.OP_CHEB_STEP, xs_, ys_, aux=aux)
            b_.record(stream)
            b_.synchronize()
            ts.append(a_.elapsed_time(b_) / reps)
        us = 1e3 * min(ts)
        fb = tile_step_bytes(n_u, n_cells, 4, "cheb_step")
        finest = {"bytes": fb, "us": us, "achieved_gbs": fb / (us * 1e-6) / 1e9,
                  "frac": fb / (us * 1e-6) / 1e9 / peak_gbs, "launches": reps, "buffer_sets": nsets,
                  "how": f"{reps} back-to-back launches of gs_apply_level(GS_OP_CHEB_STEP) on level {L}, one event "
                         f"pair around them, cycling {nsets} vector sets of {set_bytes / 1e6:.0f} MB (> L2)"}
        del sets
    except Exception as ex:  # secondary figure: never break the bench line
        finest = {"error": str(ex)}

    cheb_roof = level_weighted_roofline(per_level, sizes, "cheb_step", 4, peak_gbs)
    roof = None
    if cheb_roof is not None:
        tr = NCU_TRAFFIC_BYTES.get("cheb_step")
        roof = {"bound": "hbm", "kernel": "cheb_step (fused Chebyshev step, FP32, all MG levels: strip kernel where a level has a 0 tile height, cell tiles elsewhere)",
                "achieved": cheb_roof["achieved"], "peak": peak_gbs, "unit": "GB/s", "frac": cheb_roof["frac"],
                "traffic": tr, "traffic_over_algorithmic": (tr / tile_step_bytes(n_u, n_cells, 4, "cheb_step")
                                                            if tr else None),
                "launches": cheb_roof["launches"], "avg_launch_us": 1e3 * cheb_roof["ms"] / cheb_roof["launches"],
                "bytes_per_launch": cheb_roof["bytes_per_launch"], "per_level": cheb_roof["per_level"],
                "finest": finest,
                "how": "sum over levels of algorithmic bytes x launches / summed device time of the class in one "
                       "solve (CUDA event pair per launch, which lengthens short launches: a lower bound); "
                       "finest: the finest-level step alone, back to back, inputs beyond L2",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"}
    saddle = None
    if "saddle_fp64" in prof and prof["saddle_fp64"][0] > 0:
        nl, ms = prof["saddle_fp64"]
        fl = n_cells * (534 + 2 * 75)
        ach = fl / (ms / nl * 1e-3) / 1e12
        saddle = {"bound": "alu", "achieved": ach, "peak": args.fp64_peak_tflops, "unit": "TFLOP/s",
                  "frac": ach / args.fp64_peak_tflops, "launches": nl, "avg_launch_us": 1e3 * ms / nl,
                  "peak_source": "nominal FP64 peak: 2 DFMA per SM per clock x 152 SMs x 2.07 GHz (ncu peak_sustained)"}

    # the line's roofline is the kernel with the most device time in the profiled solve: the FP64
    # saddle operator, or the Chebyshev step on the levels of one kernel variant (strip kernel where
    # tile_rows reports 0, cell tiles elsewhere)
    rows_l = [solver.info().tile_rows[l] for l in range(p.levels)]
    cheb_by_kernel = {}
    for l in range(p.levels):
        st_ = per_level.get(l, {}).get("cheb_step")
        if st_ and st_[0]:
            key = "strip" if rows_l[l] == 0 else "tile"
            cheb_by_kernel[key] = cheb_by_kernel.get(key, 0.0) + st_[1]
    dominant = roof
    cheb_max = max(cheb_by_kernel.values()) if cheb_by_kernel else 0.0
    if saddle is not None and (roof is None or prof["saddle_fp64"][1] > cheb_max):
        fl = n_cells * (534 + 2 * 75)
        tr = NCU_TRAFFIC_BYTES.get("saddle_fp64")
        dominant = dict(saddle, kernel="saddle_fp64 (FP64 saddle operator of the FGMRES matvec, 32 x 8 cell tiles)",
                        traffic=tr, traffic_over_algorithmic=tr / (8 * 2 * N + 8 * n_cells) if tr else None,
                        flops_per_launch=fl, cheb_step_ms_by_kernel=cheb_by_kernel,
                        how="algorithmic flops (684 per cell: the sum-factorised A, B and B^T) / average device "
                            "time per launch in the profiled solve; the FP64 pipe is the binding unit")

    krylov_table = None
    try:  # secondary figures: never let them break the bench line
        krylov_table = krylov_rooflines(prof, N, int(statistics.median(its)), args.restart, peak_gbs,
                                        args.fp64_peak_tflops)
    except Exception as ex:
        krylov_table = {"error": str(ex)}

    # ---- A x throughput (FP64 / FP32): back to back on operands beyond L2 ----
    ax64 = time_apply_rotating(solver, n_u, n_cells, torch.float64, dev, stream, peak_gbs)
    ax32 = time_apply_rotating(solver, n_u, n_cells, torch.float32, dev, stream, peak_gbs)

    # ---- FP64 multigrid comparison (plain FP64 GPU solve) ----
    fp64 = None
    if not args.skip_fp64 and rank == 0:
        s64 = gs.Solver.from_problem(p, device=dev, mg_precision=64, restart=args.restart, max_iter=4000)
        x64 = torch.zeros_like(f)
        s64.solve(rhs, x64, tol=TOL, allow_noconv=True)
        t64 = []
        for _ in range(max(1, min(2, args.steps))):
            x64.zero_()
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            it64, rel64, _ = s64.solve(rhs, x64, tol=TOL, allow_noconv=True)
            b.record(stream)
            b.synchronize()
            t64.append(a.elapsed_time(b))
        diff = float(torch.linalg.vector_norm(x64 - x) / torch.linalg.vector_norm(x64))
        fp64 = {"time_to_solve_ms": statistics.median(t64), "iterations": it64, "rel_residual": rel64,
                "solution_rel_diff_vs_fp32mg": diff}
        s64.close()

    # ---- the same solve with the double-float Krylov basis (krylov_fp64 = 2; the default is FP64) ----
    # ---- Krylov variants on the same system: the double-float basis (krylov_fp64 = 2), the
    # selective second Gram-Schmidt pass (orth = 1) and CGS2 with an explicit second pass (orth = 3) ----
    def krylov_variant(**opts):
        try:
            sk = gs.Solver.from_problem(p, device=dev, restart=args.restart, max_iter=4000,
                                        tile_autotune=args.tile_autotune, **opts)
            xk = torch.zeros_like(f)
            sk.solve(rhs, xk, tol=TOL, allow_noconv=True)
            tk = []
            for _ in range(max(1, min(3, args.steps))):
                xk.zero_()
                flush.fill_(1.0)
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                itk, relk, _ = sk.solve(rhs, xk, tol=TOL, allow_noconv=True)
                b_.record(stream)
                b_.synchronize()
                tk.append(a_.elapsed_time(b_))
            out = {"time_to_solve_ms": statistics.median(tk), "iterations": itk, "rel_residual": relk,
                   "solution_rel_diff_vs_default": float(torch.linalg.vector_norm(xk - x) /
                                                         torch.linalg.vector_norm(x))}
            sk.close()
            return out
        except Exception as ex:
            return {"error": str(ex)}

    kfp64 = krylov_variant(krylov_fp64=2) if rank == 0 else None
    korth = krylov_variant(orth=1) if rank == 0 else None
    kcgs2 = krylov_variant(orth=3) if rank == 0 else None
    # the Schur approximation by the 1/eta-weighted pressure mass alone (schur_kind = 1), without the
    # Cahouet-Chabard term of the default; it needs ~13x the iterations on this reaction-dominated case
    kmass = krylov_variant(schur_kind=1) if rank == 0 and not args.skip_mono else None

    # ---- the preconditioner of Sec. 4 itself: saddle-point multigrid with the block smoother, with
    # the paper's m = 2 smoothing steps and with m = 6 ----
    mono = None
    if not args.skip_mono and rank == 0:
        mono = []
        for msteps in (2, 6):
            sm = gs.Solver.from_problem(p, device=dev, precond_kind=1, mono_smooth=msteps, restart=args.restart,
                                        max_iter=4000)
            xm = torch.zeros_like(f)
            sm.solve(rhs, xm, tol=TOL, allow_noconv=True)
            tm = []
            for _ in range(max(1, min(3, args.steps))):
                xm.zero_()
                flush.fill_(1.0)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                itm, relm, stm = sm.solve(rhs, xm, tol=TOL, allow_noconv=True)
                b.record(stream)
                b.synchronize()
                tm.append(a.elapsed_time(b))
            mono.append({"precond": f"saddle-point multigrid, block smoother K_j (m = {msteps}, k_A = 4, "
                                    "n_S = k_S = 1), FP32 MG",
                         "time_to_solve_ms": statistics.median(tm), "iterations": itm, "rel_residual": relm,
                         "status": stm, "solution_rel_diff_vs_block": float(torch.linalg.vector_norm(xm - x) /
                                                                            torch.linalg.vector_norm(x))})
            sm.close()

    # ---- end to end through the public API with host buffers ----
    fh = torch.tensor(p.f).pin_memory()
    gh = torch.tensor(p.g).pin_memory()
    xh = torch.empty(N, dtype=torch.float64).pin_memory()
    fd = torch.empty_like(f)
    gd = torch.empty_like(g)
    e2e_ms = []
    for i in range(1 + max(1, min(args.steps, 3))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        fd.copy_(fh, non_blocking=True)
        gd.copy_(gh, non_blocking=True)
        solver.lift_rhs(fd, gd, rhs)
        x.zero_()
        solver.solve(rhs, x, tol=TOL, allow_noconv=True)
        xh.copy_(x, non_blocking=True)
        torch.cuda.synchronize(dev)
        if i > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_t = statistics.median(e2e_ms)

    if rank == 0:
        cb = None
        if not args.skip_cpu_baseline and world == 1:
            try:
                res, _, cores = oracle_all_cores(1, 0)
                cb = cpu_baseline_entry(res, cores)
            except Exception as ex:  # the baseline must not break the GPU line
                cb = {"value": None, "unit": "GDoF/s", "cores": os.cpu_count(), "kind": "oracle",
                      "sample": f"failed: {ex}"}
        ts = sorted(times)
        line = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": f"channel {WORKLOAD['nx']}x{WORKLOAD['ny']} Q2-Q1, obstacle + bar (eta 1e4), "
                                   f"alpha 1e3, {WORKLOAD['levels']} MG levels, FGMRES({args.restart}) FP64 + FP32 MG",
                       "unknowns": N, "tol": TOL, "l2": "flushed (256 MiB write) between timed steps",
                       "parallelism": f"replicas x{world}"},
            "time_to_solve_ms": {"p50": statistics.median(ts), "p99": ts[min(len(ts) - 1, int(math.ceil(0.99 * len(ts))) - 1)]},
            "iterations": statistics.median(its), "rel_residual": max(rels),
            "tile_rows": {"levels": [solver.info().tile_rows[l] for l in range(p.levels)],
                          "saddle": solver.info().saddle_tile_rows},
            "ax_gdofs": {"fp64": ax64, "fp32": ax32},
            "fp64_multigrid": fp64,
            "monolithic_precond": mono,
            "roofline": dominant,
            "rooflines": {"cheb_step": roof, "saddle_fp64": saddle},
            "krylov_rooflines": krylov_table,
            "krylov_double_float_basis": kfp64,
            "krylov_selective_reorth": korth,
            "krylov_explicit_cgs2": kcgs2,
            "schur_mass_only": kmass,
            "kernel_profile_ms": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items() if v[0]},
            "kernel_profile_note": "one CUDA event pair per launch (lengthens short launches); sums exceed the solve time",
            "cpu_baseline": cb,
            "e2e": {"value": N / (e2e_t * 1e-3) / 1e9, "unit": "GDoF/s", "ms": e2e_t,
                    "h2d_bytes_per_step": 2 * N * 8, "d2h_bytes_per_step": N * 8},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# --------------------------------------------------------------------------------------------
# batched workload: many uneven instances through the batching engine vs one after the other
# --------------------------------------------------------------------------------------------
def run_batched(args):
    import torch
    from paper_2305_08986_gb300 import build as gsbuild
    gsbuild.build(verbose=False)
    from paper_2305_08986_gb300 import gs, inputs
    dev = torch.device("cuda", 0)
    probs = inputs.batch_instances(args.instances, seed=0, align_coarse=not args.unaligned)
    t0 = time.perf_counter()
    solvers, rhs, xs = [], [], []
    for p in probs:
        s = gs.Solver.from_problem(p, device=dev, deflate=args.deflate, max_iter=args.max_iter)
        f = torch.tensor(p.f, device=dev)
        g = torch.tensor(p.g, device=dev)
        b = torch.empty_like(f)
        s.lift_rhs(f, g, b)
        solvers.append(s)
        rhs.append(b)
        xs.append(torch.zeros_like(b))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    unknowns = sum(s.n_total for s in solvers)
    st = torch.cuda.current_stream(dev)

    def timed(fn):
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        out = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    def engine_run():
        return gs.batch_solve(solvers, rhs, xs, tol=TOL)

    def sequential_run():
        its = []
        for s, b, x in zip(solvers, rhs, xs):
            it, rr, _ = s.solve(b, x, tol=TOL, allow_noconv=True)
            its.append(it)
        return its

    for _ in range(max(1, args.warmup)):
        timed(engine_run)
    eng_ms = []
    for _ in range(max(1, min(args.steps, 5))):
        ms, (status, its, rels) = timed(engine_run)
        eng_ms.append(ms)
    failed = [i for i, r in enumerate(rels) if not r <= TOL]
    x_eng = [x.clone() for x in xs]
    timed(sequential_run)
    seq_ms = []
    for _ in range(max(1, min(args.steps, 2))):
        ms, its_seq = timed(sequential_run)
        seq_ms.append(ms)
    diff = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(x_eng, xs))
    eng = gs.Engine(len(solvers))
    for i, (s, b, x) in enumerate(zip(solvers, rhs, xs)):
        x.zero_()
        eng.add(s, b, x, TOL, tag=i)
    eng.run()
    stats = eng.stats()
    eng.close()
    n2 = sum(1 for p in probs if p.dim == 2)
    boxes = "unaligned box inclusion (as drawn)" if args.unaligned else "box inclusion aligned with the coarsest mesh"
    line = {"workload": f"batched: {len(probs)} instances ({n2} 2D in 16^2..256^2, {len(probs) - n2} 3D in 8^3..32^3), "
                        f"{boxes}, contrast U(1e2,1e6), alpha U(1,1e3), FP32 MG / FP64 FGMRES(50), rel-res 1e-8"
                        + (", rigid-body deflation of the inclusion" if args.deflate else "")
                        + f", at most {args.max_iter} iterations",
            "metric": "solve throughput", "unit": "GDoF/s", "unknowns": unknowns,
            "value": unknowns / (statistics.median(eng_ms) * 1e-3) / 1e9,
            "engine_ms": {"p50": statistics.median(eng_ms), "max": max(eng_ms)},
            "sequential_ms": statistics.median(seq_ms),
            "speedup_vs_sequential": statistics.median(seq_ms) / statistics.median(eng_ms),
            "iterations": {"mean": statistics.fmean(its), "max": max(its)},
            "not_converged_count": len(failed),
            "not_converged": [{"i": i, "dim": probs[i].dim, "n": probs[i].n[0], "levels": probs[i].levels,
                               "alpha": probs[i].alpha, "its": its[i], "rel": rels[i]} for i in failed],
            "solution_rel_diff_engine_vs_sequential": diff,
            "setup_s": t_setup, "engine_stats": stats, "steps": args.steps, "warmup": args.warmup}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------
# serving: Poisson arrivals through the continuous-batching server vs sequential plain FP64
# --------------------------------------------------------------------------------------------
def run_serving(args):
    os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")
    import numpy as np
    import torch
    from paper_2305_08986_gb300 import build as gsbuild
    gsbuild.build(verbose=False)
    from paper_2305_08986_gb300 import gs, inputs, serving
    dev = torch.device("cuda", 0)
    rates = [float(r) for r in args.rates.split(",")]
    specs = inputs.serving_specs(args.requests, seed=1)
    fps = [serving.request_footprint(sp) for sp in specs]
    # sequential plain FP64 baseline: service time of each of the first requests alone (problem arrays,
    # setup, FP64-multigrid solve, copy back), then the same arrivals through one FIFO server
    nb = min(args.baseline_requests, len(specs))
    svc = []
    for sp in specs[:nb]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p = sp.build()
        s = gs.Solver.from_problem(p, device=dev, mg_precision=64)
        f = torch.tensor(p.f, device=dev)
        g = torch.tensor(p.g, device=dev)
        b = torch.empty_like(f)
        s.lift_rhs(f, g, b)
        x = torch.zeros_like(b)
        s.solve(b, x, tol=TOL, allow_noconv=True)
        x.cpu()
        s.close()
        del s, f, g, b, x
        svc.append(time.perf_counter() - t0)
    out = {"workload": f"serving: up to {args.requests} requests or {args.rate_seconds:g} s of arrivals per rate, "
                       "2D 32^2..1536^2 and 3D 8^3..96^3 log-uniform, box inclusion contrast log-uniform in [1, 1e6], "
                       f"rel-res 1e-8, HBM admission cap {args.hbm_cap_gb:g} GB, continuous batching "
                       "(FP32 MG / FP64 FGMRES)",
           "footprint_gb": {"mean": statistics.fmean(fps) / 1e9, "max": max(fps) / 1e9,
                            "p50": statistics.median(fps) / 1e9},
           "baseline": f"sequential plain FP64 (FP64 multigrid): each of the first {nb} requests run alone "
                       "(arrays + setup + solve + copy back), then replayed through one FIFO server with the "
                       "same arrival times",
           "rates": {}}
    for rate in rates:
        count = int(min(len(specs), max(1, math.ceil(rate * args.rate_seconds))))
        rng = np.random.default_rng(int(rate * 1000) + 7)
        offs = np.cumsum(rng.exponential(1.0 / rate, size=count))
        stream = [(float(o), serving.Request(i, sp, tol=TOL)) for i, (o, sp) in enumerate(zip(offs, specs[:count]))]
        srv = serving.StokesServer(hbm_cap_bytes=args.hbm_cap_gb * 1e9, max_slots=256, setup_workers=8)
        t0 = serving.run_stream(srv, stream, timeout_s=1200.0)
        summ = serving.summarize(srv.results, t0)
        summ["arrival_span_s"] = float(offs[-1])
        summ["peak_running"] = srv.peak_running
        summ["peak_admitted_gb"] = srv.peak_used / 1e9
        summ["cap_bound"] = srv.cap_waits > 0
        summ["admissions_held_by_cap"] = srv.cap_waits
        summ["engine_steps"] = srv.engine.stats()["steps"]
        srv.close()
        del srv
        torch.cuda.empty_cache()
        k = min(nb, count)
        tfree, lat = 0.0, []
        for o, d in zip(offs[:k], svc[:k]):
            start = max(o, tfree)
            tfree = start + d
            lat.append(tfree - o)
        lat.sort()
        q = lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))]
        summ["sequential_fp64"] = {"requests": k, "p50_ms": 1e3 * q(0.5), "p99_ms": 1e3 * q(0.99),
                                   "solves_per_s": k / (tfree - offs[0] + svc[0])}
        out["rates"][f"{rate:g}"] = summ
        print(json.dumps({"rate": rate, **summ}), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------------------------
# mesh-extension workload (Eq. "extenstion"): CG + velocity V-cycle on the channel, tol 1e-6
# --------------------------------------------------------------------------------------------
def run_extension(args):
    import torch
    from paper_2305_08986_gb300 import build as gsbuild
    gsbuild.build(verbose=False)
    from paper_2305_08986_gb300 import gs, inputs
    dev = torch.device("cuda", 0)
    p = inputs.config_extension(nx=WORKLOAD["nx"], ny=WORKLOAD["ny"], levels=WORKLOAD["levels"])
    f = torch.tensor(p.f, device=dev)
    g = torch.tensor(p.g, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)
    out = {"workload": f"mesh extension {WORKLOAD['nx']}x{WORKLOAD['ny']} Q2 (channel solid as obstacle cells, "
                       f"bar bending 0.02 at the tip), mu_A of Eq. mu_distribution, {WORKLOAD['levels']} MG levels, "
                       "flexible PCG FP64 + one velocity V-cycle, rel-res 1e-6",
           "l2": "flushed (256 MiB write) before every timed run"}
    for prec in (32, 64):
        s = gs.Solver.from_problem(p, device=dev, mg_precision=prec)
        b = torch.empty_like(f)
        s.lift_rhs(f, g, b)
        bu = b[:s.n_u].contiguous()
        x = torch.zeros_like(bu)
        s.solve_A(bu, x, tol=1e-6, allow_noconv=True)  # warm-up
        ts = []
        for _ in range(max(1, args.steps)):
            x.zero_()
            flush.fill_(1.0)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            it, rr, _ = s.solve_A(bu, x, tol=1e-6, allow_noconv=True)
            e.record(st)
            e.synchronize()
            ts.append(a.elapsed_time(e))
        key = ("fp32_multigrid" if prec == 32 else "fp64_multigrid") + ("_kA6" if kdeg == 6 else "")
        out[key] = {
            "time_to_solve_ms": statistics.median(ts), "iterations": it, "rel_residual": rr, "unknowns": s.n_u}
        s.close()
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------------------------
# 3D spheres workload (64^3, 64 stiff spheres): deflated solve, FP32 vs FP64 multigrid, 3D A x
# --------------------------------------------------------------------------------------------
def run_spheres(args):
    import torch
    from paper_2305_08986_gb300 import build as gsbuild
    gsbuild.build(verbose=False)
    from paper_2305_08986_gb300 import gs, inputs
    dev = torch.device("cuda", 0)
    p = inputs.config_spheres(n=64, levels=5)
    f = torch.tensor(p.f, device=dev)
    g = torch.tensor(p.g, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)
    out = {"workload": "spheres 64^3 Q2-Q1 (6.71 M unknowns), 64 spheres eta 1e6 in 1, alpha 1e2, 5 MG levels, "
                       "rigid-body deflation of the inclusions, FGMRES(200) FP64, rel-res 1e-8",
           "l2": "flushed (256 MiB write) before every timed run"}
    for prec in (32, 64):
        s = gs.Solver.from_problem(p, device=dev, mg_precision=prec, deflate=1, restart=200, max_iter=2000)
        b = torch.empty_like(f)
        s.lift_rhs(f, g, b)
        x = torch.zeros_like(b)
        s.solve(b, x, tol=TOL, allow_noconv=True)  # warm-up (graph capture)
        ts, its, rels = [], [], []
        for _ in range(max(1, min(args.steps, 3) if prec == 32 else 1)):
            x.zero_()
            flush.fill_(1.0)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            it, rr, _ = s.solve(b, x, tol=TOL, allow_noconv=True)
            e.record(st)
            e.synchronize()
            ts.append(a.elapsed_time(e))
            its.append(it)
            rels.append(rr)
        inf = s.info()
        key = "fp32_multigrid" if prec == 32 else "fp64_multigrid"
        out[key] = {"time_to_solve_ms": statistics.median(ts), "iterations": its[-1], "rel_residual": max(rels),
                    "unknowns": s.n_total, "deflation_inclusions": inf.deflation_inclusions,
                    "deflation_modes": inf.deflation_modes}
        if prec == 32:
            x32 = x.clone()
        else:  # FP32- against FP64-multigrid solution (both FP64 FGMRES to rel-res 1e-8); velocity part
            # and whole vector (the pressure inside an eta = 1e6 sphere is pinned only to ~1e-3)
            n_u = s.n_u
            out[key]["velocity_rel_diff_vs_fp32mg"] = float(torch.linalg.vector_norm(x[:n_u] - x32[:n_u]) /
                                                            torch.linalg.vector_norm(x[:n_u]))
            out[key]["solution_rel_diff_vs_fp32mg"] = float(torch.linalg.vector_norm(x - x32) /
                                                            torch.linalg.vector_norm(x))
        if prec == 32:
            for dt, name in ((torch.float32, "fp32"), (torch.float64, "fp64")):
                out.setdefault("ax_gdofs", {})[name] = time_apply_rotating(s, s.n_u, p.n_cells, dt, dev, st,
                                                                          _peaks().get("hbm_gbs", 6800.0))
        s.close()
        del s, b, x
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------------------------
# corrector stage (Sec. 3.1.2, Eq. "v_star"): the channel with the predictor solution as v°
# --------------------------------------------------------------------------------------------
def run_corrector(args):
    """Solve the predictor system of the channel, then the corrector system with that velocity as
    the convective field v° (rho = 1): FGMRES with the block-triangular preconditioner built on the
    non-symmetric block (FP32 and FP64 multigrid), L2 flushed before every timed solve."""
    import torch
    from paper_2305_08986_gb300 import build as gsbuild
    gsbuild.build(verbose=False)
    from paper_2305_08986_gb300 import gs, inputs
    dev = torch.device("cuda", 0)
    if args.dim3:  # 3D: box inclusion (contrast 1e3, aligned with the coarsest mesh), do-nothing face z+
        n3 = args.dim3
        p = inputs.config_box_inclusion(3, (n3,) * 3, inputs.levels_for(n3, 3), 1e3, 100.0, seed=0,
                                        faces=inputs.all_faces(3) & ~inputs.FACE_ZP, align_coarse=True)
    else:
        p = inputs.config_channel(**WORKLOAD)
    f = torch.tensor(p.f, device=dev)
    g = torch.tensor(p.g, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)
    where = (f"box inclusion {args.dim3}^3 Q2-Q1 (contrast 1e3, alpha 100)" if args.dim3 else
             f"channel {WORKLOAD['nx']}x{WORKLOAD['ny']} Q2-Q1")
    out = {"workload": f"corrector stage, {where}, v° = the predictor solution, rho 1, convection + "
                       f"streamline diffusion (Eq. a_stab), {p.levels} MG levels, FGMRES({args.restart}) FP64, "
                       "rel-res 1e-8", "unknowns": len(p.f),
           "l2": "flushed (256 MiB write) before every timed solve"}
    # k_A = 4 (the predictor's degree) and k_A = 6, the corrector column of Table
    # "NS-solver-parameters-1"
    for prec, kdeg in ((32, 4), (32, 6), (64, 4)):
        s = gs.Solver.from_problem(p, device=dev, mg_precision=prec, corrector=1, restart=args.restart,
                                   max_iter=4000, tile_autotune=args.tile_autotune, cheb_degree=kdeg)
        b = torch.empty_like(f)
        s.lift_rhs(f, g, b)
        x = torch.zeros_like(b)
        it_p, _, _ = s.solve(b, x, tol=1e-10, allow_noconv=True)
        vcirc = x[:s.n_u].cpu().numpy()
        t0 = time.perf_counter()
        s.set_corrector(vcirc, 1.0)
        t_set = time.perf_counter() - t0
        s.lift_rhs(f, g, b)
        x.zero_()
        s.solve(b, x, tol=TOL, allow_noconv=True)  # warm-up (graph capture)
        ts = []
        for _ in range(max(1, min(args.steps, 5))):
            x.zero_()
            flush.fill_(1.0)
            a_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(st)
            it, rr, _ = s.solve(b, x, tol=TOL, allow_noconv=True)
            e_.record(st)
            e_.synchronize()
            ts.append(a_.elapsed_time(e_))
        key = ("fp32_multigrid" if prec == 32 else "fp64_multigrid") + ("_kA6" if kdeg == 6 else "")
        out[key] = {
            "time_to_solve_ms": statistics.median(ts), "iterations": it, "rel_residual": rr,
            "predictor_iterations": it_p, "set_corrector_s": t_set, "unknowns": s.n_total}
        s.close()
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------------------------
# one solve inside an NVTX range (the command the committed launch-list summaries were taken with)
# --------------------------------------------------------------------------------------------
def run_solve_once(args):
    """Build the channel solver, solve once to warm up (graph capture), then solve once more inside
    the NVTX range "timed_solve", so that a profiler can select exactly one solve's launches."""
    import torch
    from paper_2305_08986_gb300 import build as gsbuild
    gsbuild.build(verbose=False)
    from paper_2305_08986_gb300 import gs, inputs
    dev = torch.device("cuda", 0)
    p = inputs.config_channel(**WORKLOAD)
    s = gs.Solver.from_problem(p, device=dev, restart=args.restart, max_iter=4000, tile_autotune=args.tile_autotune)
    f = torch.tensor(p.f, device=dev)
    g = torch.tensor(p.g, device=dev)
    rhs = torch.empty_like(f)
    s.lift_rhs(f, g, rhs)
    x = torch.zeros_like(f)
    s.solve(rhs, x, tol=TOL, allow_noconv=True)
    x.zero_()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_solve")
    it, rel, _ = s.solve(rhs, x, tol=TOL, allow_noconv=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"workload": "solve_once", "iterations": it, "rel_residual": rel,
                      "tile_rows": [s.info().tile_rows[l] for l in range(p.levels)]}), flush=True)
    s.close()


# --------------------------------------------------------------------------------------------
# one operator, repeated (the command the committed ncu summaries were taken with)
# --------------------------------------------------------------------------------------------
def run_op(args):
    """Repeat one operator on a one-level context and print its device time per launch: a32 / a64
    (gs_vmult_A), saddle64 (gs_vmult), chebstep (GS_OP_CHEB_STEP, FP32) on the channel geometry at
    --mesh, or on the 3D sphere workload with --dim3 n.  --steps launches run back to back (one
    CUDA event pair around them) cycling through copies of the operands that together exceed
    three times L2, so no launch finds its inputs in L2 and none pays for another's dirty lines."""
    import torch
    from paper_2305_08986_gb300 import build as gsbuild
    gsbuild.build(verbose=False)
    from paper_2305_08986_gb300 import gs, inputs
    dev = torch.device("cuda", 0)
    if args.dim3:
        p = inputs.config_spheres(n=args.dim3, levels=1)
    else:
        nx, ny = (int(v) for v in args.mesh.split("x"))
        p = inputs.config_channel(nx=nx, ny=ny, levels=1)
    st = torch.cuda.current_stream(dev)
    for op in args.op.split(","):
        prec = 64 if op.endswith("64") else 32
        s = gs.Solver.from_problem(p, levels=1, coarse_mode=1, mg_precision=prec, restart=2,
                                   tile_autotune=args.tile_autotune)
        dt = torch.float64 if prec == 64 else torch.float32
        es = 8 if prec == 64 else 4
        nu = s.n_u
        if op == "saddle64":
            per_set = 2 * s.n_total * es
        elif op == "chebstep":
            per_set = 5 * nu * es
        else:
            per_set = 2 * nu * es
        nsets = max(2, int(math.ceil(3 * 129e6 / per_set)) + 1)
        sets = []
        for _ in range(nsets):
            if op == "saddle64":
                xx = torch.randn(s.n_total, dtype=dt, device=dev)
                sets.append((xx, torch.empty_like(xx), None))
            elif op == "chebstep":
                xx = torch.randn(nu, dtype=dt, device=dev)
                aux = torch.randn(3 * nu, dtype=dt, device=dev)
                aux[2 * nu:].abs_().mul_(1e-3)
                sets.append((xx, torch.empty_like(xx), aux))
            else:
                xx = torch.randn(nu, dtype=dt, device=dev)
                sets.append((xx, torch.empty_like(xx), None))

        def run(i):
            xx, yy, aux = sets[i % nsets]
            if op == "saddle64":
                s.vmult(xx, yy)
            elif op == "chebstep":
                s.apply_level(0, gs.OP_CHEB_STEP, xx, yy, aux=aux)
            else:
                s.vmult_A(xx, yy)
        for i in range(nsets):
            run(i)
        reps = max(args.steps, nsets)
        ts = []
        for _ in range(3):
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(st)
            for i in range(reps):
                run(i)
            b_.record(st)
            b_.synchronize()
            ts.append(a_.elapsed_time(b_) / reps)
        t = min(ts)
        print(json.dumps({"op": op, "mesh": args.mesh if not args.dim3 else f"{args.dim3}^3", "n_u": nu,
                          "us_per_launch": 1e3 * t, "launches": reps, "buffer_sets": nsets,
                          "tile_rows": s.info().tile_rows[0], "gdofs": nu / (t * 1e-3) / 1e9}), flush=True)
        del sets
        s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gs", choices=["gs", "reference"])
    ap.add_argument("--restart", type=int, default=50)
    ap.add_argument("--fp64-peak-tflops", type=float, default=1.25,
                    help="FP64 peak of ALU-bound rooflines: 2 DFMA per SM per clock (ncu peak_sustained) x 152 SMs x 2 "
                         "flops x 2.07 GHz = 1.26 TFLOP/s, the nominal 1.25 TFLOP/s")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-mono", action="store_true", help="skip the Sec. 4 saddle-point multigrid comparison")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--tile-autotune", type=int, default=5, choices=[0, 1, 2, 3, 4, 5],
                    help="2D velocity-block kernel of the channel solver: 5 (default here) the size rule (strip "
                         "kernel on levels of >= 32768 cells, 32 x 8 tiles below: the choice the timing autotuner "
                         "makes on this workload, fixed so that profiler runs launch the same kernels); 0 the timing "
                         "autotuner; 1 / 2 / 3: tiles of 32 x 16 / 17 / 8; 4: the strip kernel everywhere")
    ap.add_argument("--op", default="chebstep,a32,a64", help="--workload op: operators to repeat")
    ap.add_argument("--mesh", default="1280x224", help="--workload op: channel mesh")
    ap.add_argument("--dim3", type=int, default=0, help="--workload op: 3D sphere mesh n^3 instead")
    ap.add_argument("--workload", default="channel",
                    choices=["channel", "batched", "serving", "spheres", "extension", "op", "solve_once",
                             "corrector"],
                    help="channel: the contract line; batched / serving: the engine workloads; spheres: the 3D "
                         "64^3 inclusion workload (extra lines)")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--unaligned", action="store_true", help="--workload batched: boxes as drawn, not snapped")
    ap.add_argument("--deflate", type=int, default=0, choices=[0, 1], help="--workload batched: deflation option")
    ap.add_argument("--max-iter", type=int, default=1000, help="--workload batched: FGMRES iteration limit")
    ap.add_argument("--requests", type=int, default=2000, help="--workload serving: requests per rate at most")
    ap.add_argument("--rate-seconds", type=float, default=60.0, help="--workload serving: arrival span per rate")
    ap.add_argument("--baseline-requests", type=int, default=100,
                    help="--workload serving: requests timed alone for the sequential FP64 baseline")
    ap.add_argument("--rates", default="10,30,100,300,1000")
    ap.add_argument("--hbm-cap-gb", type=float, default=150.0)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload == "batched" and args.impl == "gs":
        return run_batched(args)
    if args.workload == "serving" and args.impl == "gs":
        return run_serving(args)
    if args.workload == "spheres" and args.impl == "gs":
        return run_spheres(args)
    if args.workload == "extension" and args.impl == "gs":
        return run_extension(args)
    if args.workload == "op" and args.impl == "gs":
        return run_op(args)
    if args.workload == "solve_once" and args.impl == "gs":
        return run_solve_once(args)
    if args.workload == "corrector" and args.impl == "gs":
        return run_corrector(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
