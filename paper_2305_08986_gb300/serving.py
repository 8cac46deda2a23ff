"""Serving loop for generalized Stokes solves on one GPU (continuous batching).

Requests (a mesh, eta per cell, alpha, load and boundary data, a tolerance) arrive at any time.
The server admits them first come, first served while the sum of the admitted requests' device
footprints stays under an HBM cap, builds each admitted request's context on a setup thread (its
own CUDA stream: multigrid hierarchy, Chebyshev bounds, coarse inverse, lifted right-hand side),
and hands ready contexts to the batching engine (gs_engine_*), which advances every running
solve by one FGMRES iteration per step with one launch per kernel for all of them.  Requests
join at the next step after their setup and leave when they converge; the solution is copied to
host memory and the request's memory is released.  Latency = result on host - arrival.

The ctypes calls release the GIL, so setups (gs_create, host-synchronising) overlap the engine's
steps on the device.
"""
from __future__ import annotations

import collections
import concurrent.futures
import statistics
import threading
import time
from dataclasses import dataclass, field
from typing import Any, Dict, List, Optional

from . import gs


@dataclass
class Request:
    rid: int
    problem: Any            # inputs.Problem (dim, n, length, levels, eta, alpha, dirichlet_faces, void, f, g),
                            # or a description with the same mesh fields and a build() that returns one
                            # (its arrays are then made on the setup thread)
    t_arrival: float = 0.0  # seconds on the server clock (time.perf_counter())
    tol: float = 1e-8
    opts: Dict[str, int] = field(default_factory=dict)


@dataclass
class Result:
    rid: int
    status: int
    iterations: int
    rel_residual: float
    t_arrival: float
    t_admitted: float
    t_ready: float
    t_done: float
    x: Any = None           # host tensor (float64) when keep_solutions

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def request_footprint(p, opts=None) -> int:
    """Device bytes one request holds while admitted: the context workspace plus the load,
    Dirichlet data, right-hand side and solution vectors."""
    opts = opts or {}
    ws = gs.footprint_bytes(p.dim, p.n, p.length, p.levels, p.void, p.dirichlet_faces, **opts)
    return int(ws + 4 * 8 * p.n_total + 4096)


class StokesServer:
    def __init__(self, hbm_cap_bytes: float = 150e9, max_slots: int = 256, setup_workers: int = 4,
                 keep_solutions: bool = False, device: str = "cuda"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.cap = int(hbm_cap_bytes)
        self.max_slots = int(max_slots)
        self.keep = keep_solutions
        self.engine_stream = torch.cuda.Stream(self.device)
        self.engine = gs.Engine(self.max_slots, 0, stream=self.engine_stream, device=device)
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=setup_workers)
        self._tls = threading.local()
        self.queue: collections.deque = collections.deque()
        self.setups: List = []            # (request, footprint, t_admitted, future)
        self.running: Dict[int, tuple] = {}  # rid -> (request, footprint, t_admitted, t_ready, solver, b, x)
        self.used = 0
        self.peak_used = 0
        self.cap_waits = 0                # requests that waited at the head of the queue for memory
        self._held = None
        self.peak_running = 0
        self.results: List[Result] = []

    # ---- request intake ------------------------------------------------------------------------
    def submit(self, req: Request):
        self.queue.append(req)

    def busy(self) -> bool:
        return bool(self.queue or self.setups or self.running)

    def _setup(self, req: Request):
        torch = self.torch
        st = getattr(self._tls, "stream", None)
        if st is None:
            st = self._tls.stream = torch.cuda.Stream(self.device)
        p = req.problem.build() if hasattr(req.problem, "build") else req.problem
        with torch.cuda.device(self.device), torch.cuda.stream(st):
            s = gs.Solver.from_problem(p, stream=st, **req.opts)
            f = torch.as_tensor(p.f, dtype=torch.float64).pin_memory().to(self.device, non_blocking=True)
            g = torch.as_tensor(p.g, dtype=torch.float64).pin_memory().to(self.device, non_blocking=True)
            b = torch.empty_like(f)
            s.lift_rhs(f, g, b)
            x = torch.zeros_like(b)
            st.synchronize()
        return s, b, x

    # ---- one scheduler iteration ------------------------------------------------------------------
    def pump(self) -> bool:
        """Admit, start setups, add ready solves, run one engine step, retire finished solves.
        Returns True if any work was done."""
        now = time.perf_counter
        worked = False
        # admission: FIFO by HBM footprint and free slots (setups in flight hold a slot)
        while self.queue:
            req = self.queue[0]
            fp = request_footprint(req.problem, req.opts)
            if fp > self.cap:
                self.queue.popleft()
                self.results.append(Result(req.rid, gs.GS_ENOMEM, 0, float("nan"), req.t_arrival, now(), now(), now()))
                continue
            if self.used + fp > self.cap:
                if self._held != req.rid:
                    self._held = req.rid
                    self.cap_waits += 1
                break
            if len(self.setups) + len(self.running) >= self.max_slots:
                break
            self.queue.popleft()
            self.used += fp
            self.peak_used = max(self.peak_used, self.used)
            self.setups.append((req, fp, now(), self.pool.submit(self._setup, req)))
            worked = True
        # ready setups join the engine
        still = []
        for req, fp, ta, fut in self.setups:
            if not fut.done():
                still.append((req, fp, ta, fut))
                continue
            s, b, x = fut.result()
            if not self.engine.add(s, b, x, req.tol, tag=req.rid):
                still.append((req, fp, ta, fut))  # cannot happen: slots are reserved at admission
                continue
            self.running[req.rid] = (req, fp, ta, now(), s, b, x)
            worked = True
        self.setups = still
        self.peak_running = max(self.peak_running, len(self.running))
        if self.engine.active() > 0:
            self.engine.step()
            worked = True
        for r in self.engine.poll():
            req, fp, ta, tr, s, b, x = self.running.pop(int(r["tag"]))
            xh = x.cpu()  # the result reaches the host
            self.results.append(Result(req.rid, r["status"], r["iterations"], r["rel_residual"], req.t_arrival, ta, tr,
                                       now(), xh if self.keep else None))
            s.close()
            del s, b, x
            self.used -= fp
        return worked

    def close(self):
        self.pool.shutdown(wait=True)
        self.engine.close()


def run_stream(server: StokesServer, stream, t0: Optional[float] = None, timeout_s: float = 600.0):
    """Replay a list of (arrival_offset_s, Request) in real time through the server."""
    t0 = time.perf_counter() if t0 is None else t0
    pending = collections.deque(sorted(stream, key=lambda a: a[0]))
    deadline = t0 + timeout_s
    while pending or server.busy():
        tnow = time.perf_counter()
        while pending and t0 + pending[0][0] <= tnow:
            off, req = pending.popleft()
            req.t_arrival = t0 + off
            server.submit(req)
        if not server.pump():
            # idle: wait for the next arrival or a setup to finish
            nxt = (t0 + pending[0][0] - time.perf_counter()) if pending else 0.001
            time.sleep(max(0.0, min(nxt, 0.002)))
        if time.perf_counter() > deadline:
            raise TimeoutError("serving run exceeded its time limit")
    return t0


def summarize(results: List[Result], t0: float) -> Dict[str, float]:
    ok = [r for r in results if r.status == gs.GS_OK]
    lat = sorted(r.latency for r in ok)

    def pct(q):
        if not lat:
            return float("nan")
        k = min(len(lat) - 1, max(0, int(round(q * (len(lat) - 1)))))
        return lat[k]

    t_end = max((r.t_done for r in results), default=t0)
    span = max(t_end - min((r.t_arrival for r in results), default=t0), 1e-9)
    return {
        "requests": len(results),
        "ok": len(ok),
        "p50_ms": 1e3 * pct(0.50),
        "p99_ms": 1e3 * pct(0.99),
        "mean_ms": 1e3 * (statistics.fmean(lat) if lat else float("nan")),
        "solves_per_s": len(ok) / span,
        "mean_iterations": statistics.fmean(r.iterations for r in ok) if ok else float("nan"),
    }
