"""Python binding of libgs.so (ctypes): argument marshalling only.

Every step of the solve runs in the CUDA library; this module checks shapes, dtypes and
devices of torch tensors, allocates the device workspace the library asks for (torch's
allocator is the only device allocator), and forwards raw pointers and the current CUDA
stream.  The names follow include/gs.h.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2305_08986_gb300.build` "
                      "(or __graft_entry__.build()); there is no fallback implementation")
_lib = ctypes.CDLL(LIB_PATH)

GS_OK, GS_EINVAL, GS_ENOMEM, GS_ECUDA, GS_ENOCONV, GS_EBREAKDOWN, GS_ETIMEOUT, GS_EBUSY = range(8)
(OP_A, OP_RESIDUAL_A, OP_DIAG_A, OP_SMOOTH, OP_RESTRICT, OP_PROLONGATE, OP_B, OP_BT,
 OP_SCHUR_MASS, OP_SCHUR_INV, OP_COARSE, OP_PRECOND, OP_A_RAW, OP_PLAP, OP_PLAP_INV, OP_PRESTRICT,
 OP_PPROLONGATE, OP_SCHUR_DIAG, OP_SADDLE_SMOOTH, OP_SADDLE_VCYCLE, OP_SADDLE_COARSE, OP_CHEB_STEP,
 OP_WAIT_PROBE) = range(23)


class GsMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("len", ctypes.c_double * 3),
                ("cell_void", ctypes.POINTER(ctypes.c_uint8)), ("dirichlet_faces", ctypes.c_uint32)]


class GsOptions(ctypes.Structure):
    _fields_ = [("cheb_degree", ctypes.c_int), ("smooth_steps", ctypes.c_int), ("restart", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("mg_precision", ctypes.c_int), ("schur_degree", ctypes.c_int),
                ("lanczos_steps", ctypes.c_int), ("seed", ctypes.c_int), ("coarse_mode", ctypes.c_int),
                ("schur_kind", ctypes.c_int), ("orth", ctypes.c_int), ("graphs", ctypes.c_int),
                ("plap_degree", ctypes.c_int), ("krylov_fp64", ctypes.c_int), ("tile_autotune", ctypes.c_int),
                ("deflate", ctypes.c_int), ("precond_kind", ctypes.c_int), ("mono_smooth", ctypes.c_int),
                ("mono_cycles", ctypes.c_int), ("corrector", ctypes.c_int)]


class GsInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("dim", ctypes.c_int), ("n_total", ctypes.c_longlong),
                ("n_u", ctypes.c_longlong), ("n_p", ctypes.c_longlong), ("pressure_nullspace", ctypes.c_int),
                ("last_iterations", ctypes.c_int), ("last_rel_residual", ctypes.c_double),
                ("lambda_max", ctypes.c_double * 16), ("level_n_u", ctypes.c_longlong * 16),
                ("coarse_free", ctypes.c_int), ("footprint_bytes", ctypes.c_size_t),
                ("kernel_launches", ctypes.c_longlong), ("schur_cc", ctypes.c_int),
                ("pressure_coarse_free", ctypes.c_int), ("plambda_max", ctypes.c_double * 16),
                ("tile_rows", ctypes.c_int * 16), ("saddle_tile_rows", ctypes.c_int),
                ("deflation_inclusions", ctypes.c_int), ("deflation_modes", ctypes.c_int),
                ("precond_kind", ctypes.c_int), ("saddle_coarse_free", ctypes.c_int)]


class GsKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


_vp = ctypes.c_void_p
_lib.gs_footprint_bytes.restype = ctypes.c_size_t
_lib.gs_footprint_bytes.argtypes = [ctypes.POINTER(GsMesh), ctypes.c_int, ctypes.POINTER(GsOptions)]
_lib.gs_create.restype = ctypes.c_int
_lib.gs_create.argtypes = [ctypes.POINTER(GsMesh), ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                           ctypes.POINTER(GsOptions), _vp, _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]
_lib.gs_create_ex.restype = ctypes.c_int
_lib.gs_create_ex.argtypes = [ctypes.POINTER(GsMesh), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(GsOptions), _vp, _vp, ctypes.c_size_t,
                              ctypes.POINTER(_vp)]
_lib.gs_vmult.restype = ctypes.c_int
_lib.gs_vmult.argtypes = [_vp, _vp, _vp]
_lib.gs_vmult_A.restype = ctypes.c_int
_lib.gs_vmult_A.argtypes = [_vp, _vp, _vp, ctypes.c_int]
_lib.gs_vcycle.restype = ctypes.c_int
_lib.gs_vcycle.argtypes = [_vp, _vp, _vp]
_lib.gs_solve.restype = ctypes.c_int
_lib.gs_solve.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_double)]
_lib.gs_solve_A.restype = ctypes.c_int
_lib.gs_solve_A.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_double)]
_lib.gs_lift_rhs.restype = ctypes.c_int
_lib.gs_lift_rhs.argtypes = [_vp, _vp, _vp, _vp]
_lib.gs_batch_solve.restype = ctypes.c_int
_lib.gs_batch_solve.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                ctypes.c_double, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
_lib.gs_apply_level.restype = ctypes.c_int
_lib.gs_apply_level.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
_lib.gs_get_info.restype = ctypes.c_int
_lib.gs_get_info.argtypes = [_vp, ctypes.POINTER(GsInfo)]
_lib.gs_profile.restype = ctypes.c_int
_lib.gs_profile.argtypes = [_vp, ctypes.c_int]
_lib.gs_profile_read.restype = ctypes.c_int
_lib.gs_profile_read.argtypes = [_vp, ctypes.POINTER(GsKernelStat), ctypes.c_int]
_lib.gs_profile_read_level.restype = ctypes.c_int
_lib.gs_profile_read_level.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(GsKernelStat), ctypes.c_int]
_lib.gs_set_corrector.restype = ctypes.c_int
_lib.gs_set_corrector.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.c_double]
_lib.gs_coarse_solve_noalloc.restype = ctypes.c_int
_lib.gs_coarse_solve_noalloc.argtypes = [_vp, _vp, _vp]
_lib.gs_set_stream.restype = ctypes.c_int
_lib.gs_set_stream.argtypes = [_vp, _vp]
_lib.gs_destroy.restype = None
_lib.gs_destroy.argtypes = [_vp]
_lib.gs_strerror.restype = ctypes.c_char_p
_lib.gs_strerror.argtypes = [ctypes.c_int]
_lib.gs_last_error.restype = ctypes.c_char_p
_lib.gs_last_error.argtypes = []


class GsEngineResult(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_longlong), ("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("t_added", ctypes.c_double), ("t_done", ctypes.c_double)]


class GsEngineStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("batched_launches", ctypes.c_longlong),
                ("plan_builds", ctypes.c_longlong), ("plan_kernels", ctypes.c_longlong),
                ("completed", ctypes.c_longlong)]


_lib.gs_engine_create.restype = ctypes.c_int
_lib.gs_engine_create.argtypes = [ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)]
_lib.gs_engine_add.restype = ctypes.c_int
_lib.gs_engine_add.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_longlong]
_lib.gs_engine_step.restype = ctypes.c_int
_lib.gs_engine_step.argtypes = [_vp, ctypes.POINTER(ctypes.c_int)]
_lib.gs_engine_poll.restype = ctypes.c_int
_lib.gs_engine_poll.argtypes = [_vp, ctypes.POINTER(GsEngineResult), ctypes.c_int]
_lib.gs_engine_active.restype = ctypes.c_int
_lib.gs_engine_active.argtypes = [_vp]
_lib.gs_engine_get_stats.restype = ctypes.c_int
_lib.gs_engine_get_stats.argtypes = [_vp, ctypes.POINTER(GsEngineStats)]
_lib.gs_engine_destroy.restype = None
_lib.gs_engine_destroy.argtypes = [_vp]

EXPORTED = ["gs_footprint_bytes", "gs_create", "gs_create_ex", "gs_vmult", "gs_vmult_A", "gs_vcycle", "gs_solve", "gs_solve_A",
            "gs_lift_rhs",
            "gs_batch_solve", "gs_apply_level", "gs_get_info", "gs_set_stream", "gs_destroy", "gs_strerror",
            "gs_last_error", "gs_profile", "gs_profile_read", "gs_profile_read_level", "gs_coarse_solve_noalloc",
            "gs_set_corrector",
            "gs_engine_create",
            "gs_engine_add", "gs_engine_step", "gs_engine_poll", "gs_engine_active", "gs_engine_get_stats",
            "gs_engine_destroy"]


class GsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.gs_strerror(status).decode()
        detail = _lib.gs_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")


def _check(status: int, where: str, allow=()):
    if status != GS_OK and status not in allow:
        raise GsError(status, where)
    return status


def make_mesh(dim, n, length, cell_void=None, dirichlet_faces=None):
    m = GsMesh()
    m.dim = int(dim)
    for a in range(3):
        m.n[a] = int(n[a]) if a < dim else 1
        m.len[a] = float(length[a]) if a < dim else 1.0
    keep = None
    if cell_void is not None:
        keep = np.ascontiguousarray(np.asarray(cell_void, dtype=np.uint8))
        m.cell_void = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    m.dirichlet_faces = ((1 << (2 * dim)) - 1) if dirichlet_faces is None else int(dirichlet_faces)
    return m, keep


def make_options(**kw):
    o = GsOptions()
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def footprint_bytes(dim, n, length, levels, cell_void=None, dirichlet_faces=None, **opts) -> int:
    m, _keep = make_mesh(dim, n, length, cell_void, dirichlet_faces)
    o = make_options(**opts)
    return int(_lib.gs_footprint_bytes(ctypes.byref(m), int(levels), ctypes.byref(o)))


def _ptr(t, dtype=None, numel=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One generalized Stokes problem resident on the GPU (hierarchy + Krylov workspace)."""

    def __init__(self, dim, n, length, levels, eta, alpha, cell_void=None, dirichlet_faces=None,
                 device="cuda", stream=None, **opts):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.dim = int(dim)
        self.levels = int(levels)
        mesh, keep = make_mesh(dim, n, length, cell_void, dirichlet_faces)
        self._mesh, self._keep = mesh, keep
        o = make_options(**opts)
        nbytes = int(_lib.gs_footprint_bytes(ctypes.byref(mesh), self.levels, ctypes.byref(o)))
        if nbytes == 0:
            raise GsError(GS_EINVAL, "gs_footprint_bytes")
        self.footprint = nbytes
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        eta = np.ascontiguousarray(np.asarray(eta, dtype=np.float64))
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = st
        ctx = ctypes.c_void_p()
        dp = ctypes.POINTER(ctypes.c_double)
        with torch.cuda.device(self.device):
            if np.ndim(alpha) > 0:  # alpha per cell (gs_create_ex)
                al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
                if al.shape != eta.shape:
                    raise ValueError("alpha: a scalar or one value per cell")
                _check(_lib.gs_create_ex(ctypes.byref(mesh), self.levels, eta.ctypes.data_as(dp),
                                         al.ctypes.data_as(dp), ctypes.byref(o), ctypes.c_void_p(st.cuda_stream),
                                         ctypes.c_void_p(self._ws_ptr), ctypes.c_size_t(nbytes), ctypes.byref(ctx)),
                       "gs_create_ex")
            else:
                _check(_lib.gs_create(ctypes.byref(mesh), self.levels, eta.ctypes.data_as(dp), float(alpha),
                                      ctypes.byref(o), ctypes.c_void_p(st.cuda_stream), ctypes.c_void_p(self._ws_ptr),
                                      ctypes.c_size_t(nbytes), ctypes.byref(ctx)), "gs_create")
        self.ctx = ctx
        info = self.info()
        self.n_total, self.n_u, self.n_p = info.n_total, info.n_u, info.n_p

    @classmethod
    def from_problem(cls, p, device="cuda", stream=None, levels=None, **opts):
        return cls(p.dim, p.n, p.length, p.levels if levels is None else levels, p.eta, p.alpha,
                   p.void, p.dirichlet_faces, device=device, stream=stream, **opts)

    # ---- operations ----
    def vmult(self, x, y):
        T = self.torch.float64
        _check(_lib.gs_vmult(self.ctx, _ptr(x, T, self.n_total, "x"), _ptr(y, T, self.n_total, "y")), "gs_vmult")

    def vmult_A(self, x, y):
        fp32 = x.dtype == self.torch.float32
        T = self.torch.float32 if fp32 else self.torch.float64
        _check(_lib.gs_vmult_A(self.ctx, _ptr(x, T, self.n_u, "x"), _ptr(y, T, self.n_u, "y"), int(fp32)),
               "gs_vmult_A")

    def vcycle(self, r, z):
        T = self.torch.float64
        _check(_lib.gs_vcycle(self.ctx, _ptr(r, T, self.n_u, "r"), _ptr(z, T, self.n_u, "z")), "gs_vcycle")

    def solve(self, rhs, x, tol=1e-8, allow_noconv=False):
        T = self.torch.float64
        it = ctypes.c_int()
        rel = ctypes.c_double()
        s = _lib.gs_solve(self.ctx, _ptr(rhs, T, self.n_total, "rhs"), _ptr(x, T, self.n_total, "x"), float(tol),
                          ctypes.byref(it), ctypes.byref(rel))
        _check(s, "gs_solve", allow=(GS_ENOCONV,) if allow_noconv else ())
        return it.value, rel.value, s

    def solve_A(self, rhs, x, tol=1e-6, allow_noconv=False):
        """Mesh-extension solve A x = rhs on the velocity block (length d*N_v), CG + V-cycle."""
        T = self.torch.float64
        it = ctypes.c_int()
        rel = ctypes.c_double()
        s = _lib.gs_solve_A(self.ctx, _ptr(rhs, T, self.n_u, "rhs"), _ptr(x, T, self.n_u, "x"), float(tol),
                            ctypes.byref(it), ctypes.byref(rel))
        _check(s, "gs_solve_A", allow=(GS_ENOCONV,) if allow_noconv else ())
        return it.value, rel.value, s

    def lift_rhs(self, f, g, rhs):
        T = self.torch.float64
        _check(_lib.gs_lift_rhs(self.ctx, _ptr(f, T, self.n_total, "f"), _ptr(g, T, self.n_total, "g"),
                                _ptr(rhs, T, self.n_total, "rhs")), "gs_lift_rhs")

    def apply_level(self, level, op, x, y, aux=None, prec=None):
        if prec is None:
            prec = 32 if y.dtype == self.torch.float32 else 64
        xp = _ptr(x, name="x") if x is not None else None
        ap = _ptr(aux, name="aux") if aux is not None else None
        _check(_lib.gs_apply_level(self.ctx, int(level), int(op), int(prec), xp, _ptr(y, name="y"), ap),
               "gs_apply_level")

    def info(self):
        inf = GsInfo()
        _check(_lib.gs_get_info(self.ctx, ctypes.byref(inf)), "gs_get_info")
        return inf

    def profile(self, enable: bool):
        _check(_lib.gs_profile(self.ctx, int(bool(enable))), "gs_profile")

    def profile_read(self, level=None):
        """{class: (launches, device ms)} over all launches, or over those of one multigrid level
        (level=-1: launches tied to no level)."""
        arr = (GsKernelStat * 32)()
        if level is None:
            n = _lib.gs_profile_read(self.ctx, arr, 32)
        else:
            n = _lib.gs_profile_read_level(self.ctx, int(level), arr, 32)
        return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n)}

    def set_corrector(self, vcirc=None, rho=0.0):
        """Corrector stage with the given convective field v° (numpy, d N_v entries of the finest
        level); None returns to the predictor stage (gs_set_corrector)."""
        if vcirc is None:
            _check(_lib.gs_set_corrector(self.ctx, None, 0.0), "gs_set_corrector")
            return
        v = np.ascontiguousarray(np.asarray(vcirc, dtype=np.float64))
        if v.shape != (self.n_u,):
            raise ValueError(f"vcirc: expected {self.n_u} entries, got {v.shape}")
        _check(_lib.gs_set_corrector(self.ctx, v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(rho)),
               "gs_set_corrector")

    def set_stream(self, stream):
        self.stream = stream
        _check(_lib.gs_set_stream(self.ctx, ctypes.c_void_p(stream.cuda_stream)), "gs_set_stream")

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.torch.cuda.current_stream(self.device).synchronize()
            _lib.gs_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_solve(solvers, rhs_list, x_list, tol=1e-8):
    n = len(solvers)
    ctxs = (ctypes.c_void_p * n)(*[s.ctx.value for s in solvers])
    rp = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rhs_list])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in x_list])
    its = (ctypes.c_int * n)()
    rels = (ctypes.c_double * n)()
    s = _lib.gs_batch_solve(ctxs, n, rp, xp, float(tol), its, rels)
    return s, list(its), list(rels)


class Engine:
    """Batching engine (gs_engine_*): many solves advanced together, one FGMRES iteration of each
    per step, one launch per kernel per step for all of them."""

    def __init__(self, max_slots, max_restart=0, stream=None, device="cuda"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.stream = st
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(_lib.gs_engine_create(int(max_slots), int(max_restart), ctypes.c_void_p(st.cuda_stream),
                                         ctypes.byref(h)), "gs_engine_create")
        self.h = h
        self.max_slots = int(max_slots)
        self._held = {}  # tag -> (solver, rhs, x): kept alive while the solve runs

    def add(self, solver, rhs, x, tol=1e-8, tag=0):
        """Queue a solve; returns False when every slot is taken."""
        T = self.torch.float64
        s = _lib.gs_engine_add(self.h, solver.ctx, _ptr(rhs, T, solver.n_total, "rhs"),
                               _ptr(x, T, solver.n_total, "x"), float(tol), int(tag))
        if s == GS_EBUSY:
            return False
        _check(s, "gs_engine_add")
        self._held[int(tag)] = (solver, rhs, x)
        return True

    def step(self):
        """One iteration of every solve in the engine; returns the number still running."""
        n = ctypes.c_int()
        _check(_lib.gs_engine_step(self.h, ctypes.byref(n)), "gs_engine_step")
        return n.value

    def poll(self, max_results=4096):
        arr = (GsEngineResult * max_results)()
        n = _lib.gs_engine_poll(self.h, arr, max_results)
        out = []
        for i in range(n):
            r = arr[i]
            out.append({"tag": r.tag, "status": r.status, "iterations": r.iterations,
                        "rel_residual": r.rel_residual, "t_added": r.t_added, "t_done": r.t_done})
            self._held.pop(int(r.tag), None)
        return out

    def active(self):
        return int(_lib.gs_engine_active(self.h))

    def stats(self):
        st = GsEngineStats()
        _check(_lib.gs_engine_get_stats(self.h, ctypes.byref(st)), "gs_engine_get_stats")
        return {k: getattr(st, k) for k, _ in GsEngineStats._fields_}

    def run(self):
        """Step until every solve has finished; returns the finished solves."""
        out = []
        while self.active() > 0:
            self.step()
            out.extend(self.poll())
        out.extend(self.poll())
        return out

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.gs_engine_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
