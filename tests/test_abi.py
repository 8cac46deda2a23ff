"""CPU checks of the C-ABI library: it builds, loads, and exports every entry point the header declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_A-Z0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2305_08986_gb300 import build
    return build.build(verbose=False)


def test_header_declares_the_path():
    names = _declared()
    for n in ["gs_create", "gs_vmult", "gs_vmult_A", "gs_vcycle", "gs_solve", "gs_lift_rhs",
              "gs_footprint_bytes", "gs_batch_solve", "gs_destroy", "gs_strerror", "gs_apply_level"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gs_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binds(lib_path):
    from paper_2305_08986_gb300 import gs
    for n in _declared():
        assert hasattr(gs._lib, n)
    assert set(gs.EXPORTED) == set(_declared())
    assert gs._lib.gs_strerror(gs.GS_ENOCONV) == b"no convergence"


def test_footprint_host_logic(lib_path):
    from paper_2305_08986_gb300 import gs
    a = gs.footprint_bytes(2, (16, 16), (1.0, 1.0), 3)
    b = gs.footprint_bytes(2, (16, 16), (1.0, 1.0), 3, mg_precision=64)
    c = gs.footprint_bytes(2, (32, 32), (1.0, 1.0), 3)
    assert 0 < a < b and a < c
    # invalid inputs are rejected on the host without touching a GPU
    assert gs.footprint_bytes(2, (15, 16), (1.0, 1.0), 2) == 0      # not coarsenable
    assert gs.footprint_bytes(1, (16,), (1.0,), 1) == 0              # unsupported dimension
    assert gs.footprint_bytes(3, (8, 8, 8), (1.0, 1.0, 1.0), 20) == 0


def test_engine_argument_checks(lib_path):
    """Host-side validation of the batching engine entry points (no CUDA call is reached)."""
    import ctypes
    from paper_2305_08986_gb300 import gs
    h = ctypes.c_void_p()
    assert gs._lib.gs_engine_create(0, 0, None, ctypes.byref(h)) == gs.GS_EINVAL
    assert gs._lib.gs_engine_create(70000, 0, None, ctypes.byref(h)) == gs.GS_EINVAL
    assert gs._lib.gs_engine_add(None, None, None, None, 1e-8, 0) == gs.GS_EINVAL
    assert gs._lib.gs_engine_step(None, None) == gs.GS_EINVAL
    assert gs._lib.gs_engine_poll(None, None, 4) == 0
    assert gs._lib.gs_engine_active(None) == 0
    assert gs._lib.gs_strerror(gs.GS_EBUSY) == b"busy (no free slot)"


def test_new_entry_points_reject_bad_arguments_on_the_host(lib_path):
    """gs_create_ex, gs_solve_A and the saddle-point multigrid options are validated before any
    CUDA call: NULL pointers, a missing alpha array, deflation with precond_kind 1."""
    import ctypes
    import numpy as np
    from paper_2305_08986_gb300 import gs
    m, _keep = gs.make_mesh(2, (16, 16), (1.0, 1.0))
    eta = np.ones(256)
    dp = ctypes.POINTER(ctypes.c_double)
    ctx = ctypes.c_void_p()
    o = gs.make_options()
    # alpha_per_cell NULL
    assert gs._lib.gs_create_ex(ctypes.byref(m), 3, eta.ctypes.data_as(dp), None, ctypes.byref(o), None,
                                ctypes.c_void_p(256), ctypes.c_size_t(1 << 40), ctypes.byref(ctx)) == gs.GS_EINVAL
    # negative alpha on an active cell
    al = np.ones(256)
    al[7] = -1.0
    assert gs._lib.gs_create_ex(ctypes.byref(m), 3, eta.ctypes.data_as(dp), al.ctypes.data_as(dp), ctypes.byref(o),
                                None, ctypes.c_void_p(256), ctypes.c_size_t(1 << 40), ctypes.byref(ctx)) == gs.GS_EINVAL
    # deflation belongs to the block-triangular preconditioner
    o2 = gs.make_options(precond_kind=1, deflate=1)
    assert gs._lib.gs_create(ctypes.byref(m), 3, eta.ctypes.data_as(dp), 1.0, ctypes.byref(o2), None,
                             ctypes.c_void_p(256), ctypes.c_size_t(1 << 40), ctypes.byref(ctx)) == gs.GS_EINVAL
    assert gs._lib.gs_solve_A(None, None, None, 1e-6, None, None) == gs.GS_EINVAL
    # the saddle-point multigrid reserves its level vectors and coarse inverse in the workspace
    a = gs.footprint_bytes(2, (16, 16), (1.0, 1.0), 3)
    b = gs.footprint_bytes(2, (16, 16), (1.0, 1.0), 3, precond_kind=1)
    c = gs.footprint_bytes(2, (16, 16), (1.0, 1.0), 3, precond_kind=1, mono_cycles=2)
    assert 0 < a < b < c
