"""The C-ABI library builds, loads and exports every symbol include/vrps.h declares; host-side
argument checks reject bad input before any CUDA call (CPU only, no compute)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vrps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vrps_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    b = __graft_entry__._build_module()
    b.build()
    return ctypes.CDLL(b.LIB)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("vrps_proj_fwd", "vrps_proj_adj", "vrps_prox_tv", "vrps_solve", "vrps_geom_par2d",
                 "vrps_geom_cone3d"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_exports_same_names():
    import paper_2602_09527_gb300 as vr
    for name in ("proj_fwd", "proj_adj", "prox_tv", "solve", "power_iteration", "objective",
                 "philox_schedule"):
        assert callable(getattr(vr, name))


def _err(lib):
    lib.vrps_last_error.restype = ctypes.c_char_p
    return lib.vrps_last_error().decode()


def test_invalid_geometry_rejected_on_host(lib):
    h = ctypes.c_void_p()
    ang = (ctypes.c_double * 2)(0.0, 1.0)
    f = lib.vrps_geom_par2d
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                  ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    assert f(0, 8, 1.0, 2, ang, 8, 1.0, 1, ctypes.byref(h)) == -1
    assert "positive" in _err(lib)
    assert f(8, 8, -1.0, 2, ang, 8, 1.0, 1, ctypes.byref(h)) == -1
    assert f(8, 8, 1.0, 2, ang, 8, 1.0, 3, ctypes.byref(h)) == -1      # N > angles
    assert f(8, 8, 1.0, 2, None, 8, 1.0, 1, ctypes.byref(h)) == -1
    nan = (ctypes.c_double * 2)(0.0, float("nan"))
    assert f(8, 8, 1.0, 2, nan, 8, 1.0, 1, ctypes.byref(h)) == -1
    assert h.value is None


def test_invalid_cone_rejected_on_host(lib):
    h = ctypes.c_void_p()
    b = (ctypes.c_double * 4)(0.0, 1.0, 2.0, 3.0)
    f = lib.vrps_geom_cone3d
    f.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + \
                 [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    # source inside the volume
    assert f(16, 16, 16, 1.0, 4, b, 8, 8, 1.0, 1.0, 5.0, 10.0, 1, ctypes.byref(h)) == -1
    assert "source" in _err(lib)
    # sdd <= sod
    assert f(16, 16, 16, 1.0, 4, b, 8, 8, 1.0, 1.0, 50.0, 40.0, 1, ctypes.byref(h)) == -1


def test_null_handles_rejected(lib):
    lib.vrps_proj_fwd.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.vrps_proj_fwd(None, 0, None, None, None) == -1
    lib.vrps_philox_schedule.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.vrps_philox_schedule(1, 0, 0, -1, 4, 0.5, None, None) == -1
    assert lib.vrps_geom_free(None) == 0


def test_check_error_rejects_null_handle(lib):
    lib.vrps_check_error.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.vrps_check_error(None, None) == -1


def test_batch_scheduling_knobs_reject_bad_input(lib):
    lib.vrps_batch_set_grid_share.argtypes = [ctypes.c_void_p, ctypes.c_double]
    lib.vrps_batch_set_stream_priority.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.vrps_batch_set_grid_share(None, 0.5) == -1
    assert lib.vrps_batch_set_stream_priority(None, 0) == -1


def test_status_codes_match_header():
    """The binding names every status code the header defines, and nothing else."""
    src = open(os.path.join(ROOT, "include", "vrps.h")).read()
    codes = {int(v): k for k, v in re.findall(r"VRPS_(OK|ERR_[A-Z_]+)\s*=\s*(-?\d+)", src)}
    from paper_2602_09527_gb300 import _binding
    assert {c: n.replace("ERR_", "") for c, n in codes.items()} == _binding.STATUS


def test_selftest_rejects_bad_poll_counts_on_host(lib):
    lib.vrps_selftest_bounded_wait.argtypes = [ctypes.c_uint32, ctypes.c_void_p]
    assert lib.vrps_selftest_bounded_wait(0, None) == -1
    assert lib.vrps_selftest_bounded_wait((1 << 24) + 1, None) == -1
    assert "polls" in _err(lib)
