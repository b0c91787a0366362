"""The allocation-free 2D prox entry point, called through the C ABI.

vrps_prox_tv2d_noalloc is for callers that cannot let the library allocate device memory
(an application owning the whole device budget through its own pool, or a latency-critical
loop that cannot afford cudaMalloc's implicit synchronisation).  Its scratch is a fixed
device array shared by every call, so these checks make two calls in a row and compare each
with the allocating entry point vrps_prox_tv on the same inputs.  This file is collected last
so that a run stopping at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from tests._gpu import dev, host, need_gpu, rel, torch

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _lib():
    need_gpu()
    import paper_2602_09527_gb300 as vr
    lib = vr.lib
    lib.vrps_prox_tv2d_noalloc.restype = ctypes.c_int
    lib.vrps_prox_tv2d_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_float, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p]
    return vr, lib


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _noalloc(lib, nx, ny, v, x, tau, iters, nonneg, dual):
    code = lib.vrps_prox_tv2d_noalloc(nx, ny, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                      float(tau), int(iters), int(nonneg),
                                      ctypes.c_void_p(dual.data_ptr()) if dual is not None else None, _stream())
    assert code == 0, lib.vrps_last_error()


@pytest.mark.parametrize("nx,ny", [(512, 512), (37, 53)])
def test_noalloc_matches_prox_tv_twice(nx, ny):
    vr, lib = _lib()
    g = vr.Geometry.par2d(nx, ny, 1.0, [0.0], 4, 1.0, 1)
    rng = np.random.default_rng(nx)
    for call in range(2):                      # two calls in a row share the fixed scratch
        v = dev(rng.uniform(-0.2, 1.0, size=nx * ny))
        tau, iters = 0.03 + 0.02 * call, 20 + 17 * call
        x_ref = vr.prox_tv(g, v, tau, iters, nonneg=True)
        x = torch.empty_like(v)
        _noalloc(lib, nx, ny, v, x, tau, iters, 1, None)          # cold start
        torch.cuda.synchronize()
        assert rel(host(x), host(x_ref)) < TOL
        # warm start: the returned dual matches too
        w0 = rng.standard_normal(2 * nx * ny) * 0.2
        d_ref, d_new = dev(w0), dev(w0)
        x_ref = vr.prox_tv(g, v, tau, iters, nonneg=False, dual=d_ref)
        _noalloc(lib, nx, ny, v, x, tau, iters, 0, d_new)
        torch.cuda.synchronize()
        assert rel(host(x), host(x_ref)) < TOL
        assert rel(host(d_new), host(d_ref)) < TOL
    g.close()


def test_noalloc_rejects_oversize():
    vr, lib = _lib()
    v = torch.zeros(4, device="cuda")
    code = lib.vrps_prox_tv2d_noalloc(1024, 1024, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(v.data_ptr() + 4),
                                      0.1, 3, 1, None, _stream())
    assert code == -1
    assert b"capacity" in lib.vrps_last_error()
