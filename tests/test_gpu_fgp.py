"""FGP-TV prox: CUDA path vs the float64 oracle at a fixed number of inner iterations from the
same warm start (2D and 3D), including the returned dual.  Tolerance 1e-5 relative L2."""
import math

import numpy as np
import pytest

from tests._gpu import dev, host, need_gpu, rel, torch

from oracle import tv

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _geom2(nx, ny):
    need_gpu()
    import paper_2602_09527_gb300 as vr
    return vr, vr.Geometry.par2d(nx, ny, 1.0, [0.0], 4, 1.0, 1)


def _geom3(nx, ny, nz):
    need_gpu()
    import paper_2602_09527_gb300 as vr
    return vr, vr.Geometry.cone3d(nx, ny, nz, 1.0, [0.0, 1.0], 8, 8, 1.0, 1.0, 10.0 * max(nx, ny), 20.0 * max(nx, ny), 1)


@pytest.mark.parametrize("shape", [(64, 64), (53, 37), (8, 129), (1, 1), (2, 1)])
@pytest.mark.parametrize("iters", [0, 1, 2, 7, 50])
def test_fgp2d_cold(shape, iters):
    ny, nx = shape
    vr, g = _geom2(nx, ny)
    v = np.random.default_rng(iters + nx).uniform(-0.3, 1.0, size=shape)
    for nonneg in (True, False):
        x = vr.prox_tv(g, dev(v), 0.07, iters, nonneg=nonneg)
        ref, _ = tv.fgp(v, 0.07, iters, nonneg=nonneg)
        assert rel(host(x), ref) < TOL or np.max(np.abs(host(x) - ref.ravel())) < 1e-6


@pytest.mark.parametrize("iters", [1, 3, 100])
def test_fgp2d_warm_dual_roundtrip(iters):
    vr, g = _geom2(45, 31)
    rng = np.random.default_rng(5)
    v = rng.uniform(0, 1, size=(31, 45))
    w0 = rng.standard_normal(2 * 31 * 45)
    w0 = (w0.reshape(2, -1) / np.maximum(1.0, np.sqrt((w0.reshape(2, -1) ** 2).sum(0)))).ravel()
    d = dev(w0)
    x = vr.prox_tv(g, dev(v), 0.2, iters, dual=d)
    ref, wref = tv.fgp(v, 0.2, iters, w0=w0)
    assert rel(host(x), ref) < TOL
    assert rel(host(d), wref) < TOL
    # a second call warm-starts from the returned dual (its momentum restarts at t = 1)
    x2 = vr.prox_tv(g, dev(v), 0.2, iters, dual=d)
    ref2, _ = tv.fgp(v, 0.2, iters, w0=wref)
    assert rel(host(x2), ref2) < TOL


def test_fgp2d_full_size_100_iters():
    vr, g = _geom2(512, 512)
    v = np.random.default_rng(9).uniform(0, 1, size=(512, 512))
    x = vr.prox_tv(g, dev(v), 0.01, 100)
    ref, _ = tv.fgp(v, 0.01, 100)
    assert rel(host(x), ref) < TOL


@pytest.mark.parametrize("shape", [(16, 20, 24), (5, 33, 9), (1, 1, 3), (130, 37, 70)])
@pytest.mark.parametrize("iters", [0, 1, 4, 30])
def test_fgp3d(shape, iters):
    nz, ny, nx = shape
    vr, g = _geom3(nx, ny, nz)
    rng = np.random.default_rng(iters + nz)
    v = rng.uniform(-0.2, 1.0, size=shape)
    w0 = rng.standard_normal(3 * v.size) * 0.3
    w0 = (w0.reshape(3, -1) / np.maximum(1.0, np.sqrt((w0.reshape(3, -1) ** 2).sum(0)))).ravel()
    d = dev(w0)
    x = vr.prox_tv(g, dev(v), 0.05, iters, dual=d)
    ref, wref = tv.fgp(v, 0.05, iters, w0=w0)
    assert rel(host(x), ref) < TOL
    assert rel(host(d), wref) < TOL or iters == 0


def test_prox_rejects_bad_args():
    vr, g = _geom2(8, 8)
    v = torch.zeros(64, device="cuda")
    with pytest.raises(vr.VrpsError):
        vr.prox_tv(g, v, -1.0, 5)
    with pytest.raises(vr.VrpsError):
        vr.prox_tv(g, v, 0.1, -1)
    with pytest.raises(vr.VrpsError):
        vr.prox_tv(g, v, 0.1, 3, x=v)


def test_fgp3d_after_autotune():
    """The 3D autotuner picks the streaming chunk; the prox still matches the oracle, also with
    chunks that do not divide the volume."""
    vr, g = _geom3(40, 24, 75)
    t = vr.autotune(g, reps=1)
    assert t["fgp3d_chunk_planes"] in (4, 8, 16, 32, 64, 128)
    rng = np.random.default_rng(17)
    v = rng.uniform(-0.2, 1.0, size=(75, 24, 40))
    x = vr.prox_tv(g, dev(v), 0.05, 12)
    ref, _ = tv.fgp(v, 0.05, 12)
    assert rel(host(x), ref) < TOL


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(70, 45), (16, 130), (300, 170)])
def test_fgp2d_tiles(tile, shape):
    """The 2D output tiles (the 32-wide one 32 or 27 rows high, chosen for the SM count, or
    either by hand; 32 x 16; 16 x 16) give the oracle's K-step FGP."""
    vr, g = _geom2(shape[1], shape[0])
    vr.set_launch_shape(g, fgp_tile=tile)
    rng = np.random.default_rng(tile + shape[0])
    v = rng.uniform(-0.2, 1.0, size=shape)
    w0 = rng.standard_normal(2 * v.size) * 0.3
    w0 = (w0.reshape(2, -1) / np.maximum(1.0, np.sqrt((w0.reshape(2, -1) ** 2).sum(0)))).ravel()
    d = dev(w0)
    x = vr.prox_tv(g, dev(v), 0.05, 21, dual=d)
    ref, wref = tv.fgp(v, 0.05, 21, w0=w0)
    assert rel(host(x), ref) < TOL
    assert rel(host(d), wref) < TOL


@pytest.mark.parametrize("shape", [(512, 512), (1024, 1024), (200, 333)])
def test_fgp2d_tiles_same_bits(shape):
    """Temporal blocking recomputes the halo with the same operations, so every output tile
    (and the balanced height the 32-wide tile takes at these sizes) gives identical bits,
    dual included, and the result is the oracle's."""
    vr, g = _geom2(shape[1], shape[0])
    rng = np.random.default_rng(shape[0])
    v = rng.uniform(-0.2, 4.0, size=shape)
    outs = []
    for tile in (0, 1, 2, 3, 4):
        vr.set_launch_shape(g, fgp_tile=tile)
        d = torch.zeros(2 * v.size, device="cuda")
        x = vr.prox_tv(g, dev(v), 1.0, 20, dual=d)
        outs.append((x.clone(), d.clone()))
    for x, d in outs[1:]:
        assert torch.equal(x, outs[0][0]) and torch.equal(d, outs[0][1])
    ref, _ = tv.fgp(v, 1.0, 20)
    assert rel(host(outs[0][0]), ref) < TOL
