"""2D parallel-beam projector: CUDA path (through the C ABI) vs the float64 oracle.

Tolerance: relative L2 error of a single FP32 projection <= 1e-5 against float64.
Geometries span several tiles and ragged edges (odd sizes, unequal subsets, pixel and
bin spacings != 1, angles exactly at 0, 45 and 90 degrees)."""
import math

import numpy as np
import pytest

from tests._gpu import dev, host, need_gpu, rel, torch

import synthetic
from oracle import joseph2d as J

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _vr():
    need_gpu()
    import paper_2602_09527_gb300 as vr
    return vr


GEOMS = {
    "par2d_64": dict(nx=64, ny=64, pixel=1.0, angles=synthetic.uniform_angles(90, math.pi), nb=96, ds=1.0, N=10),
    "ragged": dict(nx=37, ny=53, pixel=0.9, angles=np.concatenate([synthetic.uniform_angles(43, math.pi),
                                                                   [math.pi / 4, math.pi / 2, 0.0, 3 * math.pi / 4]]),
                   nb=61, ds=1.1, N=4),
    "fine_bins": dict(nx=40, ny=24, pixel=1.0, angles=synthetic.uniform_angles(30, math.pi), nb=120, ds=0.45, N=3),
}


def _pair(name):
    vr = _vr()
    p = GEOMS[name]
    g = vr.Geometry.par2d(p["nx"], p["ny"], p["pixel"], p["angles"], p["nb"], p["ds"], p["N"])
    og = J.Geometry2D(p["nx"], p["ny"], p["pixel"], p["angles"], p["nb"], p["ds"], p["N"])
    return vr, g, og


@pytest.mark.parametrize("name", list(GEOMS))
def test_forward_every_subset(name):
    vr, g, og = _pair(name)
    x = np.random.default_rng(1).uniform(size=(og.ny, og.nx))
    for i in list(range(og.n_subsets)) + [-1]:
        ids = og.all_angles() if i == -1 else og.subset(i)
        y = vr.proj_fwd(g, i, dev(x))
        assert rel(host(y), J.forward(og, x, ids)) < TOL, (name, i)


@pytest.mark.parametrize("name", list(GEOMS))
def test_adjoint_every_subset(name):
    vr, g, og = _pair(name)
    rng = np.random.default_rng(2)
    for i in list(range(og.n_subsets)) + [-1]:
        ids = og.all_angles() if i == -1 else og.subset(i)
        r = rng.standard_normal((len(ids), og.n_bins))
        x = vr.proj_adj(g, i, dev(r))
        assert rel(host(x), J.adjoint(og, r, ids)) < TOL, (name, i)


@pytest.mark.parametrize("name", list(GEOMS))
def test_adjoint_identity_fp32(name):
    vr, g, og = _pair(name)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(og.n)
    y = rng.standard_normal(og.m)
    Ax = host(vr.proj_fwd(g, -1, dev(x)))
    ATy = host(vr.proj_adj(g, -1, dev(y)))
    xf = x.astype(np.float32).astype(np.float64)
    yf = y.astype(np.float32).astype(np.float64)
    lhs, rhs = float(Ax @ yf), float(xf @ ATy)
    scale = float(np.abs(Ax).sum() * np.abs(yf).max())
    assert abs(lhs - rhs) <= 2e-6 * scale


def test_dense_matrix_small():
    """Every column of A and every row of A^T from unit vectors, against the oracle's dense A."""
    vr = _vr()
    ang = [0.0, 0.3, math.pi / 4, 1.1, math.pi / 2, 2.0, 3 * math.pi / 4, 2.9]
    g = vr.Geometry.par2d(6, 5, 1.0, ang, 9, 1.0, 2)
    og = J.Geometry2D(6, 5, 1.0, ang, 9, 1.0, 2)
    A = J.dense_matrix(og)
    cols = torch.eye(og.n, device="cuda", dtype=torch.float32)
    G = np.stack([host(vr.proj_fwd(g, -1, cols[c].contiguous())) for c in range(og.n)], axis=1)
    assert np.max(np.abs(G - A)) < 1e-5
    rows = torch.eye(og.m, device="cuda", dtype=torch.float32)
    GT = np.stack([host(vr.proj_adj(g, -1, rows[r].contiguous())) for r in range(og.m)], axis=0)
    assert np.max(np.abs(GT - A)) < 1e-5


def test_degenerate_sizes():
    vr = _vr()
    for (nx, ny, nb, ang) in ((1, 1, 1, [0.0]), (1, 7, 3, [0.2, 1.4]), (9, 1, 5, [math.pi / 2]),
                              (3, 3, 1, [math.pi / 4])):
        g = vr.Geometry.par2d(nx, ny, 1.0, ang, nb, 1.0, 1)
        og = J.Geometry2D(nx, ny, 1.0, ang, nb, 1.0, 1)
        x = np.random.default_rng(nx * 10 + ny).uniform(size=(ny, nx))
        y = host(vr.proj_fwd(g, -1, dev(x)))
        ref = J.forward(og, x, og.all_angles())
        assert np.max(np.abs(y - ref.ravel())) < 1e-5 * max(1.0, np.abs(ref).max())
        r = np.random.default_rng(5).standard_normal(og.m)
        a = host(vr.proj_adj(g, -1, dev(r)))
        ref = J.adjoint(og, r.reshape(len(ang), nb), og.all_angles())
        assert np.max(np.abs(a - ref.ravel())) < 1e-5 * max(1.0, np.abs(ref).max())


def test_check_error_clear_after_projections():
    """The forward's bounded bulk-copy waits never expire in normal work: after projections of
    every subset the handle's device error word reads clear (vrps_check_error)."""
    vr, g, og = _pair("par2d_64")
    x = dev(np.random.default_rng(3).uniform(size=(og.ny, og.nx)))
    for i in list(range(og.n_subsets)) + [-1]:
        vr.proj_fwd(g, i, x)
    vr.check_error(g)


def test_bad_subset_raises():
    vr, g, og = _pair("par2d_64")
    x = torch.zeros(og.n, device="cuda")
    with pytest.raises(vr.VrpsError):
        vr.proj_fwd(g, og.n_subsets, x, torch.zeros(10, device="cuda"))


def test_full_size_512_sampled_angles():
    """512^2, 720 angles, 768 bins, 20 subsets: the full forward on the GPU, checked row by
    row on a sample of angles (both marching orientations, 45 and 90 degrees); the full
    adjoint checked on single-angle sinograms and by the adjoint identity."""
    vr = _vr()
    spec = synthetic.Par2DSpec(512, 512, 1.0, synthetic.uniform_angles(720, math.pi), 768, 1.0, 20)
    g = vr.Geometry.from_spec(spec)
    og = J.Geometry2D.from_spec(spec)
    x = synthetic.rasterize_ellipses(synthetic.random_ellipses(10, 256.0, np.random.default_rng(7)),
                                     512, 512, 1.0)
    y = host(vr.proj_fwd(g, -1, dev(x))).reshape(720, 768)
    sample = [0, 1, 97, 180, 263, 360, 500, 719]
    ref = J.forward(og, x, sample)
    for k, a in enumerate(sample):
        assert rel(y[a], ref[k]) < TOL, a
    # adjoint of a sinogram supported on a few angles
    rng = np.random.default_rng(8)
    r = np.zeros((720, 768))
    r[sample] = rng.standard_normal((len(sample), 768))
    xa = host(vr.proj_adj(g, -1, dev(r)))
    assert rel(xa, J.adjoint(og, r[sample], sample)) < TOL
    # subset forward equals the matching rows of the full forward (same kernels, same rays)
    ys = host(vr.proj_fwd(g, 7, dev(x))).reshape(-1, 768)
    assert np.array_equal(ys, y[og.subset(7)])


def test_autotuned_shapes_keep_parity():
    """vrps_autotune picks a forward band and adjoint shape by timing; the tuned projector
    still matches the oracle at every candidate's tolerance."""
    vr = _vr()
    spec = synthetic.Par2DSpec(256, 192, 1.0, synthetic.uniform_angles(120, math.pi), 300, 1.0, 6)
    g = vr.Geometry.from_spec(spec)
    og = J.Geometry2D.from_spec(spec)
    t = vr.autotune(g, reps=2)
    assert t["fwd_band_bytes"] in (16 << 10, 24 << 10, 32 << 10, 48 << 10, 64 << 10, 96 << 10)
    assert t["adj_pixels_per_thread"] in (1, 2) and t["fwd_adj_us"] > 0
    rng = np.random.default_rng(31)
    x = rng.uniform(0, 1, size=(192, 256))
    rows = list(range(2, 120, 6))
    y = host(vr.proj_fwd(g, 2, dev(x))).reshape(len(rows), 300)
    assert rel(y, J.forward(og, x, rows)) < TOL
    r = rng.standard_normal((len(rows), 300))
    assert rel(host(vr.proj_adj(g, 2, dev(r))), J.adjoint(og, r, rows)) < TOL
    # the all-angle passes got their own shapes, timed on the full sinogram
    full = t["all_angles"]
    assert full["fwd_band_bytes"] in (16 << 10, 24 << 10, 32 << 10, 48 << 10, 64 << 10, 96 << 10)
    assert full["fwd_bands_per_cta"] in (1, 2, 4, 8) and full["adj_angle_shares"] in (1, 2, 4, 8)
    yf = host(vr.proj_fwd(g, -1, dev(x))).reshape(120, 300)
    assert rel(yf, J.forward(og, x, list(range(120)))) < TOL
    rf = rng.standard_normal((120, 300))
    assert rel(host(vr.proj_adj(g, -1, dev(rf))), J.adjoint(og, rf, list(range(120)))) < TOL
    # a batched job on the tuned geometry (snapshot passes with the all-angle shapes) equals
    # vrps_solve on it, bit for bit
    b = dev(J.forward(og, x, list(range(120))))
    L = vr.power_iteration(g, 30, seed=1)
    kw = dict(p=0.3, gamma=1 / L, seed=12, estimator="SVRG", fgp_iters=9, max_iters=20)
    xs, _, _ = vr.solve(b, g, 0.01, "VR_PROXSKIP", **kw)
    xs = xs.clone()
    B = vr.Batch()
    jid = B.submit(g, b, alpha=0.01, **kw)
    B.wait(jid)
    assert torch.equal(B.result(jid), xs)
    B.close()
    # setting shapes by hand applies them to every pass again
    vr.set_launch_shape(g)
    assert vr.launch_shape_full(g) == [0, 0, 0]


@pytest.mark.parametrize("shape", [(16 << 10, 1, 1, 1), (16 << 10, 3, 2, 2), (24 << 10, 4, 1, 3), (48 << 10, 8, 2, 4),
                                   (8 << 10, 2, 2, 7)])
@pytest.mark.parametrize("dims", [(200, 136, 150), (96, 250, 180), (90, 90, 130)])
def test_forward_band_groups_keep_parity(shape, dims):
    """Forward bands walked several per CTA (double-buffered copies, rays kept in registers) and
    adjoint tiles split into angle shares, on non-square images where the two marching
    orientations have different line counts and a side that is not a multiple of 4 (plain
    loads instead of bulk copies)."""
    vr = _vr()
    nx, ny, nb = dims
    spec = synthetic.Par2DSpec(nx, ny, 1.0, synthetic.uniform_angles(64, math.pi), nb, 1.0, 2)
    g = vr.Geometry.from_spec(spec)
    og = J.Geometry2D.from_spec(spec)
    vr.set_launch_shape(g, fwd_band_bytes=shape[0], fwd_group=shape[1], adj_pixels_per_thread=shape[2],
                        adj_split=shape[3])
    x = np.random.default_rng(3).uniform(0, 1, size=(ny, nx))
    for s_ in (0, 1):
        rows = list(range(s_, 64, 2))
        y = host(vr.proj_fwd(g, s_, dev(x))).reshape(len(rows), nb)
        assert rel(y, J.forward(og, x, rows)) < TOL, (s_, shape)
    r = np.random.default_rng(4).standard_normal((32, nb))
    assert rel(host(vr.proj_adj(g, 1, dev(r))), J.adjoint(og, r, list(range(1, 64, 2)))) < TOL
    # the full operator (all 64 angles: shares of 16 and more) through the adjoint identity
    xa = np.random.default_rng(5).standard_normal((ny, nx))
    ra = np.random.default_rng(6).standard_normal((64, nb))
    lhs = float((host(vr.proj_fwd(g, -1, dev(xa))) * ra.ravel()).sum())
    rhs = float((xa.ravel() * host(vr.proj_adj(g, -1, dev(ra)))).sum())
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_largest_2d_size_sampled():
    """2048^2 pixels, 3072 angles, 3072 bins (the largest batched size class doubled): the
    subset forward checked on sampled angles against the oracle, and the full operator by the
    adjoint identity."""
    vr = _vr()
    spec = synthetic.Par2DSpec(2048, 2048, 1.0, synthetic.uniform_angles(3072, math.pi), 3072, 1.0, 24)
    g = vr.Geometry.from_spec(spec)
    og = J.Geometry2D.from_spec(spec)
    x = synthetic.rasterize_ellipses(synthetic.random_ellipses(10, 1024.0, np.random.default_rng(11)),
                                     2048, 2048, 1.0)
    rows = list(range(5, 3072, 24))
    y = host(vr.proj_fwd(g, 5, dev(x))).reshape(len(rows), 3072)
    for k in (0, 32, 64, 127):
        assert rel(y[k], J.forward(og, x, [rows[k]])[0]) < TOL, k
    torch.manual_seed(12)
    xa = torch.randn(g.n, device="cuda")
    ya = torch.randn(g.m, device="cuda")
    lhs = float((vr.proj_fwd(g, -1, xa).double() * ya.double()).sum())
    rhs = float((xa.double() * vr.proj_adj(g, -1, ya).double()).sum())
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_bounded_wait_expires_and_device_stays_usable():
    """The grid barrier of the cooperative prox gives up after its poll limit when a CTA never
    arrives (a one-CTA probe on a counter that needs two arrivals), reports it in the error
    word, and the context keeps working: a prox afterwards still matches the oracle."""
    vr = _vr()
    vr.selftest_bounded_wait(1000)
    with pytest.raises(vr.VrpsError):
        vr.selftest_bounded_wait(0)
    g = vr.Geometry.par2d(40, 33, 1.0, [0.0], 4, 1.0, 1)
    rng = np.random.default_rng(3)
    v = rng.uniform(-0.2, 1.0, size=(33, 40))
    x = vr.prox_tv(g, dev(v), 0.05, 13)
    from oracle import tv
    ref, _ = tv.fgp(v, 0.05, 13)
    assert rel(host(x), ref) < 1e-5
    vr.check_error(g)
