"""3D cone-beam projector and solver: CUDA path vs the float64 oracle.

Small volumes with ragged sizes and views at multiples of 22.5 degrees (the dominant axis
switches inside the 45-degree views), a scaled copy of the 256^3 / 384^2 / SOD 500 /
SDD 1000 geometry, and a short VR-ProxSkip run.  Tolerance 1e-5 per projection, 1e-4 for
iterates."""
import math

import numpy as np
import pytest

from tests._gpu import dev, host, need_gpu, rel, torch

import synthetic
from oracle import joseph3d as J
from oracle import solvers

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _vr():
    need_gpu()
    import paper_2602_09527_gb300 as vr
    return vr


SMALL = synthetic.Cone3DSpec(nx=21, ny=18, nz=13, voxel=0.5, betas=synthetic.uniform_angles(16, 2 * math.pi),
                             nu=23, nv=17, du=0.8, dv=0.7, sod=40.0, sdd=80.0, n_subsets=3)
SCALED = synthetic.Cone3DSpec(nx=64, ny=64, nz=64, voxel=2.0, betas=synthetic.uniform_angles(36, 2 * math.pi),
                              nu=96, nv=96, du=4.0, dv=4.0, sod=500.0, sdd=1000.0, n_subsets=6)

# ragged against the adjoint's 32 x 8 x 16 voxel tiles and the prox's 32 x 16 x 64 chunks
RAGGED = synthetic.Cone3DSpec(nx=45, ny=19, nz=37, voxel=0.5, betas=synthetic.uniform_angles(8, 2 * math.pi),
                              nu=61, nv=52, du=0.8, dv=0.8, sod=60.0, sdd=120.0, n_subsets=2)


def _pair(spec):
    vr = _vr()
    return vr, vr.Geometry.from_spec(spec), J.GeometryCone.from_spec(spec)


def test_forward_small_every_subset():
    vr, g, og = _pair(SMALL)
    x = np.random.default_rng(1).uniform(size=og.shape())
    for i in list(range(og.n_subsets)) + [-1]:
        ids = og.all_views() if i == -1 else og.subset(i)
        y = vr.proj_fwd(g, i, dev(x))
        assert rel(host(y), J.forward(og, x, ids)) < TOL, i


def test_adjoint_small_every_subset():
    vr, g, og = _pair(SMALL)
    rng = np.random.default_rng(2)
    for i in list(range(og.n_subsets)) + [-1]:
        ids = og.all_views() if i == -1 else og.subset(i)
        r = rng.standard_normal((len(ids), og.nv, og.nu))
        x = vr.proj_adj(g, i, dev(r))
        assert rel(host(x), J.adjoint(og, r, ids)) < TOL, i


def test_ragged_tiles_every_subset():
    vr, g, og = _pair(RAGGED)
    rng = np.random.default_rng(12)
    x = rng.uniform(0.0, 1.0, size=(37, 19, 45))
    for s_ in range(2):
        rows = list(range(s_, 8, 2))
        y = host(vr.proj_fwd(g, s_, dev(x))).reshape(len(rows), 52, 61)
        assert rel(y, J.forward(og, x, rows)) < TOL, s_
        r = rng.standard_normal((len(rows), 52, 61))
        xa = host(vr.proj_adj(g, s_, dev(r)))
        assert rel(xa, J.adjoint(og, r, rows)) < TOL, s_


def test_full_size_sampled_views():
    """The 256^3 / 384^2 / 360-view geometry the 3D bench runs: subset 0 (12 views) forward on a
    random volume, compared on three sampled views, and the adjoint of random data placed on
    two of its views (zero-mean data: no smoothing hides position errors)."""
    w = synthetic.WORKLOADS_3D["cone3d_256"]
    spec = synthetic.Cone3DSpec(nx=w["n"], ny=w["n"], nz=w["n"], voxel=w["voxel"],
                                betas=synthetic.uniform_angles(w["n_views"], 2 * math.pi), nu=w["det"],
                                nv=w["det"], du=w["d"], dv=w["d"], sod=w["sod"], sdd=w["sdd"],
                                n_subsets=w["n_subsets"])
    vr, g, og = _pair(spec)
    n, d, N = w["n"], w["det"], w["n_subsets"]
    rows = list(range(0, w["n_views"], N))
    rng = np.random.default_rng(21)
    x = rng.uniform(0.0, 1.0, size=(n, n, n))
    y = host(vr.proj_fwd(g, 0, dev(x))).reshape(len(rows), d, d)
    for r_i in (0, 4, 7):        # 0, 120 and 210 degrees
        assert rel(y[r_i], J.forward(og, x, [rows[r_i]])[0]) < TOL, r_i
    r = np.zeros((len(rows), d, d))
    pick = [3, 5]                # 90 and 150 degrees
    r[pick] = rng.standard_normal((2, d, d))
    xa = host(vr.proj_adj(g, 0, dev(r)))
    assert rel(xa, J.adjoint(og, r[pick], [rows[i] for i in pick])) < TOL


def test_adjoint_identity_fp32():
    vr, g, og = _pair(SMALL)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(og.n)
    y = rng.standard_normal(og.m)
    Ax = host(vr.proj_fwd(g, -1, dev(x)))
    ATy = host(vr.proj_adj(g, -1, dev(y)))
    yf = y.astype(np.float32).astype(np.float64)
    xf = x.astype(np.float32).astype(np.float64)
    scale = float(np.abs(Ax).sum() * np.abs(yf).max())
    assert abs(Ax @ yf - xf @ ATy) <= 2e-6 * scale


def test_dense_tiny():
    vr = _vr()
    spec = synthetic.Cone3DSpec(nx=4, ny=3, nz=3, voxel=1.0, betas=np.array([0.0, 0.5, math.pi / 4, 2.0]),
                                nu=5, nv=4, du=1.3, dv=1.2, sod=20.0, sdd=40.0, n_subsets=1)
    g = vr.Geometry.from_spec(spec)
    og = J.GeometryCone.from_spec(spec)
    A = J.dense_matrix(og)
    cols = torch.eye(og.n, device="cuda", dtype=torch.float32)
    G = np.stack([host(vr.proj_fwd(g, -1, cols[c].contiguous())) for c in range(og.n)], axis=1)
    assert np.max(np.abs(G - A)) < 1e-5 * max(1.0, np.abs(A).max())
    rows = torch.eye(og.m, device="cuda", dtype=torch.float32)
    GT = np.stack([host(vr.proj_adj(g, -1, rows[r].contiguous())) for r in range(og.m)], axis=0)
    assert np.max(np.abs(GT - A)) < 1e-5 * max(1.0, np.abs(A).max())


def test_scaled_geometry_sampled_views():
    vr, g, og = _pair(SCALED)
    ells = synthetic.random_ellipsoids(10, 64.0, np.random.default_rng(4))
    x = synthetic.rasterize_ellipsoids(ells, 64, 64, 64, 2.0)
    y = host(vr.proj_fwd(g, -1, dev(x))).reshape(36, 96, 96)
    sample = [0, 4, 9, 17, 31]     # 0, 40, 90, 170, 310 degrees
    ref = J.forward(og, x, sample)
    for k, v in enumerate(sample):
        assert rel(y[v], ref[k]) < TOL, v
    r = np.zeros((36, 96, 96))
    r[[4, 9]] = np.random.default_rng(5).standard_normal((2, 96, 96))
    xa = host(vr.proj_adj(g, -1, dev(r)))
    assert rel(xa, J.adjoint(og, r[[4, 9]], [4, 9])) < TOL


def test_unsupported_wide_cone():
    vr = _vr()
    with pytest.raises(vr.VrpsError) as e:
        vr.Geometry.cone3d(8, 8, 8, 1.0, [0.0], 8, 400, 1.0, 1.0, 20.0, 40.0, 1)
    assert e.value.code == -6


def test_cone_solver_short_run():
    vr = _vr()
    spec = synthetic.Cone3DSpec(nx=16, ny=16, nz=12, voxel=1.0, betas=synthetic.uniform_angles(24, 2 * math.pi),
                                nu=24, nv=18, du=1.5, dv=1.5, sod=60.0, sdd=120.0, n_subsets=4)
    ells = synthetic.random_ellipsoids(6, 6.0, np.random.default_rng(6))
    b = synthetic.ellipsoid_cone_projections(ells, spec)
    g = vr.Geometry.from_spec(spec)
    op = solvers.Operator(J.GeometryCone.from_spec(spec))
    L = solvers.power_iteration(op, 100, seed=2)
    x, rep, _ = vr.solve(dev(b), g, 0.01, "VR_PROXSKIP", p=0.3, gamma=1 / L, seed=8, estimator="SVRG",
                         fgp_iters=10, max_iters=12)
    ref = solvers.run(op, b, 0.01, "VR_PROXSKIP", 1 / L, 12, 10, p=0.3, seed=8, estimator="SVRG")
    assert rel(host(x), ref.x) < 1e-4
    assert rep["prox_calls"] == ref.prox_calls


def test_adjoint_z_chunk_same_bits():
    """16 or 32 voxels per thread along z: a voxel's contributions arrive in the same order, so
    the adjoint is bit-identical (and matches the oracle); other values are rejected."""
    vr, g, og = _pair(RAGGED)
    rng = np.random.default_rng(31)
    r = dev(rng.standard_normal((4, 52, 61)))
    outs = []
    for zc in (16, 32):
        vr.set_launch_shape(g, adj_pixels_per_thread=zc)
        assert vr.launch_shape(g)[2] == zc
        outs.append(host(vr.proj_adj(g, 0, r)))
    vr.set_launch_shape(g)
    assert np.array_equal(outs[0], outs[1])
    assert rel(outs[0], J.adjoint(og, host(r).reshape(4, 52, 61), list(range(0, 8, 2)))) < TOL
    with pytest.raises(vr.VrpsError):
        vr.set_launch_shape(g, adj_pixels_per_thread=8)
    t = vr.autotune(g, reps=1)
    assert t["adj3d_voxels_per_thread"] in (16, 32)
