"""Batched 3D cone-beam jobs (vrps_batch_* with 3D geometries): every job's result is
bit-identical to vrps_solve with the same arguments, alone and in any mix, admitted at once or
between ticks, with and without CUDA-graph replay; one batched job against the float64 oracle
(1e-4); a batch keeps to one dimensionality."""
import math

import numpy as np
import pytest

from tests._gpu import dev, host, need_gpu, rel, torch

import synthetic
from oracle import joseph3d as J
from oracle import solvers

pytestmark = pytest.mark.gpu


def _vr():
    need_gpu()
    import paper_2602_09527_gb300 as vr
    return vr


# (nx, ny, nz, views, nu, nv, N, estimator, p, fgp_iters, iters, storage, correction epochs)
MIX = [
    (24, 24, 16, 24, 32, 24, 4, "SVRG", 0.2, 20, 14, "FP32", 0),
    (45, 19, 37, 16, 61, 52, 4, "SAGA", 0.3, 10, 12, "FP32", 0),      # ragged against every tile
    (32, 32, 32, 30, 48, 48, 5, "LSVRG", 0.25, 33, 15, "FP32", 0),     # 33 FGP iterations
    (20, 28, 12, 18, 30, 20, 3, "SAGA", 0.4, 8, 12, "BF16", 1),
    (16, 16, 70, 12, 24, 96, 3, "SGD", 0.5, 0, 9, "FP32", 0),          # two prox z chunks, no FGP iteration
    (36, 36, 20, 20, 52, 30, 4, "SVRG", 0.3, 12, 16, "FP16", 1),
]


def _problem(vr, i, spec):
    nx, ny, nz, nviews, nu, nv, N = spec[:7]
    voxel = 1.0
    cs = synthetic.Cone3DSpec(nx=nx, ny=ny, nz=nz, voxel=voxel, betas=synthetic.uniform_angles(nviews, 2 * math.pi),
                              nu=nu, nv=nv, du=1.5, dv=1.5, sod=4.0 * max(nx, ny, nz), sdd=8.0 * max(nx, ny, nz),
                              n_subsets=N)
    rng = np.random.default_rng(300 + i)
    ells = synthetic.random_ellipsoids(5, 0.4 * min(nx, ny, nz), rng)
    b = synthetic.ellipsoid_cone_projections(ells, cs)
    b = b + 0.01 * np.abs(b).max() * rng.standard_normal(b.shape)
    g = vr.Geometry.from_spec(cs)
    L = vr.power_iteration(g, 40, seed=3)
    return cs, g, b, L


def _kw(spec, L, i):
    est, p, fgp, K, storage, corr = spec[7:]
    fac = 1 / 3 if est == "SAGA" else 1.0
    return dict(alpha=0.02, p=p, gamma=fac / L, seed=700 + i, job=i, estimator=est, fgp_iters=fgp,
                max_iters=K, storage=storage, correction_epochs=corr)


def _solo(vr, g, b, kw):
    kw = dict(kw)
    x, rep, _ = vr.solve(dev(b), g, kw.pop("alpha"), "VR_PROXSKIP", p=kw.pop("p"), gamma=kw.pop("gamma"),
                         seed=kw.pop("seed"), **kw)
    torch.cuda.synchronize()
    return x.clone(), rep


@pytest.fixture(scope="module")
def mix():
    vr = _vr()
    probs = [_problem(vr, i, s) for i, s in enumerate(MIX)]
    solo = [_solo(vr, g, b, _kw(MIX[i], L, i)) for i, (cs, g, b, L) in enumerate(probs)]
    return vr, probs, solo


def _check(B, ids, probs, solo, which):
    for i, jid in zip(which, ids):
        rep = B.wait(jid)
        x = B.result(jid)
        xs, rs = solo[i]
        assert torch.equal(x, xs), (i, float((x - xs).abs().max()))
        assert rep["prox_calls"] == rs["prox_calls"], i
        assert rep["iterations"] == rs["iterations"], i
        assert rep["snapshots"] == rs["snapshots"], i


@pytest.mark.parametrize("graphs", [True, False])
def test_mix_bit_identical_to_solo(mix, graphs):
    vr, probs, solo = mix
    B = vr.Batch(graphs=graphs)
    ids = [B.submit(g, dev(b), **_kw(MIX[i], L, i)) for i, (cs, g, b, L) in enumerate(probs)]
    while B.step(4):
        pass
    _check(B, ids, probs, solo, range(len(MIX)))
    B.close()


def test_staggered_admission(mix):
    """Jobs join between ticks while others run; results still equal the solo runs."""
    vr, probs, solo = mix
    B = vr.Batch(graphs=True)
    order = [2, 0, 4, 1, 5, 3]
    ids = []
    for n, i in enumerate(order):
        cs, g, b, L = probs[i]
        ids.append(B.submit(g, dev(b), **_kw(MIX[i], L, i)))
        B.step(1 + n)
    while B.step(3):
        pass
    _check(B, ids, probs, solo, order)
    B.close()


def test_single_job_against_oracle():
    vr = _vr()
    spec = synthetic.Cone3DSpec(nx=16, ny=16, nz=12, voxel=1.0, betas=synthetic.uniform_angles(24, 2 * math.pi),
                                nu=24, nv=18, du=1.5, dv=1.5, sod=60.0, sdd=120.0, n_subsets=4)
    ells = synthetic.random_ellipsoids(6, 6.0, np.random.default_rng(16))
    b = synthetic.ellipsoid_cone_projections(ells, spec)
    g = vr.Geometry.from_spec(spec)
    op = solvers.Operator(J.GeometryCone.from_spec(spec))
    L = solvers.power_iteration(op, 100, seed=2)
    B = vr.Batch()
    jid = B.submit(g, dev(b), alpha=0.01, p=0.3, gamma=1 / (3 * L), seed=18, estimator="SAGA", fgp_iters=10,
                   max_iters=14)
    rep = B.wait(jid)
    ref = solvers.run(op, b, 0.01, "VR_PROXSKIP", 1 / (3 * L), 14, 10, p=0.3, seed=18, estimator="SAGA")
    assert rel(host(B.result(jid)), ref.x) < 1e-4
    assert rep["prox_calls"] == ref.prox_calls
    B.close()


def test_batch_keeps_one_dimensionality(mix):
    vr, probs, solo = mix
    cs, g, b, L = probs[0]
    B = vr.Batch()
    jid = B.submit(g, dev(b), **_kw(MIX[0], L, 0))
    ps = synthetic.Par2DSpec(nx=32, ny=32, pixel=1.0, angles=synthetic.uniform_angles(30, math.pi), n_bins=48,
                             bin_spacing=1.0, n_subsets=3)
    g2 = vr.Geometry.from_spec(ps)
    b2 = torch.zeros(g2.m, device="cuda")
    with pytest.raises(vr.VrpsError) as e:
        B.submit(g2, b2, alpha=0.01, p=0.5, gamma=1e-3, max_iters=3)
    assert e.value.code == -1
    with pytest.raises(vr.VrpsError):
        B.submit(probs[1][1], dev(probs[1][2]), **dict(_kw(MIX[1], probs[1][3], 1), fgp_iters=129))
    B.wait(jid)
    B.close()


def test_footprint_3d_covers_workspace(mix):
    vr, probs, solo = mix
    cs, g, b, L = probs[2]
    f = vr.job_footprint(g, max_iters=15, storage="FP32")
    assert f >= 4 * g.n * 16 + 4 * g.m * 4
