"""Batched / served jobs (vrps_batch_*): every job's result is bit-identical to vrps_solve with
the same arguments, alone and in any mix, with jobs admitted between ticks, with and
without CUDA-graph replay; one batched job also against the float64 oracle (1e-4)."""
import math

import numpy as np
import pytest

from tests._gpu import dev, host, need_gpu, rel, torch

import synthetic
from oracle import joseph2d, solvers

pytestmark = pytest.mark.gpu


def _vr():
    need_gpu()
    import paper_2602_09527_gb300 as vr
    return vr


# (side_x, side_y, angles, bins, N, estimator, p, fgp_iters, iters, storage, correction epochs)
MIX = [
    (64, 64, 90, 96, 10, "SVRG", 0.1, 50, 60, "FP32", 0),
    (48, 80, 72, 120, 8, "SAGA", 0.3, 20, 50, "FP32", 0),
    (96, 96, 144, 144, 12, "SAGA", 0.2, 16, 70, "BF16", 2),
    (30, 30, 45, 45, 5, "LSVRG", 0.5, 12, 40, "FP32", 0),     # sides not multiples of 4
    (128, 128, 192, 192, 16, "SVRG", 0.1, 100, 48, "BF16", 1),
    (40, 56, 60, 84, 6, "SGD", 0.25, 0, 30, "FP32", 0),       # no inner FGP iteration
    (72, 72, 108, 108, 9, "SAGA", 0.2, 24, 45, "FP16", 2),
]


def _problem(vr, i, spec):
    sx, sy, na, nb, N = spec[:5]
    rng = np.random.default_rng(100 + i)
    ells = synthetic.random_ellipses(6, min(sx, sy) / 2.0, rng)
    ps = synthetic.Par2DSpec(nx=sx, ny=sy, pixel=1.0, angles=synthetic.uniform_angles(na, math.pi), n_bins=nb,
                             bin_spacing=1.0, n_subsets=N)
    b = synthetic.gaussian_noise(synthetic.ellipse_sinogram(ells, ps.angles, ps.bin_centers()), 0.01, rng)
    g = vr.Geometry.from_spec(ps)
    L = vr.power_iteration(g, 60, seed=7)
    return ps, g, b, L


def _kw(spec, L, i):
    est, p, fgp, K, storage, corr = spec[5:]
    fac = 1 / 3 if est == "SAGA" else 1.0
    return dict(alpha=0.02, p=p, gamma=fac / L, seed=900 + i, job=i, estimator=est, fgp_iters=fgp,
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
    solo = []
    for i, (ps, g, b, L) in enumerate(probs):
        solo.append(_solo(vr, g, b, _kw(MIX[i], L, i)))
    return vr, probs, solo


@pytest.mark.parametrize("graphs", [True, False])
def test_mix_bit_identical_to_solo(mix, graphs):
    vr, probs, solo = mix
    B = vr.Batch(graphs=graphs)
    ids = []
    for i, (ps, g, b, L) in enumerate(probs):
        ids.append(B.submit(g, dev(b), **_kw(MIX[i], L, i)))
    while B.step(4):
        pass
    for i, jid in enumerate(ids):
        rep = B.wait(jid)
        x = B.result(jid)
        assert torch.equal(x, solo[i][0]), (i, rel(host(x), host(solo[i][0])))
        assert rep["iterations"] == solo[i][1]["iterations"]
        assert rep["prox_calls"] == solo[i][1]["prox_calls"]
        assert rep["snapshots"] == solo[i][1]["snapshots"]
        assert abs(rep["passes"] - solo[i][1]["passes"]) < 1e-9
    B.close()


def test_priority_and_grid_share_keep_bits(mix):
    """A batch on a highest-priority stream whose persistent grids take a third of the GPU gives
    the same bits (scheduling knobs only); both knobs are refused once a job was submitted."""
    vr, probs, solo = mix
    B = vr.Batch(priority=-100, grid_share=1.0 / 3.0)
    ids = [B.submit(probs[i][1], dev(probs[i][2]), **_kw(MIX[i], probs[i][3], i)) for i in range(len(MIX))]
    while B.step(4):
        pass
    for i, jid in enumerate(ids):
        B.wait(jid)
        assert torch.equal(B.result(jid), solo[i][0]), i
    import ctypes
    assert vr.lib.vrps_batch_set_grid_share(B.handle, ctypes.c_double(0.5)) == -1
    assert vr.lib.vrps_batch_set_stream_priority(B.handle, 0) == -1
    B.close()


def test_staggered_admission_and_alone(mix):
    """Jobs joining while others run, and a job running alone, give the same bits."""
    vr, probs, solo = mix
    B = vr.Batch()
    first = [B.submit(probs[i][1], dev(probs[i][2]), **_kw(MIX[i], probs[i][3], i)) for i in (0, 3)]
    B.step(7)
    later = [B.submit(probs[i][1], dev(probs[i][2]), **_kw(MIX[i], probs[i][3], i)) for i in (1, 4)]
    B.step(3)
    last = [B.submit(probs[i][1], dev(probs[i][2]), **_kw(MIX[i], probs[i][3], i)) for i in (2, 5)]
    order = {first[0]: 0, first[1]: 3, later[0]: 1, later[1]: 4, last[0]: 2, last[1]: 5}
    for jid, i in order.items():
        B.wait(jid)
        assert torch.equal(B.result(jid), solo[i][0]), i
    B.close()
    A = vr.Batch()
    jid = A.submit(probs[2][1], dev(probs[2][2]), **_kw(MIX[2], probs[2][3], 2))
    A.wait(jid)
    assert torch.equal(A.result(jid), solo[2][0])
    A.close()


def test_grouped_forward_shapes_in_the_mix(mix):
    """Jobs whose geometries walk several forward bands per CTA (and others that do not) stay
    bit-identical to their solo runs."""
    vr, probs, solo = mix
    for i in (0, 2, 4):
        vr.set_launch_shape(probs[i][1], fwd_band_bytes=16 << 10, fwd_group=3, adj_split=2)
    try:
        ref = [_solo(vr, probs[i][1], probs[i][2], _kw(MIX[i], probs[i][3], i))[0] for i in range(len(MIX))]
        B = vr.Batch()
        ids = [B.submit(probs[i][1], dev(probs[i][2]), **_kw(MIX[i], probs[i][3], i)) for i in range(len(MIX))]
        for i, jid in enumerate(ids):
            B.wait(jid)
            assert torch.equal(B.result(jid), ref[i]), i
        B.close()
    finally:
        for i in (0, 2, 4):
            vr.set_launch_shape(probs[i][1])


def test_batched_job_matches_oracle():
    vr = _vr()
    P = synthetic.make_problem_2d(32, 40, 48, 5, seed=21, noise="gauss", alpha=0.02)
    g = vr.Geometry.from_spec(P.spec)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    L = solvers.power_iteration(op, 200, seed=3)
    B = vr.Batch()
    jid = B.submit(g, dev(P.b), alpha=P.alpha, p=0.3, gamma=1 / (3 * L), seed=77, estimator="SAGA", fgp_iters=20,
                   max_iters=30)
    B.wait(jid)
    ref = solvers.run(op, P.b, P.alpha, "VR_PROXSKIP", 1 / (3 * L), 30, 20, p=0.3, seed=77, estimator="SAGA")
    assert rel(host(B.result(jid)), ref.x) < 1e-4
    B.close()


def test_busy_geometry_and_bad_jobs_rejected(mix):
    vr, probs, _ = mix
    ps, g, b, L = probs[0]
    B = vr.Batch()
    B.submit(g, dev(b), **_kw(MIX[0], L, 0))
    with pytest.raises(vr.VrpsError):
        B.submit(g, dev(b), **_kw(MIX[0], L, 0))          # geometry in use
    g2 = vr.Geometry.from_spec(ps)
    bad = _kw(MIX[0], L, 0)
    bad["gamma"] = 0.0
    with pytest.raises(vr.VrpsError):
        B.submit(g2, dev(b), **bad)
    bad = _kw(MIX[0], L, 0)
    bad["fgp_iters"] = 200
    with pytest.raises(vr.VrpsError):
        B.submit(g2, dev(b), **bad)
    B.close()
    assert vr.job_footprint(g2, max_iters=100) > 4 * g2.n * 10
    g2.close()


def test_launch_count_per_tick(mix):
    """A tick is 3 + (FGP blocks of 6 iterations) launches however many jobs run."""
    vr, probs, _ = mix
    B = vr.Batch()
    for i in (0, 1, 3):
        B.submit(probs[i][1], dev(probs[i][2]), **_kw(MIX[i], probs[i][3], i))
    B.step(1)
    B.sync()
    n0 = vr.kernel_launches()
    B.step(5)
    B.sync()
    per_tick = (vr.kernel_launches() - n0) / 5
    assert per_tick == 3 + math.ceil(50 / 6)
    B.close()


def test_served_stream_results_equal_solo(mix):
    """Requests arriving over time through the request loop (admission by footprint with a
    budget that holds only some jobs at once) finish, and each result equals vrps_solve's."""
    vr, probs, solo = mix
    from paper_2602_09527_gb300 import serve
    pools = {i: [probs[i][1]] for i in range(len(MIX))}
    reqs = []
    for t, i in enumerate([3, 0, 5, 1, 2, 4, 6]):
        kw = _kw(MIX[i], probs[i][3], i)
        reqs.append(serve.Request(key=i, b=dev(probs[i][2]), arrival=0.01 * t, alpha=kw["alpha"], gamma=kw["gamma"],
                                  seed=kw["seed"], p=kw["p"], estimator=kw["estimator"], fgp_iters=kw["fgp_iters"],
                                  max_iters=kw["max_iters"], storage=kw["storage"],
                                  correction_epochs=kw["correction_epochs"]))
    budget = 3 * max(vr.job_footprint(probs[i][1], max_iters=100) for i in range(len(MIX)))
    srv = serve.BatchServer(pools, budget)
    st = srv.run(reqs)
    srv.close()
    assert st.completed == len(reqs)
    assert all(l > 0 for l in st.latencies)
    assert st.peak_bytes <= budget
    for r, i in zip(reqs, [3, 0, 5, 1, 2, 4, 6]):
        assert r.finished >= r.admitted >= r.arrival
        # the request loop passes job word 0; compare with the solo run of the same settings
        kw = _kw(MIX[i], probs[i][3], i)
        kw["job"] = 0
        x, _ = _solo(vr, probs[i][1], probs[i][2], kw)
        assert torch.equal(r.x, x), i


def test_mixed_server_3d_batch(mix):
    """2D requests in one batch and 3D requests in a second batch on its own stream, each within
    its share of the memory budget: all finish, and each 3D result equals vrps_solve's on the
    same inputs."""
    vr, probs, solo = mix
    from paper_2602_09527_gb300 import serve
    spec3 = synthetic.Cone3DSpec(nx=20, ny=20, nz=16, voxel=1.0, betas=synthetic.uniform_angles(24, 2 * math.pi),
                                 nu=28, nv=24, du=1.5, dv=1.5, sod=60.0, sdd=120.0, n_subsets=4)
    g3 = [vr.Geometry.from_spec(spec3) for _ in range(2)]
    x0 = np.random.default_rng(5).uniform(0, 1, size=(16, 20, 20))
    from oracle import joseph3d
    b3 = dev(joseph3d.forward(joseph3d.GeometryCone.from_spec(spec3), x0, list(range(24))))
    L3 = vr.power_iteration(g3[0], 30, seed=3)
    reqs = []
    for t, i in enumerate([0, 1, 3]):
        kw = _kw(MIX[i], probs[i][3], i)
        reqs.append(serve.Request(key=i, b=dev(probs[i][2]), arrival=0.005 * t, alpha=kw["alpha"], gamma=kw["gamma"],
                                  seed=kw["seed"], p=kw["p"], estimator=kw["estimator"], fgp_iters=kw["fgp_iters"],
                                  max_iters=kw["max_iters"]))
    s3 = [dict(seed=44, estimator="SAGA", p=0.2), dict(seed=45, estimator="SVRG", p=0.3)]
    for q, k in enumerate(s3):
        reqs.insert(1 + 2 * q, serve.Request(key="cone", b=b3, arrival=0.002 + 0.004 * q, alpha=0.01,
                                             gamma=1 / (3 * L3), fgp_iters=10, max_iters=40, **k))
    srv = serve.MixedServer({i: [probs[i][1]] for i in (0, 1, 3)}, {"cone": g3}, 1 << 36)
    st = srv.run(reqs)
    srv.close()
    assert st.completed == len(reqs)
    got = [r for r in reqs if r.key == "cone"]
    for r, k in zip(got, s3):
        x, _, _ = vr.solve(b3, g3[0], 0.01, "VR_PROXSKIP", gamma=1 / (3 * L3), fgp_iters=10, max_iters=40, **k)
        torch.cuda.synchronize()
        assert torch.equal(r.x, x), k
    for g in g3:
        g.close()
