"""Solver path (vrps_solve and helpers) vs the float64 oracle on the same Philox trajectory.

Tolerances: FP32 iterates after a fixed iteration count within 1e-4 relative L2 of the
float64 oracle; Philox draws bit-identical; objective and Lipschitz estimate within 1e-6
and 1e-5 relative."""
import math

import numpy as np
import pytest

from tests._gpu import dev, host, need_gpu, rel, torch

import synthetic
from oracle import joseph2d, philox, solvers

pytestmark = pytest.mark.gpu


def _vr():
    need_gpu()
    import paper_2602_09527_gb300 as vr
    return vr


@pytest.fixture(scope="module")
def small():
    vr = _vr()
    P = synthetic.make_problem_2d(32, 40, 48, 5, seed=21, noise="gauss", alpha=0.02)
    g = vr.Geometry.from_spec(P.spec)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    L = solvers.power_iteration(op, 200, seed=3)
    return vr, P, g, op, L


@pytest.mark.parametrize("N,p", [(10, 0.1), (7, 0.5), (20, 1.0), (3, 0.013), (1, 0.9999)])
def test_philox_schedule_bit_identical(N, p):
    vr = _vr()
    seed, count = 20260209 + N, 200000
    got = vr.philox_schedule(seed, 3, 0, count, N, p).cpu().numpy()
    i, th, coin = philox.schedule(seed, count, N, p, job=3)
    assert np.array_equal(got[:, 0], i)
    assert np.array_equal(got[:, 1].astype(bool), th)
    assert np.array_equal(got[:, 2].astype(bool), coin)
    # an offset window is the same stream
    part = vr.philox_schedule(seed, 3, 1000, 500, N, p).cpu().numpy()
    assert np.array_equal(part, got[1000:1500])


def test_power_iteration_matches_oracle(small):
    vr, P, g, op, _ = small
    lam = vr.power_iteration(g, 60, seed=5)
    ref = solvers.power_iteration(op, 60, seed=5)
    assert abs(lam - ref) / ref < 1e-5


def test_objective_matches_oracle(small):
    vr, P, g, op, _ = small
    x = np.random.default_rng(0).uniform(size=(32, 32))
    F, d, t = vr.objective(g, dev(x), dev(P.b), P.alpha)
    xf = x.astype(np.float32).astype(np.float64)
    bf = P.b.astype(np.float32).astype(np.float64)
    ref = solvers.objective(op, bf, xf, P.alpha)
    assert abs(F - ref) / ref < 1e-6


CASES = [
    ("ISTA", "SVRG", 1.0, 1.0),
    ("FISTA", "SVRG", 1.0, 1.0),
    ("SVRG", "SVRG", 1.0, 1.0),
    ("SAGA", "SVRG", 1 / 3, 1.0),
    ("PROXSKIP", "SVRG", 1.0, 0.3),
    ("VR_PROXSKIP", "SVRG", 1.0, 0.3),
    ("VR_PROXSKIP", "SAGA", 1 / 3, 0.3),
    ("VR_PROXSKIP", "LSVRG", 1.0, 0.3),
    ("VR_PROXSKIP", "SGD", 0.2, 0.3),
]


@pytest.mark.parametrize("algo,est,fac,p", CASES)
def test_trajectory_matches_oracle(small, algo, est, fac, p):
    vr, P, g, op, L = small
    K, seed = 30, 77
    x, rep, _ = vr.solve(dev(P.b), g, P.alpha, algo, p=p, gamma=fac / L, seed=seed, estimator=est,
                         fgp_iters=20, max_iters=K)
    ref = solvers.run(op, P.b, P.alpha, algo, fac / L, K, 20, p=p, seed=seed, estimator=est)
    assert rel(host(x), ref.x) < 1e-4, (algo, est)
    assert rep["prox_calls"] == ref.prox_calls
    assert rep["iterations"] == K
    if est in ("SVRG", "LSVRG") and algo in ("SVRG", "VR_PROXSKIP"):
        assert rep["snapshots"] == ref.snapshots


def test_p_one_skip_equals_nonskip_on_gpu(small):
    vr, P, g, op, L = small
    a, _, _ = vr.solve(dev(P.b), g, P.alpha, "SVRG", gamma=1 / L, seed=4, fgp_iters=20, max_iters=25)
    b, _, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=1.0, gamma=1 / L, seed=4, estimator="SVRG",
                       fgp_iters=20, max_iters=25)
    assert rel(host(b), host(a)) < 1e-5
    c, _, _ = vr.solve(dev(P.b), g, P.alpha, "ISTA", gamma=1 / L, seed=4, fgp_iters=20, max_iters=25)
    d, _, _ = vr.solve(dev(P.b), g, P.alpha, "PROXSKIP", p=1.0, gamma=1 / L, seed=4, fgp_iters=20, max_iters=25)
    assert rel(host(d), host(c)) < 1e-5


def test_host_io_equals_device_io(small):
    vr, P, g, op, L = small
    a, ra, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=0.2, gamma=1 / L, seed=9, fgp_iters=10,
                        max_iters=40)
    bh = torch.tensor(P.b.astype(np.float32).ravel()).pin_memory()
    b, rb, _ = vr.solve(bh, g, P.alpha, "VR_PROXSKIP", p=0.2, gamma=1 / L, seed=9, fgp_iters=10, max_iters=40)
    assert not b.is_cuda
    assert np.array_equal(host(a), b.numpy().astype(np.float64))
    assert ra["prox_calls"] == rb["prox_calls"]


def test_deterministic_rerun(small):
    vr, P, g, op, L = small
    a, _, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=0.3, gamma=1 / L, seed=5, estimator="SAGA",
                       fgp_iters=10, max_iters=30)
    b, _, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=0.3, gamma=1 / L, seed=5, estimator="SAGA",
                       fgp_iters=10, max_iters=30)
    assert torch.equal(a, b)


def test_history_and_target_gap(small):
    vr, P, g, op, L = small
    _, rep, hist = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=0.3, gamma=1 / L, seed=5, fgp_iters=20,
                            max_iters=200, eval_every=10, history_cap=64)
    assert rep["evaluations"] == 20 and len(hist) == 20
    F = [h[1] for h in hist]
    assert F[-1] < F[0]
    fstar = min(F) * (1 - 1e-3)
    _, rep2, hist2 = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=0.3, gamma=1 / L, seed=5, fgp_iters=20,
                              max_iters=200, eval_every=10, history_cap=64, f_star=fstar, target_gap=5e-2)
    assert rep2["reached"] == 1 and rep2["iterations"] < 200
    assert (hist2[-1][1] - fstar) / fstar <= 5e-2


def test_auto_step_uses_power_iteration(small):
    vr, P, g, op, L = small
    _, rep, _ = vr.solve(dev(P.b), g, P.alpha, "SAGA", gamma=0.0, seed=1, fgp_iters=5, max_iters=3,
                         power_iters=200)
    assert abs(rep["lipschitz"] - L) / L < 1e-4
    assert abs(rep["gamma"] - 1 / (3 * rep["lipschitz"])) < 1e-12


def test_par2d_64_full_trajectory():
    """64^2, 90 angles, 96 bins, Gaussian 1 %, N = 10, ProxSVRGSkip p = 0.1, 50 FGP iterations,
    50 epochs (500 iterations), same seed: FP32 GPU vs float64 oracle."""
    vr = _vr()
    P = synthetic.make_problem_2d(64, 90, 96, 10, seed=20260209, noise="gauss", alpha=0.01)
    g = vr.Geometry.from_spec(P.spec)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    L = solvers.power_iteration(op, 100, seed=20260209)
    K = 500
    x, rep, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=0.1, gamma=1 / L, seed=20260209,
                         estimator="SVRG", fgp_iters=50, max_iters=K)
    ref = solvers.run(op, P.b, P.alpha, "VR_PROXSKIP", 1 / L, K, 50, p=0.1, seed=20260209, estimator="SVRG")
    assert rel(host(x), ref.x) < 1e-4
    assert rep["prox_calls"] == ref.prox_calls


def test_solve_rejects_bad_args(small):
    vr, P, g, op, L = small
    with pytest.raises(vr.VrpsError):
        vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=1.5, gamma=1.0, seed=1, max_iters=3)
    with pytest.raises(vr.VrpsError):
        vr.solve(dev(P.b), g, P.alpha, "ISTA", gamma=1.0, seed=1, max_iters=0)
