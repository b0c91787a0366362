"""Reduced-precision storage (bfloat16, or float16 with a power-of-two scale) of the solver's
sinogram-sized state (b and the SVRG / SAGA table) with float32 arithmetic, finished by float32
correction epochs, against the float64 oracle on the same Philox trajectory.  Tolerance: the
objective of the final iterate within 1e-3 relative of the oracle's."""
import numpy as np
import pytest

from tests._gpu import dev, host, need_gpu, rel

import synthetic
from oracle import joseph2d, solvers

pytestmark = pytest.mark.gpu

TOL_F = 1e-3


def _vr():
    need_gpu()
    import paper_2602_09527_gb300 as vr
    return vr


@pytest.fixture(scope="module")
def c1():
    """64^2, 90 angles, 96 bins, Gaussian 1 %, N = 10 (the small 2D workload)."""
    vr = _vr()
    P = synthetic.make_problem_2d(64, 90, 96, 10, seed=20260209, noise="gauss", alpha=0.01)
    g = vr.Geometry.from_spec(P.spec)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    L = solvers.power_iteration(op, 100, seed=20260209)
    return vr, P, g, op, L


@pytest.mark.parametrize("storage", ["BF16", "FP16"])
@pytest.mark.parametrize("est,fac", [("SVRG", 1.0), ("SAGA", 1 / 3)])
def test_reduced_storage_objective_within_1e3(c1, est, fac, storage):
    vr, P, g, op, L = c1
    K, seed = 300, 20260209
    x, rep, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=0.1, gamma=fac / L, seed=seed, estimator=est,
                         fgp_iters=50, max_iters=K, storage=storage, correction_epochs=2)
    ref = solvers.run(op, P.b, P.alpha, "VR_PROXSKIP", fac / L, K, 50, p=0.1, seed=seed, estimator=est)
    F = solvers.objective(op, P.b, host(x), P.alpha)
    Fr = solvers.objective(op, P.b, ref.x, P.alpha)
    assert abs(F - Fr) / Fr < TOL_F, (est, F, Fr)
    assert rep["prox_calls"] == ref.prox_calls
    # the reduced-precision run is a different trajectory, but a close one
    assert rel(host(x), ref.x) < 5e-2


def test_bf16_without_correction_differs_from_fp32(c1):
    """Storage really is bfloat16 in the first phase: without the correction the run differs
    from the float32 run by far more than float32 rounding."""
    vr, P, g, op, L = c1
    kw = dict(p=0.1, gamma=1 / L, seed=5, estimator="SVRG", fgp_iters=20, max_iters=60)
    a, _, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", **kw)
    b, _, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", storage="BF16", **kw)
    d = rel(host(b), host(a))
    assert 1e-4 < d < 5e-2


def test_fp16_closer_than_bf16(c1):
    """float16 keeps 3 more mantissa bits than bfloat16: without correction its run stays
    closer to the float32 run."""
    vr, P, g, op, L = c1
    kw = dict(p=0.1, gamma=1 / (3 * L), seed=6, estimator="SAGA", fgp_iters=20, max_iters=80)
    a, _, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", **kw)
    b, _, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", storage="BF16", **kw)
    h, _, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", storage="FP16", **kw)
    assert rel(host(h), host(a)) < 0.5 * rel(host(b), host(a))


def test_correction_covering_whole_run_equals_fp32(c1):
    """correction_epochs * N >= iterations: the whole run uses float32 storage."""
    vr, P, g, op, L = c1
    kw = dict(p=0.2, gamma=1 / (3 * L), seed=8, estimator="SAGA", fgp_iters=10, max_iters=20)
    a, _, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", **kw)
    b, _, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", storage="BF16", correction_epochs=2, **kw)
    assert np.array_equal(host(a), host(b))
