"""GPU preconditioned PDHG (vrps_pdhg) against the float64 oracle PDHG: same iteration count,
same steps, 2D and 3D; and its converged objective against the oracle's minimiser."""
import math

import numpy as np
import pytest

from tests._gpu import dev, host, need_gpu, rel

import synthetic
from oracle import joseph2d, joseph3d, pdhg, solvers

pytestmark = pytest.mark.gpu


def _vr():
    need_gpu()
    import paper_2602_09527_gb300 as vr
    return vr


@pytest.mark.parametrize("alpha,nonneg", [(0.02, True), (0.0, True), (0.05, False)])
def test_pdhg_2d_matches_oracle(alpha, nonneg):
    vr = _vr()
    P = synthetic.make_problem_2d(24, 30, 36, 3, seed=5, noise="gauss", alpha=alpha)
    g = vr.Geometry.from_spec(P.spec)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    K = 150
    x, rep, hist = vr.pdhg(dev(P.b), g, alpha, K, nonneg=nonneg, eval_every=50, history_cap=8)
    ref, rh = pdhg.pdhg(op, P.b, alpha, K, nonneg=nonneg, eval_every=50)
    assert rel(host(x), ref.reshape(-1)) < 1e-4
    assert rep["iterations"] == K and rep["evaluations"] == 3
    for (k, F), (kr, Fr) in zip(hist, rh):
        assert k == kr and abs(F - Fr) / Fr < 1e-5


def test_pdhg_3d_matches_oracle():
    vr = _vr()
    spec = synthetic.Cone3DSpec(nx=12, ny=10, nz=9, voxel=1.0, betas=synthetic.uniform_angles(10, 2 * math.pi),
                                nu=16, nv=12, du=1.5, dv=1.5, sod=40.0, sdd=80.0, n_subsets=2)
    g = vr.Geometry.from_spec(spec)
    og = joseph3d.GeometryCone.from_spec(spec)
    op = solvers.Operator(og)
    x0 = np.random.default_rng(2).uniform(0, 1, size=(9, 10, 12))
    b = joseph3d.forward(og, x0, list(range(10)))
    x, _, _ = vr.pdhg(dev(b), g, 0.01, 60)
    ref, _ = pdhg.pdhg(op, b, 0.01, 60)
    assert rel(host(x), ref.reshape(-1)) < 1e-4


def test_pdhg_converges_to_the_oracle_minimum():
    vr = _vr()
    P = synthetic.make_problem_2d(16, 20, 24, 2, seed=9, noise="gauss", alpha=0.03)
    g = vr.Geometry.from_spec(P.spec)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    x, rep, _ = vr.pdhg(dev(P.b), g, 0.03, 3000)
    ref, _ = pdhg.pdhg(op, P.b, 0.03, 3000)
    F = solvers.objective(op, P.b, host(x).reshape(16, 16), 0.03)
    Fr = solvers.objective(op, P.b, ref, 0.03)
    assert abs(F - Fr) / Fr < 1e-6
