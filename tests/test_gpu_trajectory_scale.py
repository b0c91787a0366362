"""Whole-trajectory parity at the benchmark scales: FP32 CUDA path vs the float64 oracle on the
same Philox draws (subset i_k, skip coin theta_k), in the launch shapes the bench times.

* 512^2 parallel beam, 720 angles, 768 bins, 20 subsets, Poisson 1e4 photons, TV weight 1.0:
  ProxSVRGSkip p = 0.1 with 100 FGP iterations for two epochs (40 iterations: snapshots at
  k = 0 and 20, prox steps at k = 15, 16, 32 for this seed).  Iterates within 1e-4 relative L2.
* The 256^3 cone geometry scaled to 64^3 (voxel 2, 90 views over 360 degrees, 96^2 detector of
  pitch 4, SOD 500, SDD 1000, 30 subsets, Gaussian 1 %): ProxSVRGSkip p = 0.1, 50 3D FGP
  iterations, one epoch (30 iterations).  Iterates within 1e-4.
* One size class of the batched workload (256^2, 384 angles, 384 bins, 20 subsets, Gaussian 1 %,
  TV weight 0.02 on a unit-radius field of view): ProxSAGASkip p = 0.1 run to just after its
  ninth prox step (46 iterations).  Float32 storage: iterates within 1e-4.  Sinogram and SAGA
  table stored in bfloat16 (and float16): the objective of that prox output within 1e-3
  relative of the oracle's.  (The float32 correction epoch that ends a reduced-storage run
  rebuilds the SAGA table at the current point, so after it the trajectory is a different one
  by design; the correction is checked at convergence on the 64^2 problem.)

The step is 1 / L_up with L_up = max row sum x max column sum of A (Schur's bound on ||A||_2^2,
computed by the oracle from A 1 and A^T 1), so that no input comes from the CUDA path."""
import math

import numpy as np
import pytest

from tests._gpu import dev, host, need_gpu, rel

import synthetic
from oracle import joseph2d, joseph3d, solvers

pytestmark = pytest.mark.gpu

TOL_X = 1e-4
TOL_F = 1e-3
SEED = 20260209


def _vr():
    need_gpu()
    import paper_2602_09527_gb300 as vr
    return vr


def _schur_bound(op):
    rows = op.fwd(np.ones(op.shape))
    cols = op.adj(np.ones_like(rows))
    return float(rows.max()) * float(cols.max())


def test_par2d_512_two_epochs_svrg_skip():
    vr = _vr()
    P = synthetic.make_problem_2d(512, 720, 768, 20, seed=SEED, noise="poisson", alpha=1.0)
    g = vr.Geometry.from_spec(P.spec)
    vr.autotune(g, reps=3)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    gamma = 1.0 / _schur_bound(op)
    K = 40
    x, rep, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=0.1, gamma=gamma, seed=SEED, estimator="SVRG",
                         fgp_iters=100, max_iters=K)
    ref = solvers.run(op, P.b, P.alpha, "VR_PROXSKIP", gamma, K, 100, p=0.1, seed=SEED, estimator="SVRG")
    assert ref.snapshot_iters == [0, 20] and ref.prox_calls == 3
    assert rep["prox_calls"] == ref.prox_calls and rep["snapshots"] == ref.snapshots
    err = rel(host(x), ref.x)
    assert err < TOL_X, err


def test_cone_64_one_epoch_svrg_skip():
    vr = _vr()
    P = synthetic.make_problem_3d(64, 2.0, 90, 96, 4.0, 500.0, 1000.0, 30, seed=SEED, alpha=0.01)
    g = vr.Geometry.from_spec(P.spec)
    vr.autotune(g, reps=2)
    op = solvers.Operator(joseph3d.GeometryCone.from_spec(P.spec))
    gamma = 1.0 / _schur_bound(op)
    K = 30
    x, rep, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=0.1, gamma=gamma, seed=SEED, estimator="SVRG",
                         fgp_iters=50, max_iters=K)
    ref = solvers.run(op, P.b, P.alpha, "VR_PROXSKIP", gamma, K, 50, p=0.1, seed=SEED, estimator="SVRG")
    assert ref.snapshot_iters == [0] and ref.prox_calls == 2
    assert rep["prox_calls"] == ref.prox_calls and rep["snapshots"] == ref.snapshots
    err = rel(host(x), ref.x)
    assert err < TOL_X, err


@pytest.fixture(scope="module")
def c4_class():
    vr = _vr()
    side = 256
    alpha = 0.02 * (side / 2) ** 2        # 0.02 on a unit-radius field of view, in pixel units
    P = synthetic.make_problem_2d(side, 384, 384, 20, seed=SEED + 1, noise="gauss", alpha=alpha)
    g = vr.Geometry.from_spec(P.spec)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    gamma = 1.0 / (3.0 * _schur_bound(op))
    K = 46                                # prox steps at k = 6, 17, 19, 22, 24, 32, 35, 44, 45
    ref = solvers.run(op, P.b, P.alpha, "VR_PROXSKIP", gamma, K, 50, p=0.1, seed=SEED + 1, estimator="SAGA")
    assert ref.prox_calls == 9 and np.array_equal(ref.x, ref.last_prox)
    Fr = solvers.objective(op, P.b, ref.x, P.alpha)
    return vr, P, g, op, gamma, K, ref, Fr


def _saga(c, **kw):
    vr, P, g, op, gamma, K, ref, Fr = c
    x, rep, _ = vr.solve(dev(P.b), g, P.alpha, "VR_PROXSKIP", p=0.1, gamma=gamma, seed=SEED + 1, estimator="SAGA",
                         fgp_iters=50, max_iters=K, **kw)
    assert rep["prox_calls"] == ref.prox_calls
    return x


def test_batched_size_class_fp32_saga_trajectory(c4_class):
    x = _saga(c4_class)
    err = rel(host(x), c4_class[6].x)
    assert err < TOL_X, err


@pytest.mark.parametrize("storage", ["BF16", "FP16"])
def test_batched_size_class_reduced_storage_saga(c4_class, storage):
    vr, P, g, op, gamma, K, ref, Fr = c4_class
    x = _saga(c4_class, storage=storage)
    F = solvers.objective(op, P.b, host(x), P.alpha)
    assert abs(F - Fr) / Fr < TOL_F, (storage, F, Fr)
