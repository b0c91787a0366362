"""Pins of the float64 PDHG reference minimiser (oracle/pdhg.py) against independent results:
alpha = 0 reduces the problem to nonnegative least squares (scipy.optimize.nnls on the dense
Joseph matrix); A = I reduces it to the exact TV prox (oracle.tv.prox_pdhg, pinned by closed
forms); scalar and diagonally preconditioned steps reach the same minimiser; and no iterate
of a long FISTA run gets below the PDHG objective."""
import numpy as np
import pytest
import scipy.optimize as so

import synthetic
from oracle import joseph2d, pdhg, solvers, tv


def _small(alpha):
    P = synthetic.make_problem_2d(6, 8, 9, 2, seed=3, noise="gauss", alpha=alpha)
    return P, solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))


def test_alpha_zero_is_nnls():
    P, op = _small(0.0)
    A = np.stack([op.fwd(e.reshape(6, 6)).reshape(-1) for e in np.eye(36)], axis=1)
    xn, _ = so.nnls(A, P.b.reshape(-1))
    x, _ = pdhg.pdhg(op, P.b, 0.0, 1200)
    assert np.linalg.norm(x.reshape(-1) - xn) / np.linalg.norm(xn) < 1e-10


class _Identity:
    def __init__(self, shape):
        self.shape = shape
        self.D = tv.grad_operator(shape)

    def fwd(self, x):
        return np.asarray(x, dtype=np.float64).reshape(self.shape)

    def adj(self, r):
        return np.asarray(r, dtype=np.float64).reshape(self.shape)


@pytest.mark.parametrize("shape", [(5, 6), (3, 4, 3)])
def test_identity_operator_is_tv_prox(shape):
    v = np.random.default_rng(1).uniform(-0.2, 1.0, size=shape)
    x, _ = pdhg.pdhg(_Identity(shape), v, 0.3, 1500)
    assert np.abs(x - tv.prox_pdhg(v, 0.3)).max() < 1e-9


def test_scalar_and_preconditioned_steps_agree():
    P, op = _small(0.05)
    a, _ = pdhg.pdhg(op, P.b, 0.05, 1500)
    b, _ = pdhg.pdhg(op, P.b, 0.05, 3000, precondition=False)
    assert np.abs(a - b).max() < 1e-8


def test_fista_never_below_pdhg_minimum():
    P, op = _small(0.05)
    x, _ = pdhg.pdhg(op, P.b, 0.05, 1500)
    Fmin = solvers.objective(op, P.b, x, 0.05)
    L = solvers.power_iteration(op, 200, seed=1)
    tr = solvers.run(op, P.b, 0.05, "FISTA", 1.0 / L, 300, 200, eval_every=10)
    best = min(tr.objective.values())
    assert best >= Fmin * (1 - 1e-9)
    assert best <= Fmin * (1 + 1e-3)
