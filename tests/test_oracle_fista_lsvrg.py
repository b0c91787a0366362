"""Pins of the oracle's FISTA momentum and its L-SVRG refresh rule (CPU only).

FISTA (Beck-Teboulle, reading R-10): A = I on a 1 x 2 image, where every prox the run takes
is the two-pixel closed form (a - tau, b + tau) (the split case of the TV prox with
nonnegativity inactive).  Each iteration is then an affine map of the extrapolated point
and four iterates are written out by hand: t_1 = 1, t_2 = phi, t_3, t_4 from
t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, y_{k+1} = x_{k+1} + ((t_k - 1)/t_{k+1})(x_{k+1} - x_k).
A wrong extrapolation direction (x_{k+1} - y_k), a momentum without t advancing (ISTA) or a
shifted t sequence each change x_3 or x_4 by more than 1e-3.

L-SVRG (Section 1.2, L-SVRG paragraph; reading R-7): the snapshot is taken at k = 0 and at
exactly the iterations whose probability-1/N coin shows 1.  Driven along coins that fire at
k = 0 mod N it is ProxSVRG, and along coins that always fire its estimator is the full
gradient (N (g_i - g_i) + grad f = grad f), i.e. ProxSkip with the full gradient.
"""
import math

import numpy as np
import pytest

import synthetic
from oracle import joseph2d, philox, solvers, tv


class _Identity:
    """A = I on an image of shape (1, 2), one subset (the solver's operator interface)."""

    N = 1
    shape = (1, 2)

    def __init__(self):
        self.D = tv.grad_operator(self.shape)

    def fwd(self, x, i=None):
        return np.asarray(x, dtype=np.float64).reshape(-1).copy()

    def adj(self, r, i=None):
        return np.asarray(r, dtype=np.float64).reshape(self.shape).copy()

    def data(self, b, i=None):
        return b


def test_fista_two_pixel_iterates_by_hand():
    # f(x) = 1/2 ||x - b||^2 (L = 1), gamma = 1/2, alpha = 0.2: every prox is prox_{0.1 TV + I+}
    # of v = y - (y - b)/2 = y/2 + (1.5, 0.5), whose pixels differ by more than 2 tau = 0.2 and
    # stay positive, so prox(v) = (v_1 - 0.1, v_2 + 0.1): x_{k+1} = y_k / 2 + (1.4, 0.6).
    op = _Identity()
    b = np.array([3.0, 1.0])
    tr = solvers.run(op, b, 0.2, "FISTA", 0.5, 4, fgp_iters=5, keep=(1, 2, 3, 4))

    phi = (1.0 + math.sqrt(5.0)) / 2.0                 # t_2
    t3 = (1.0 + math.sqrt(7.0 + 2.0 * math.sqrt(5.0))) / 2.0   # 1 + 4 phi^2 = 7 + 2 sqrt 5
    t4 = (1.0 + math.sqrt(1.0 + 4.0 * t3 * t3)) / 2.0
    c2, c3 = (phi - 1.0) / t3, (t3 - 1.0) / t4
    x1 = np.array([1.4, 0.6])                          # y_0 = x_0 = 0
    x2 = np.array([2.1, 0.9])                          # y_1 = x_1 (t_1 = 1: no momentum)
    y2 = x2 + c2 * np.array([0.7, 0.3])
    x3 = y2 / 2.0 + np.array([1.4, 0.6])
    y3 = x3 + c3 * (x3 - x2)
    x4 = y3 / 2.0 + np.array([1.4, 0.6])
    # the hand values (rounded) for a reader checking the algebra
    assert t3 == pytest.approx(2.1935271, abs=1e-7) and c2 == pytest.approx(0.2817535, abs=1e-7)
    assert x3 == pytest.approx([2.5486137, 1.0922630], abs=1e-7)
    for k, want in ((1, x1), (2, x2), (3, x3), (4, x4)):
        got = tr.iterates[k].reshape(-1)
        assert np.max(np.abs(got - want)) < 1e-14, (k, got, want)
    assert tr.prox_calls == 4
    # the plausible mistakes move x_4 (or x_3) visibly
    y3_wrong = x3 + c3 * (x3 - y2)                     # extrapolating from y_k instead of x_k
    assert np.max(np.abs(y3_wrong / 2.0 + np.array([1.4, 0.6]) - x4)) > 1e-3
    x3_ista = x2 / 2.0 + np.array([1.4, 0.6])          # t never advanced
    assert np.max(np.abs(x3_ista - x3)) > 1e-2


def test_fista_differs_from_ista_on_tomography():
    """On a real (tiny) problem the momentum changes the iterate: FISTA is not ISTA."""
    P = synthetic.make_problem_2d(12, 16, 18, 1, 3, noise="gauss", alpha=0.01)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    A = joseph2d.dense_matrix(op.g)
    L = float(np.linalg.norm(A, 2) ** 2)
    a = solvers.run(op, P.b, P.alpha, "FISTA", 1.0 / L, 6, 30)
    i = solvers.run(op, P.b, P.alpha, "ISTA", 1.0 / L, 6, 30)
    assert np.linalg.norm(a.x - i.x) > 1e-3 * np.linalg.norm(i.x)


@pytest.fixture(scope="module")
def prob():
    P = synthetic.make_problem_2d(16, 24, 24, 4, seed=11, noise="gauss", alpha=0.01)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    A = joseph2d.dense_matrix(op.g)
    L = float(np.linalg.norm(A, 2) ** 2)
    return op, P.b, P.alpha, L


def test_lsvrg_snapshots_at_k0_and_coin_iterations(prob):
    op, b, alpha, L = prob
    K, seed, p = 40, 31, 0.3
    tr = solvers.run(op, b, alpha, "VR_PROXSKIP", 1.0 / L, K, 10, p=p, seed=seed, estimator="LSVRG")
    _, _, coin = philox.schedule(seed, K, op.N, p)
    want = [0] + [k for k in range(1, K) if coin[k]]
    assert tr.snapshot_iters == want
    assert tr.snapshots == len(want)
    assert 3 <= len(want) < K // 2          # the seed gives a non-trivial refresh pattern


def test_lsvrg_with_svrg_coins_is_svrg(prob):
    op, b, alpha, L = prob
    K, seed, p, N = 24, 12, 0.4, op.N
    i, theta, _ = philox.schedule(seed, K, N, p)
    coins = np.array([k % N == 0 for k in range(K)])
    ls = solvers.run(op, b, alpha, "VR_PROXSKIP", 1.0 / L, K, 10, p=p, estimator="LSVRG",
                     draws=(i, theta, coins), keep=range(K + 1))
    sv = solvers.run(op, b, alpha, "VR_PROXSKIP", 1.0 / L, K, 10, p=p, estimator="SVRG",
                     draws=(i, theta, np.zeros(K, bool)), keep=range(K + 1))
    assert ls.snapshot_iters == sv.snapshot_iters == list(range(0, K, N))
    for k in range(K + 1):
        assert np.array_equal(ls.iterates[k], sv.iterates[k]), k
    # refreshing on the previous iteration's coin would follow another trajectory
    late = solvers.run(op, b, alpha, "VR_PROXSKIP", 1.0 / L, K, 10, p=p, estimator="LSVRG",
                       draws=(i, theta, np.roll(coins, 1)))
    assert not np.allclose(late.x, sv.x, rtol=0, atol=1e-9)


def test_lsvrg_with_every_coin_is_full_gradient_proxskip(prob):
    op, b, alpha, L = prob
    K, seed, p = 15, 5, 0.35
    i, theta, _ = philox.schedule(seed, K, op.N, p)
    ones = np.ones(K, bool)
    ls = solvers.run(op, b, alpha, "VR_PROXSKIP", 1.0 / L, K, 10, p=p, estimator="LSVRG",
                     draws=(i, theta, ones), keep=range(K + 1))
    fg = solvers.run(op, b, alpha, "PROXSKIP", 1.0 / L, K, 10, p=p, draws=(i, theta, ones), keep=range(K + 1))
    assert ls.snapshot_iters == list(range(K))
    for k in range(K + 1):
        assert np.array_equal(ls.iterates[k], fg.iterates[k]), k
    assert ls.prox_calls == fg.prox_calls == int(theta.sum())
