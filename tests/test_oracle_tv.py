"""Pins of the oracle's TV operator, FGP prox and exact reference prox (CPU only)."""
import numpy as np
import pytest
from scipy.optimize import lsq_linear

from oracle import tv


def _brute_grad(x):
    """Forward differences by explicit index loops, zero at the last index of each axis."""
    x = np.asarray(x)
    out = []
    for axis in reversed(range(x.ndim)):        # component order: x (last axis), y, z
        g = np.zeros_like(x)
        it = np.nditer(x, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            if idx[axis] + 1 < x.shape[axis]:
                nxt = list(idx)
                nxt[axis] += 1
                g[idx] = x[tuple(nxt)] - x[idx]
        out.append(g.reshape(-1))
    return np.concatenate(out)


@pytest.mark.parametrize("shape", [(3, 4), (5, 2), (1, 6), (3, 4, 2), (2, 3, 5)])
def test_grad_operator_brute_force(shape):
    x = np.random.default_rng(0).standard_normal(shape)
    D = tv.grad_operator(shape)
    assert np.allclose(D @ x.reshape(-1), _brute_grad(x), rtol=0, atol=1e-14)


def test_tv_hand_example():
    # 2x2 image [[0, 3], [4, 0]]: pixel (0,0): (3, 4) -> 5; pixel (0,1): (0, -3) -> 3;
    # pixel (1,0): (-4, 0) -> 4; pixel (1,1): (0, 0) -> 0.  TV = 12.
    x = np.array([[0.0, 3.0], [4.0, 0.0]])
    assert tv.tv(x) == pytest.approx(12.0, abs=1e-14)


def test_operator_norm_bound():
    for shape, bound in (((9, 11), 8.0), ((5, 6, 7), 12.0)):
        D = tv.grad_operator(shape).toarray()
        assert np.linalg.norm(D, 2) ** 2 <= bound


def test_two_pixel_closed_forms():
    tau = 0.3
    # a - b > 2 tau, both stay positive: (a - tau, b + tau)
    x, _ = tv.fgp(np.array([[2.0, 1.0]]), tau, 3000)
    assert np.allclose(x, [[1.7, 1.3]], atol=1e-9)
    # |a - b| <= 2 tau: both take the mean
    x, _ = tv.fgp(np.array([[1.2, 1.0]]), tau, 3000)
    assert np.allclose(x, [[1.1, 1.1]], atol=1e-9)
    # nonnegativity active: [0.1, -2] -> without the constraint (0.1 - .3 ... ) the mean rule
    # gives -0.95 each; with it the minimiser is z = 0 for both when the mean is negative
    x, _ = tv.fgp(np.array([[0.1, -2.0]]), tau, 3000, nonneg=True)
    assert np.allclose(x, [[0.0, 0.0]], atol=1e-9)
    x, _ = tv.fgp(np.array([[0.1, -2.0]]), tau, 3000, nonneg=False)
    assert np.allclose(x, [[-0.2, -1.7]], atol=1e-9)


def test_constant_input_is_fixed():
    v = np.full((6, 5), 0.7)
    x, w = tv.fgp(v, 0.5, 10)
    assert np.array_equal(x, v)
    assert not np.any(w)


def test_large_tau_gives_mean():
    v = np.random.default_rng(3).uniform(size=(5, 6))
    x, _ = tv.fgp(v, 50.0, 20000)
    assert np.allclose(x, v.mean(), atol=1e-6)


def test_one_dimensional_prox_matches_box_qp():
    """1D TV prox (no sign constraint) = v - D^T w*, w* = argmin ||D^T w - v||, |w| <= tau:
    a bounded least-squares problem solved by scipy's lsq_linear."""
    rng = np.random.default_rng(4)
    v = rng.standard_normal((1, 12)) * 2
    tau = 0.4
    D = tv.grad_operator((1, 12)).toarray()[:12]      # x-component rows (y rows are zero)
    res = lsq_linear(D.T, v.reshape(-1), bounds=(-tau, tau), tol=1e-14, method="bvls")
    ref = v.reshape(-1) - D.T @ res.x
    x, _ = tv.fgp(v, tau, 20000, nonneg=False)
    assert np.allclose(x.reshape(-1), ref, atol=1e-8)


@pytest.mark.parametrize("shape", [(3, 3), (4, 5), (6, 6), (3, 3, 3)])
def test_fgp_converges_to_pdhg_prox(shape):
    rng = np.random.default_rng(sum(shape))
    v = rng.uniform(-0.3, 1.0, size=shape)
    tau = 0.15
    exact = tv.prox_pdhg(v, tau, nonneg=True)
    x, _ = tv.fgp(v, tau, 20000, nonneg=True)
    assert np.max(np.abs(x - exact)) < 1e-7
    # optimality: the prox objective at x is not above that at perturbed feasible points
    obj = lambda z: 0.5 * np.sum((z - v) ** 2) + tau * tv.tv(z)
    for _ in range(20):
        z = np.maximum(x + 1e-3 * rng.standard_normal(shape), 0.0)
        assert obj(z) >= obj(x) - 1e-12


def test_warm_start_continues_iterations():
    """Warm starting from w_K and running more iterations approaches the same prox."""
    v = np.random.default_rng(5).uniform(size=(8, 8))
    x_ref, _ = tv.fgp(v, 0.2, 5000)
    x1, w1 = tv.fgp(v, 0.2, 10)
    err1 = np.abs(x1 - x_ref).max()
    x2, w2 = tv.fgp(v, 0.2, 10, w0=w1)
    err2 = np.abs(x2 - x_ref).max()
    assert err2 < err1
    nrm = np.sqrt((w2.reshape(2, -1) ** 2).sum(0))
    assert np.all(nrm <= 1 + 1e-12)
