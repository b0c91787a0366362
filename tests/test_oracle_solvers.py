"""Pins of the oracle's Algorithm-1 family (CPU only).

* staggered subsets reproduce the paper's N = 5 example and partition the angles;
* the SAGA and SVRG estimators are unbiased (exact enumeration over i);
* SAGA refreshes exactly one table slot per step;
* ProxSkip with p = 1 equals ISTA, ProxSVRGSkip(p=1) equals ProxSVRG (Section 1.1);
* a skipped step (theta = 0) leaves h unchanged bit for bit (Algorithm 1);
* ISTA decreases F monotonically for gamma = 1/L with an accurate prox;
* the power iteration finds ||A||_2^2 of the dense matrix.
"""
import math
import os

import numpy as np
import pytest

import synthetic
from oracle import joseph2d, philox, solvers, tv


def _problem(n=16, n_angles=24, nb=24, N=4, seed=11):
    P = synthetic.make_problem_2d(n, n_angles, nb, N, seed, noise="gauss", alpha=0.01)
    op = solvers.Operator(joseph2d.Geometry2D.from_spec(P.spec))
    return op, P.b, P.alpha


@pytest.fixture(scope="module")
def small():
    op, b, alpha = _problem()
    A = joseph2d.dense_matrix(op.g)
    L = float(np.linalg.norm(A, 2) ** 2)
    return op, b, alpha, L


def test_staggered_subsets_match_paper_example(golden_dir):
    g = joseph2d.Geometry2D(4, 4, 1.0, np.zeros(25), 4, 1.0, 5)
    with open(os.path.join(golden_dir, "staggered_subsets_N5.txt")) as f:
        rows = [l for l in f if l.strip() and not l.startswith("#")]
    for line in rows:
        k, ids = line.split(":")
        assert list(g.subset(int(k))) == [int(t) for t in ids.split()]
    allids = np.sort(np.concatenate([g.subset(i) for i in range(5)]))
    assert np.array_equal(allids, np.arange(25))


def test_full_gradient_is_sum_of_subset_gradients(small):
    op, b, _, _ = small
    x = np.random.default_rng(0).uniform(size=op.shape)
    full = solvers.grad_f(op, b, x)
    parts = sum(solvers.grad_fi(op, b, x, i) for i in range(op.N))
    assert np.allclose(full, parts, rtol=0, atol=1e-11)


def test_power_iteration_matches_dense_norm(small):
    op, _, _, L = small
    lam = solvers.power_iteration(op, iters=300, seed=5)
    assert lam == pytest.approx(L, rel=1e-8)


def test_estimators_unbiased(small):
    op, b, _, _ = small
    rng = np.random.default_rng(1)
    x = rng.uniform(size=op.shape)
    x_snap = rng.uniform(size=op.shape)
    N = op.N
    g_true = solvers.grad_f(op, b, x)
    # SVRG: E_i[N(grad f_i(x) - grad f_i(x~)) + grad f(x~)] = grad f(x)
    g_snap = solvers.grad_f(op, b, x_snap)
    est = [N * (solvers.grad_fi(op, b, x, i) - solvers.grad_fi(op, b, x_snap, i)) + g_snap for i in range(N)]
    assert np.allclose(np.mean(est, axis=0), g_true, atol=1e-10)
    # SAGA with an arbitrary table
    table = [rng.uniform(size=op.shape) for _ in range(N)]
    vbar = sum(table)
    est = [N * (solvers.grad_fi(op, b, x, i) - table[i]) + vbar for i in range(N)]
    assert np.allclose(np.mean(est, axis=0), g_true, atol=1e-10)


def test_p_one_proxskip_equals_ista(small):
    op, b, alpha, L = small
    gamma = 1.0 / L
    a = solvers.run(op, b, alpha, "ISTA", gamma, 12, fgp_iters=20, seed=3, keep=range(13))
    s = solvers.run(op, b, alpha, "PROXSKIP", gamma, 12, fgp_iters=20, p=1.0, seed=3, keep=range(13))
    for k in range(13):
        assert np.allclose(a.iterates[k], s.iterates[k], rtol=0, atol=1e-12)
    assert a.prox_calls == s.prox_calls == 12


def test_p_one_svrg_skip_equals_svrg(small):
    op, b, alpha, L = small
    gamma = 1.0 / L
    a = solvers.run(op, b, alpha, "SVRG", gamma, 10, fgp_iters=20, seed=4, keep=[10])
    s = solvers.run(op, b, alpha, "VR_PROXSKIP", gamma, 10, fgp_iters=20, p=1.0, seed=4,
                    estimator="SVRG", keep=[10])
    assert np.allclose(a.iterates[10], s.iterates[10], rtol=0, atol=1e-12)


def test_skipped_step_keeps_h(small):
    op, b, alpha, L = small
    gamma, p, seed = 1.0 / L, 0.3, 21
    i, theta, _ = philox.schedule(seed, 40, op.N, p)
    k0 = int(np.nonzero(~theta[1:])[0][0]) + 1          # a skipped iteration after the first
    tr_a = solvers.run(op, b, alpha, "VR_PROXSKIP", gamma, k0, 10, p=p, seed=seed)
    tr_b = solvers.run(op, b, alpha, "VR_PROXSKIP", gamma, k0 + 1, 10, p=p, seed=seed)
    assert np.array_equal(tr_a.h, tr_b.h)
    assert not np.array_equal(tr_a.x, tr_b.x)


def test_saga_refreshes_one_slot(small):
    """After two SAGA steps from x_0 (the table starts at grad f_i(x_0)), only slot i_1
    differs from grad f_j(x_0), and it holds grad f_{i_1}(x_1)."""
    op, b, alpha, L = small
    x0 = np.random.default_rng(2).uniform(size=op.shape)
    seed = 8
    t1 = solvers.run(op, b, alpha, "SAGA", 1.0 / (3 * L), 1, 10, seed=seed, x0=x0)
    t2 = solvers.run(op, b, alpha, "SAGA", 1.0 / (3 * L), 2, 10, seed=seed, x0=x0)
    i1 = int(t2.draws[0][1])
    for j in range(op.N):
        ref = solvers.grad_fi(op, b, x0, j)
        if j == i1:
            assert np.allclose(t2.table[j], solvers.grad_fi(op, b, t1.x, j), rtol=0, atol=1e-12)
            assert not np.allclose(t2.table[j], ref)
        else:
            assert np.array_equal(t2.table[j], ref)


def test_ista_monotone_with_accurate_prox(small):
    op, b, alpha, L = small
    tr = solvers.run(op, b, 0.05, "ISTA", 1.0 / L, 15, fgp_iters=400, seed=0, eval_every=1)
    F = [tr.objective[k] for k in range(1, 16)]
    assert all(F[k + 1] <= F[k] + 1e-10 * abs(F[k]) for k in range(len(F) - 1))


def test_vr_methods_decrease_objective(small):
    op, b, alpha, L = small
    F0 = solvers.objective(op, b, np.zeros(op.shape), alpha)
    for algo, est, fac, p in (("SAGA", "SVRG", 1 / 3, 1.0), ("SVRG", "SVRG", 1.0, 1.0),
                              ("VR_PROXSKIP", "SVRG", 1.0, 0.3), ("VR_PROXSKIP", "SAGA", 1 / 3, 0.3),
                              ("VR_PROXSKIP", "LSVRG", 1.0, 0.3), ("FISTA", "SVRG", 1.0, 1.0)):
        tr = solvers.run(op, b, alpha, algo, fac / L, 40, fgp_iters=20, p=p, seed=9, estimator=est)
        F = solvers.objective(op, b, tr.last_prox, alpha)
        assert F < 0.5 * F0, (algo, est)


def test_skip_variant_prox_count_follows_coins(small):
    op, b, alpha, L = small
    p, seed, K = 0.2, 5, 60
    tr = solvers.run(op, b, alpha, "VR_PROXSKIP", 1.0 / L, K, 10, p=p, seed=seed)
    _, theta, _ = philox.schedule(seed, K, op.N, p)
    assert tr.prox_calls == int(theta.sum())


def test_stopping_after_last_prox_returns_evaluated_point(small):
    """The time-to-gap measurements evaluate F at the last prox output before iteration k and
    stop a run right after that prox step (iteration j, the last with theta_j = 1 below k):
    the run's final iterate x_{j+1} is exactly the point that was evaluated."""
    op, b, alpha, L = small
    p, seed, N = 0.2, 9, op.N
    k = 6 * N
    tr = solvers.run(op, b, alpha, "VR_PROXSKIP", 1.0 / L, k, 10, p=p, seed=seed, estimator="SAGA",
                     eval_every=N)
    _, theta, _ = philox.schedule(seed, k, N, p)
    j = int(np.nonzero(theta)[0][-1])
    short = solvers.run(op, b, alpha, "VR_PROXSKIP", 1.0 / L, j + 1, 10, p=p, seed=seed, estimator="SAGA")
    assert np.array_equal(short.x, tr.last_prox)
    assert solvers.objective(op, b, short.x, alpha) == tr.objective[k]
    if j + 1 < k:
        # the iterate at k itself is a gradient step past the prox point
        assert not np.array_equal(tr.x, tr.last_prox)
