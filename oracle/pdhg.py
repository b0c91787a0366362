"""Reference minimiser of Eq. (tomography_problem) by the primal-dual hybrid gradient method,
float64 (test infrastructure: imported only by tests/, __graft_entry__.smoke() and bench.py's
CPU legs).

The paper obtains its reference solution x* with a long run of preconditioned PDHG
(Section 2.1, Section 3).  Written as a saddle point with K = [A; D]:

    min_x max_{y_A, y_D}  <A x, y_A> - f*(y_A) + <D x, y_D> - g*(y_D) + I_{x >= 0}(x),
    f(z) = 1/2 ||z - b||^2,  g(w) = alpha sum_p ||w_p||_2,

one iteration is (Chambolle and Pock 2011, with x_bar = 2 x_new - x):

    y_A <- prox_{sigma_A f*}(y_A + sigma_A A x_bar) = (y_A + sigma_A (A x_bar - b)) / (1 + sigma_A)
    y_D <- projection of y_D + sigma_D D x_bar onto {||w_p||_2 <= alpha} pixel by pixel
    x_new <- max(0, x - tau (A^T y_A + D^T y_D))

Diagonal preconditioning with exponent 1 (Pock and Chambolle, ICCV 2011): tau_j =
1 / sum_i |K_ij| (column sums of A plus those of |D|) and sigma_i = 1 / sum_j |K_ij| (ray
sums of A; 1/2 for every difference row), which needs no operator norm.  Rows or columns
with zero sum get step 0.
"""
from __future__ import annotations

import numpy as np

from . import tv


def _inv(v):
    out = np.zeros_like(v)
    nz = v > 0
    out[nz] = 1.0 / v[nz]
    return out


def pdhg(op, b, alpha: float, iters: int, nonneg: bool = True, precondition: bool = True,
         x0=None, eval_every: int = 0):
    """Returns (x, history) with history = [(iteration, F(x))] every eval_every iterations.
    op: oracle.solvers.Operator; b: data shaped like op.fwd's output."""
    D = op.D
    n = int(np.prod(op.shape))
    comps = D.shape[0] // n
    absD = abs(D)
    sino = op.fwd(np.ones(n))                 # A 1 (ray sums), also fixes the sinogram shape
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    if precondition:
        tau = _inv(op.adj(np.ones(sino.shape)).reshape(-1) + np.asarray(absD.sum(axis=0)).reshape(-1))
        sig_a = _inv(sino.reshape(-1))
        sig_d = _inv(np.asarray(absD.sum(axis=1)).reshape(-1))
    else:
        # scalar steps with tau sigma ||K||^2 < 1 (power iteration on K^T K)
        u = np.random.default_rng(0).standard_normal(n)
        lam = 0.0
        for _ in range(200):
            w = op.adj(op.fwd(u)).reshape(-1) + D.T @ (D @ u)
            lam = float(u @ w) / float(u @ u)
            u = w / np.linalg.norm(w)
        s = 0.99 / np.sqrt(lam * 1.01)
        tau = np.full(n, s)
        sig_a = np.full(b.size, s)
        sig_d = np.full(D.shape[0], s)
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(-1).copy()
    xbar = x.copy()
    ya = np.zeros(b.size)
    yd = np.zeros(D.shape[0])
    hist = []
    for k in range(iters):
        ya = (ya + sig_a * (op.fwd(xbar).reshape(-1) - b)) / (1.0 + sig_a)
        w = (yd + sig_d * (D @ xbar)).reshape(comps, n)
        nrm = np.sqrt((w * w).sum(axis=0))
        yd = (w / np.maximum(1.0, nrm / alpha) if alpha > 0 else np.zeros_like(w)).reshape(-1)
        x_new = x - tau * (op.adj(ya.reshape(sino.shape)).reshape(-1) + D.T @ yd)
        if nonneg:
            x_new = np.maximum(x_new, 0.0)
        xbar = 2.0 * x_new - x
        x = x_new
        if eval_every and (k + 1) % eval_every == 0:
            r = op.fwd(x).reshape(-1) - b
            hist.append((k + 1, 0.5 * float(r @ r) + alpha * tv.tv(x.reshape(op.shape), D)))
    return x.reshape(op.shape), hist
