"""Algorithm 1 and its family (ISTA, FISTA, ProxSGD/SAGA/SVRG/L-SVRG, their Skip variants), float64.

The problem is Eq. (tomography_problem): F(x) = 1/2 ||Ax - b||^2 + alpha TV(x) + I_{x>=0},
split over N staggered angle subsets, f = sum_i f_i, f_i(x) = 1/2 ||A_i x - b_i||^2,
grad f_i(x) = A_i^T (A_i x - b_i) (Section 1.2).

Everything is the plain definition:
  * SAGA keeps N image-space gradients v^i and their SUM vbar (Eq. (saga_estimator)); the
    table is refreshed only at j = i_k; initial table v^i = grad f_i(x_0).
  * SVRG keeps a snapshot x~ and grad f(x~), refreshed at every k with k mod N = 0, and
    recomputes grad f_{i_k}(x~) from its definition each iteration; L-SVRG refreshes at
    k = 0 and whenever the probability-1/N coin of iteration k shows 1.
  * Skip variants follow Algorithm 1 literally: x_hat = x - gamma (G - h);
    theta ~ Bernoulli(p); x+ = prox_{(gamma/p) g}(x_hat - (gamma/p) h) if theta else x_hat;
    h += (p/gamma)(x+ - x_hat).  x_0 = 0 and h_0 = 0.
  * Non-skipped methods (ISTA, ProxSGD/SAGA/SVRG/LSVRG) take x+ = prox_{gamma g}(x - gamma G).
  * FISTA: Beck-Teboulle momentum t_1 = 1, t_{k+1} = (1+sqrt(1+4t_k^2))/2, no restart.
The prox of gamma' g is FGP with tau = gamma' alpha, the dual warm-started across calls.
Random draws come from oracle.philox.schedule (i_k, theta_k, L-SVRG coin).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import joseph2d, joseph3d, philox, tv

ALGOS = ("ISTA", "FISTA", "SVRG", "SAGA", "PROXSKIP", "VR_PROXSKIP")
ESTIMATORS = ("SVRG", "SAGA", "LSVRG", "SGD")

# default step-size factors gamma = factor / L (Section 3)
STEP_FACTOR = {"ISTA": 1.99, "PROXSKIP": 1.99, "FISTA": 1.0, "SVRG": 1.0, "LSVRG": 1.0,
               "SGD": 1.0, "SAGA": 1.0 / 3.0}


class Operator:
    """A and its subsets for a 2D (joseph2d.Geometry2D) or 3D (joseph3d.GeometryCone) geometry."""

    def __init__(self, geom):
        self.g = geom
        self.is3d = isinstance(geom, joseph3d.GeometryCone)
        self.mod = joseph3d if self.is3d else joseph2d
        self.N = geom.n_subsets
        self.shape = geom.shape() if self.is3d else (geom.ny, geom.nx)
        self._D = None

    @property
    def D(self):
        if self._D is None:
            self._D = tv.grad_operator(self.shape)
        return self._D

    def ids(self, i):
        """Angle (view) indices of subset i, or all of them when i is None."""
        if i is None:
            return self.g.all_views() if self.is3d else self.g.all_angles()
        return self.g.subset(i)

    def fwd(self, x, i=None):
        return self.mod.forward(self.g, x.reshape(self.shape), self.ids(i))

    def adj(self, r, i=None):
        return self.mod.adjoint(self.g, r, self.ids(i))

    def data(self, b, i=None):
        return b[self.ids(i)]


def grad_fi(op: Operator, b, x, i):
    return op.adj(op.fwd(x, i) - op.data(b, i), i)


def grad_f(op: Operator, b, x):
    return op.adj(op.fwd(x) - b)


def objective(op: Operator, b, x, alpha):
    r = op.fwd(x) - b
    return 0.5 * float((r * r).sum()) + alpha * tv.tv(x.reshape(op.shape), op.D)


def power_iteration(op: Operator, iters: int = 100, seed: int = 0):
    """L = lambda_max(A^T A): u_0 from Philox uniforms (tag 1), normalised; each step
    w = A^T A u, lambda = <u, w>, u = w / ||w||.  Returns the last lambda."""
    u = philox.uniform01(seed, int(np.prod(op.shape))).reshape(op.shape)
    u = u / np.linalg.norm(u)
    lam = 0.0
    for _ in range(iters):
        w = op.adj(op.fwd(u))
        lam = float((u * w).sum())
        u = w / np.linalg.norm(w)
    return lam


@dataclass
class Trace:
    x: np.ndarray
    h: np.ndarray
    dual: np.ndarray
    prox_calls: int = 0
    snapshots: int = 0
    iterates: dict = field(default_factory=dict)     # k -> x_k (after iteration k-1)
    snapshot_iters: list = field(default_factory=list)   # iterations k at which x~ was taken
    objective: dict = field(default_factory=dict)    # k -> F at the last prox output
    draws: tuple = ()
    last_prox: np.ndarray | None = None
    table: list | None = None                        # SAGA gradients v^i after the run


def run(op: Operator, b, alpha: float, algo: str, gamma: float, iters: int, fgp_iters: int,
        p: float = 1.0, seed: int = 0, estimator: str = "SVRG", nonneg: bool = True,
        x0=None, job: int = 0, keep=(), eval_every: int = 0, draws=None) -> Trace:
    """Run `iters` outer iterations of the chosen member of Algorithm 1's family.

    draws: optional (i_k, theta_k, coin_k) arrays of at least `iters` entries that replace
    the Philox schedule (used by tests to drive a run along chosen draws)."""
    algo = algo.upper()
    if algo not in ALGOS:
        raise ValueError(algo)
    est = {"ISTA": "FULL", "FISTA": "FULL", "PROXSKIP": "FULL", "SVRG": "SVRG", "SAGA": "SAGA",
           "VR_PROXSKIP": estimator.upper()}[algo]
    skip = algo in ("PROXSKIP", "VR_PROXSKIP")
    if not skip:
        p = 1.0
    N = op.N
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(op.shape) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(op.shape).copy()
    h = np.zeros(op.shape)
    dual = np.zeros(len(op.shape) * x.size)
    if draws is None:
        i_k, theta_k, coin_k = philox.schedule(seed, iters, N, p, job)
    else:
        i_k, theta_k, coin_k = (np.asarray(d) for d in draws)
    tr = Trace(x=x, h=h, dual=dual, draws=(i_k, theta_k, coin_k))

    def prox(v, scale):
        nonlocal dual
        out, dual = tv.fgp(v, scale * alpha, fgp_iters, nonneg, dual, op.D)
        tr.prox_calls += 1
        return out

    table = None
    if est == "SAGA":
        table = [grad_fi(op, b, x, i) for i in range(N)]
    x_snap = g_snap = None
    y = x.copy()            # FISTA extrapolated point
    t = 1.0
    last_prox = x.copy()
    if 0 in keep:
        tr.iterates[0] = x.copy()
    for k in range(iters):
        i = int(i_k[k])
        # ---- gradient estimator G_k (estimator table of Algorithm 1)
        if est == "FULL":
            G = grad_f(op, b, y if algo == "FISTA" else x)
        elif est == "SGD":
            G = N * grad_fi(op, b, x, i)
        elif est == "SAGA":
            vbar = sum(table)
            gi = grad_fi(op, b, x, i)
            G = N * (gi - table[i]) + vbar
            table[i] = gi
        else:   # SVRG / LSVRG
            refresh = (k % N == 0) if est == "SVRG" else (k == 0 or bool(coin_k[k]))
            if refresh:
                x_snap = x.copy()
                g_snap = grad_f(op, b, x_snap)
                tr.snapshots += 1
                tr.snapshot_iters.append(k)
            G = N * (grad_fi(op, b, x, i) - grad_fi(op, b, x_snap, i)) + g_snap
        # ---- update
        if algo == "FISTA":
            x_new = prox(y - gamma * G, gamma)
            t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
            y = x_new + ((t - 1.0) / t_next) * (x_new - x)
            t = t_next
            last_prox = x_new
        elif skip:
            x_hat = x - gamma * (G - h)
            if theta_k[k]:
                x_new = prox(x_hat - (gamma / p) * h, gamma / p)
                last_prox = x_new
            else:
                x_new = x_hat
            h = h + (p / gamma) * (x_new - x_hat)
        else:
            x_new = prox(x - gamma * G, gamma)
            last_prox = x_new
        x = x_new
        if (k + 1) in keep:
            tr.iterates[k + 1] = x.copy()
        if eval_every and (k + 1) % eval_every == 0:
            tr.objective[k + 1] = objective(op, b, last_prox, alpha)
    tr.x, tr.h, tr.dual, tr.last_prox, tr.table = x, h, dual, last_prox, table
    return tr
