"""Isotropic total variation, its FGP proximal solver and an exact reference prox (oracle).

Discrete gradient D (2D: 2n x n, 3D: 3n x n): forward differences along each axis with a
zero difference at the last index (Neumann boundary).  Component order: along x (the
contiguous axis ix), along y, along z.  TV(x) = sum over pixels of ||(Dx)_pixel||_2.

prox of g = alpha TV + I_{x>=0} with scale tau (Eq. (proximal_definition)):
    prox(v) = argmin_z 1/2 ||z - v||^2 + tau TV(z) + I_{z>=0}(z).

fgp(): the fast gradient projection of Beck & Teboulle (2009) on the dual, as the paper
uses it (Section 2.1: a fixed number of warm-started inner iterations).  With dual
w (one unit vector bound per pixel), warm start w0, t_1 = 1, z_1 = w0:
    x_k     = P_+( v - tau D^T z_k )
    w_k     = P_B( z_k + D x_k / (4 d tau) )          (||D||^2 <= 4 d, d = 2 or 3)
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
    z_{k+1} = w_k + ((t_k - 1)/t_{k+1}) (w_k - w_{k-1})
and the output is P_+( v - tau D^T w_K ) with w_K kept for the next call.

prox_pdhg(): Chambolle-Pock primal-dual iterations on the same problem, an independent
algorithm used only on tiny images to obtain the exact prox the FGP must converge to.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _diff1d(n: int) -> sp.csr_matrix:
    """Forward difference on n points with a zero last row."""
    if n == 1:
        return sp.csr_matrix((1, 1))
    main = -np.ones(n)
    main[-1] = 0.0
    return sp.diags([main, np.ones(n - 1)], [0, 1], shape=(n, n), format="csr")


def grad_operator(shape) -> sp.csr_matrix:
    """D for an image of shape (ny, nx) or a volume (nz, ny, nx), row-major flattening."""
    shape = tuple(int(s) for s in shape)
    if len(shape) == 2:
        ny, nx = shape
        Dx = sp.kron(sp.identity(ny), _diff1d(nx))
        Dy = sp.kron(_diff1d(ny), sp.identity(nx))
        return sp.vstack([Dx, Dy]).tocsr()
    nz, ny, nx = shape
    Dx = sp.kron(sp.identity(nz * ny), _diff1d(nx))
    Dy = sp.kron(sp.kron(sp.identity(nz), _diff1d(ny)), sp.identity(nx))
    Dz = sp.kron(_diff1d(nz), sp.identity(ny * nx))
    return sp.vstack([Dx, Dy, Dz]).tocsr()


def tv(x: np.ndarray, D: sp.csr_matrix | None = None) -> float:
    x = np.asarray(x, dtype=np.float64)
    D = grad_operator(x.shape) if D is None else D
    g = (D @ x.reshape(-1)).reshape(-1, x.size)
    return float(np.sqrt((g * g).sum(axis=0)).sum())


def _project_ball(w: np.ndarray, comps: int) -> np.ndarray:
    w = w.reshape(comps, -1)
    nrm = np.sqrt((w * w).sum(axis=0))
    return (w / np.maximum(1.0, nrm)).reshape(-1)


def fgp(v: np.ndarray, tau: float, iters: int, nonneg: bool = True, w0: np.ndarray | None = None,
        D: sp.csr_matrix | None = None):
    """K FGP iterations from dual w0 (zeros when None). Returns (x_plus, w_K)."""
    v = np.asarray(v, dtype=np.float64)
    shape = v.shape
    d = len(shape)
    D = grad_operator(shape) if D is None else D
    DT = D.T.tocsr()
    vf = v.reshape(-1)
    comps = d
    w = np.zeros(comps * vf.size) if w0 is None else np.asarray(w0, dtype=np.float64).reshape(-1).copy()
    step = 1.0 / (4.0 * d * tau)
    proj_x = (lambda y: np.maximum(y, 0.0)) if nonneg else (lambda y: y)
    z = w.copy()
    w_prev = w.copy()
    t = 1.0
    for _ in range(iters):
        x = proj_x(vf - tau * (DT @ z))
        w_new = _project_ball(z + step * (D @ x), comps)
        t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = w_new + ((t - 1.0) / t_next) * (w_new - w_prev)
        w_prev = w_new
        t = t_next
    w_out = w_prev
    x_out = proj_x(vf - tau * (DT @ w_out))
    return x_out.reshape(shape), w_out


def prox_pdhg(v: np.ndarray, tau: float, nonneg: bool = True, iters: int = 200000, tol: float = 1e-13):
    """Exact prox by Chambolle-Pock on min_z 1/2||z-v||^2 + I_+(z) + tau ||Dz||_{2,1}.

    Primal step s, dual step r with s r ||D||^2 < 1; the z-update is the prox of
    1/2||.-v||^2 + I_+ (a clipped average), the dual update projects onto tau-balls.
    """
    v = np.asarray(v, dtype=np.float64)
    shape = v.shape
    d = len(shape)
    D = grad_operator(shape)
    DT = D.T.tocsr()
    vf = v.reshape(-1)
    L2 = 4.0 * d
    s = r = 0.99 / np.sqrt(L2)
    z = vf.copy()
    zbar = z.copy()
    y = np.zeros(D.shape[0])
    for it in range(iters):
        y = y + r * (D @ zbar)
        y = tau * _project_ball(y / tau, d)
        z_new = (z - s * (DT @ y) + s * vf) / (1.0 + s)
        if nonneg:
            z_new = np.maximum(z_new, 0.0)
        zbar = 2.0 * z_new - z
        delta = np.max(np.abs(z_new - z))
        z = z_new
        if delta < tol:
            break
    return z.reshape(shape)
