"""Ray-driven Joseph projector, 3D circular cone beam, float64 (oracle).

Geometry (the paper uses only 2D data; the 3D set-up follows the usual circular
cone-beam conventions): voxel (ix, iy, iz) centre ((i-(n-1)/2) delta) on each axis;
source S = SOD (cos b, sin b, 0); detector centre -(SDD-SOD)(cos b, sin b, 0);
detector axes e_u = (-sin b, cos b, 0), e_v = (0, 0, 1); pixel (iu, iv) centre
D0 + (iu-(nu-1)/2) du e_u + (iv-(nv-1)/2) dv e_v.  The ray runs from S to the pixel
centre P with direction d = P - S.

Joseph in 3D: the ray's dominant axis a = argmax_k |d_k| (ties go to x, then y) is
marched plane by plane; on the plane through voxel centres with index l along a the
ray point S + t d (t = (X_l - S_a)/d_a) is bilinearly interpolated between the four
nearest voxel centres of that plane, and each plane contributes delta |d| / |d_a|.
Taps outside the volume are zero.

forward() applies A, adjoint() scatters the same taps (A^T), closed_form_matrix()
evaluates one entry at a time from its definition (weight of a voxel = the bilinear
weight of the dominant-plane intersection times delta|d|/|d_a|) to pin the loops.
"""
from __future__ import annotations

import math

import numpy as np


class GeometryCone:
    def __init__(self, nx, ny, nz, voxel, betas, nu, nv, du, dv, sod, sdd, n_subsets):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.voxel = float(voxel)
        self.betas = np.asarray(betas, dtype=np.float64)
        self.nu, self.nv = int(nu), int(nv)
        self.du, self.dv = float(du), float(dv)
        self.sod, self.sdd = float(sod), float(sdd)
        self.n_subsets = int(n_subsets)

    @classmethod
    def from_spec(cls, s):
        return cls(s.nx, s.ny, s.nz, s.voxel, s.betas, s.nu, s.nv, s.du, s.dv, s.sod, s.sdd, s.n_subsets)

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    @property
    def n_views(self):
        return len(self.betas)

    @property
    def m(self):
        return self.n_views * self.nu * self.nv

    def subset(self, i):
        return np.arange(i, self.n_views, self.n_subsets)

    def all_views(self):
        return np.arange(self.n_views)

    def shape(self):
        return (self.nz, self.ny, self.nx)

    def rays(self, view):
        """Source S [3] and directions d [nv, nu, 3] of one view (d = pixel centre - S)."""
        b = float(self.betas[view])
        cb, sb = math.cos(b), math.sin(b)
        S = np.array([self.sod * cb, self.sod * sb, 0.0])
        D0 = np.array([-(self.sdd - self.sod) * cb, -(self.sdd - self.sod) * sb, 0.0])
        u = (np.arange(self.nu) - (self.nu - 1) / 2.0) * self.du
        v = (np.arange(self.nv) - (self.nv - 1) / 2.0) * self.dv
        d = np.empty((self.nv, self.nu, 3))
        d[..., 0] = (D0[0] + u * (-sb))[None, :] - S[0]
        d[..., 1] = (D0[1] + u * cb)[None, :] - S[1]
        d[..., 2] = v[:, None] - S[2]
        return S, d


def dominant_axis(d):
    """argmax |d_k| with ties resolved x, then y, then z."""
    ax, ay, az = np.abs(d[..., 0]), np.abs(d[..., 1]), np.abs(d[..., 2])
    return np.where((ax >= ay) & (ax >= az), 0, np.where(ay >= az, 1, 2))


_SIZES = ("nx", "ny", "nz")


def _plane_taps(g, S, d, axis, l):
    """Bilinear taps of rays (d: [R,3]) on plane l of `axis`.

    Returns the two transverse axes (b, c), tap indices (ib0, ic0), fractions (fb, fc).
    """
    b_ax, c_ax = [k for k in range(3) if k != axis]
    n_a = getattr(g, _SIZES[axis])
    X = (l - (n_a - 1) / 2.0) * g.voxel
    t = (X - S[axis]) / d[:, axis]
    pb = S[b_ax] + t * d[:, b_ax]
    pc = S[c_ax] + t * d[:, c_ax]
    ub = pb / g.voxel + (getattr(g, _SIZES[b_ax]) - 1) / 2.0
    uc = pc / g.voxel + (getattr(g, _SIZES[c_ax]) - 1) / 2.0
    ib0 = np.floor(ub).astype(np.int64)
    ic0 = np.floor(uc).astype(np.int64)
    return b_ax, c_ax, ib0, ic0, ub - ib0, uc - ic0


def _vol_index(g, axis, l, b_ax, ib, c_ax, ic):
    idx = [None, None, None]
    idx[axis] = np.full(ib.shape, l)
    idx[b_ax] = ib
    idx[c_ax] = ic
    ix, iy, iz = idx
    ok = (ix >= 0) & (ix < g.nx) & (iy >= 0) & (iy < g.ny) & (iz >= 0) & (iz < g.nz)
    return ok, (np.where(ok, iz, 0), np.where(ok, iy, 0), np.where(ok, ix, 0))


def _march(g, vol, view, out_rays=None, r_rays=None):
    """Forward (vol given, returns per-ray sums) or adjoint (r_rays given, scatters into vol)."""
    S, d = g.rays(view)
    d = d.reshape(-1, 3)
    axes = dominant_axis(d)
    dn = np.linalg.norm(d, axis=1)
    res = np.zeros(d.shape[0]) if r_rays is None else None
    for axis in range(3):
        sel = np.nonzero(axes == axis)[0]
        if sel.size == 0:
            continue
        ds = d[sel]
        scale = g.voxel * dn[sel] / np.abs(ds[:, axis])
        n_a = getattr(g, _SIZES[axis])
        for l in range(n_a):
            b_ax, c_ax, ib0, ic0, fb, fc = _plane_taps(g, S, ds, axis, l)
            for db, dc, w in ((0, 0, (1 - fb) * (1 - fc)), (1, 0, fb * (1 - fc)),
                              (0, 1, (1 - fb) * fc), (1, 1, fb * fc)):
                ok, (iz, iy, ix) = _vol_index(g, axis, l, b_ax, ib0 + db, c_ax, ic0 + dc)
                if r_rays is None:
                    res[sel] += np.where(ok, w * vol[iz, iy, ix], 0.0) * scale
                else:
                    np.add.at(vol, (iz[ok], iy[ok], ix[ok]), (w * scale * r_rays[sel])[ok])
    return res


def forward(g: GeometryCone, x, view_ids) -> np.ndarray:
    """A x for the given views: array [len(view_ids)][nv][nu]."""
    vol = np.asarray(x, dtype=np.float64).reshape(g.shape())
    out = np.zeros((len(view_ids), g.nv, g.nu))
    for r, v in enumerate(view_ids):
        out[r] = _march(g, vol, v).reshape(g.nv, g.nu)
    return out


def adjoint(g: GeometryCone, r, view_ids) -> np.ndarray:
    """A^T r for r [len(view_ids)][nv][nu]: volume [nz][ny][nx]."""
    r = np.asarray(r, dtype=np.float64).reshape(len(view_ids), g.nv * g.nu)
    vol = np.zeros(g.shape())
    for row, v in enumerate(view_ids):
        _march(g, vol, v, r_rays=r[row])
    return vol


def dense_matrix(g: GeometryCone, view_ids=None) -> np.ndarray:
    ids = g.all_views() if view_ids is None else view_ids
    A = np.zeros((len(ids) * g.nu * g.nv, g.n))
    for col in range(g.n):
        e = np.zeros(g.n)
        e[col] = 1.0
        A[:, col] = forward(g, e, ids).reshape(-1)
    return A


def closed_form_matrix(g: GeometryCone, view_ids=None) -> np.ndarray:
    """Entry by entry: voxel weight = bilinear weight on the ray's dominant plane x delta|d|/|d_a|."""
    ids = g.all_views() if view_ids is None else view_ids
    cen = [(np.arange(n) - (n - 1) / 2.0) * g.voxel for n in (g.nx, g.ny, g.nz)]
    A = np.zeros((len(ids), g.nv * g.nu, g.n))
    for r, v in enumerate(ids):
        S, d = g.rays(v)
        d = d.reshape(-1, 3)
        axes = dominant_axis(d)
        for ray in range(d.shape[0]):
            a = int(axes[ray])
            others = [k for k in range(3) if k != a]
            for iz in range(g.nz):
                for iy in range(g.ny):
                    for ix in range(g.nx):
                        c = (cen[0][ix], cen[1][iy], cen[2][iz])
                        t = (c[a] - S[a]) / d[ray, a]
                        w = 1.0
                        for k in others:
                            q = S[k] + t * d[ray, k]
                            w *= max(0.0, 1.0 - abs(q - c[k]) / g.voxel)
                        if w > 0.0:
                            A[r, ray, (iz * g.ny + iy) * g.nx + ix] = (
                                w * g.voxel * np.linalg.norm(d[ray]) / abs(d[ray, a]))
    return A.reshape(len(ids) * g.nv * g.nu, g.n)
