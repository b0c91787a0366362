"""Pins of the oracle's 3D cone-beam Joseph projector (CPU only).

* the ray-driven loop equals an entry-by-entry evaluation of the definition (brute force),
  including a view at 45 degrees where the dominant axis switches inside the view;
* the scatter adjoint is the exact transpose and satisfies <Ax, y> = <x, A^T y>;
* a constant volume gives the chord through the slab along the dominant axis;
* the projection of a ball converges to the chord 2 sqrt(r^2 - rho^2).
"""
import math

import numpy as np
import pytest

from oracle import joseph3d as J


def _geom(n, voxel, betas, det, d, sod, sdd, N=1):
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    nu, nv = (det, det) if np.isscalar(det) else det
    return J.GeometryCone(nx, ny, nz, voxel, np.asarray(betas, dtype=np.float64), nu, nv, d, d, sod, sdd, N)


def test_dense_equals_definition_small():
    betas = [0.0, 0.4, math.pi / 4, 2.0]
    g = _geom((5, 4, 3), 1.0, betas, (6, 5), 1.3, 20.0, 40.0)
    A = J.dense_matrix(g)
    C = J.closed_form_matrix(g)
    assert np.max(np.abs(A - C)) < 1e-12
    # the 45-degree view has rays of both dominant axes
    S, d = g.rays(2)
    ax = J.dominant_axis(d)
    assert (ax == 0).any() and (ax == 1).any()


def test_adjoint_is_transpose_small():
    g = _geom(4, 1.0, [0.1, math.pi / 4, 1.9], 5, 1.5, 15.0, 30.0)
    A = J.dense_matrix(g)
    m = A.shape[0]
    B = np.zeros((g.n, m))
    for col in range(m):
        e = np.zeros(m)
        e[col] = 1.0
        B[:, col] = J.adjoint(g, e.reshape(3, g.nv, g.nu), g.all_views()).reshape(-1)
    assert np.max(np.abs(A.T - B)) < 1e-13


def test_adjoint_identity_random():
    g = _geom(12, 0.5, [0.0, 0.7, math.pi / 4, 2.6, 4.0], 18, 1.0, 60.0, 120.0)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(g.shape())
    y = rng.standard_normal((5, g.nv, g.nu))
    lhs = float((J.forward(g, x, g.all_views()) * y).sum())
    rhs = float((x * J.adjoint(g, y, g.all_views())).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_constant_volume_slab_chord():
    n, voxel = 16, 0.5
    g = _geom(n, voxel, [0.3], 9, 0.25, 200.0, 400.0)
    y = J.forward(g, np.ones(g.shape()), [0])[0]
    S, d = g.rays(0)
    ax = J.dominant_axis(d)
    assert np.all(ax == 0)
    # for rays that stay within the outer voxel centres on every x plane, each plane's
    # bilinear taps sum to 1: value = n * voxel * |d| / |d_x| (the chord through the slab)
    half = (n - 1) / 2.0 * voxel
    ok = np.ones(d.shape[:2], bool)
    for l in (0, n - 1):
        X = (l - (n - 1) / 2.0) * voxel
        t = (X - S[0]) / d[..., 0]
        for k in (1, 2):
            ok &= np.abs(S[k] + t * d[..., k]) <= half
    assert ok.sum() > 10
    ref = n * voxel * np.linalg.norm(d, axis=-1) / np.abs(d[..., 0])
    assert np.allclose(y[ok], ref[ok], rtol=0, atol=1e-11)


def _ball(n, voxel, radius, sub=4):
    c = ((np.arange(n * sub) + 0.5) / sub - n / 2.0) * voxel
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    inside = (X * X + Y * Y + Z * Z <= radius * radius).astype(float)
    return inside.reshape(n, sub, n, sub, n, sub).mean(axis=(1, 3, 5))


def test_ball_projection_converges_to_chord():
    """A ball of radius r at the origin: a ray at distance rho from the centre has chord
    2 sqrt(r^2 - rho^2).  Checked on rays with rho < 0.8 r."""
    errs = []
    radius = 3.0
    for n in (12, 24):
        voxel = 8.0 / n
        g = _geom(n, voxel, [0.0, 0.9], 24, 0.5, 40.0, 80.0)
        y = J.forward(g, _ball(n, voxel, radius), g.all_views())
        e = []
        for r_i, v in enumerate(g.all_views()):
            S, d = g.rays(v)
            dn = d / np.linalg.norm(d, axis=-1, keepdims=True)
            # distance from the origin to the line S + t d
            proj = -(S[None, None, :] * dn).sum(-1)
            rho2 = (S * S).sum() - proj ** 2
            sel = rho2 < (0.8 * radius) ** 2
            chord = 2.0 * np.sqrt(radius * radius - rho2[sel])
            e.append((y[r_i][sel] - chord) / chord)
        errs.append(np.sqrt(np.mean(np.concatenate(e) ** 2)))
    assert errs[1] < errs[0]
    assert errs[1] < 0.01
