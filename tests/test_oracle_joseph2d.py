"""Pins of the oracle's 2D Joseph projector (CPU only).

* the ray-driven loop equals the closed-form entry formula (dense brute force);
* the scatter adjoint is the exact transpose;
* theta = 0 / 90 deg with aligned grids give exact column / row sums;
* a constant image gives the chord through the image slab along the dominant axis;
* the projection of a disc converges to the chord 2 sqrt(r^2 - s^2) as pixels shrink.
"""
import math

import numpy as np
import pytest

from oracle import joseph2d as J


def _geom(nx, ny, angles, nb, ds=1.0, pixel=1.0, N=1):
    return J.Geometry2D(nx, ny, pixel, np.asarray(angles, dtype=np.float64), nb, ds, N)


ANGLE_SETS = [
    [0.0, 0.3, math.pi / 4, 1.1, math.pi / 2, 2.0, 3 * math.pi / 4, 2.9],
    [a * math.pi / 9 for a in range(9)],
]


@pytest.mark.parametrize("nx,ny,nb,ds,pixel", [(4, 4, 7, 1.0, 1.0), (5, 3, 9, 0.7, 1.0),
                                                (6, 7, 11, 1.3, 0.8), (8, 8, 12, 1.0, 1.0)])
@pytest.mark.parametrize("angles", ANGLE_SETS)
def test_dense_equals_closed_form(nx, ny, nb, ds, pixel, angles):
    g = _geom(nx, ny, angles, nb, ds, pixel)
    A = J.dense_matrix(g)
    C = J.closed_form_matrix(g)
    assert np.max(np.abs(A - C)) < 1e-13


@pytest.mark.parametrize("nx,ny,nb", [(4, 4, 7), (5, 6, 9), (16, 16, 24)])
def test_adjoint_is_transpose(nx, ny, nb):
    g = _geom(nx, ny, ANGLE_SETS[0], nb)
    A = J.dense_matrix(g)
    B = J.dense_adjoint_matrix(g)
    assert np.max(np.abs(A.T - B)) < 1e-14


def test_adjoint_identity_random():
    g = _geom(64, 64, [a * math.pi / 90 for a in range(0, 90, 7)], 96)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((64, 64))
    ids = g.all_angles()
    y = rng.standard_normal((len(ids), 96))
    lhs = float((J.forward(g, x, ids) * y).sum())
    rhs = float((x * J.adjoint(g, y, ids)).sum())
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0) * 10


def test_theta_zero_is_column_sums():
    # 64 pixels and 96 unit bins: s_j - x_c is an integer, so every weight is 0 or 1
    g = _geom(64, 64, [0.0], 96)
    x = np.random.default_rng(1).uniform(size=(64, 64))
    y = J.forward(g, x, [0])[0]
    assert np.allclose(y[16:80], x.sum(axis=0), rtol=0, atol=1e-12)
    assert np.all(y[:16] == 0) and np.all(y[80:] == 0)


def test_theta_ninety_is_row_sums():
    g = _geom(64, 64, [math.pi / 2], 96)
    x = np.random.default_rng(2).uniform(size=(64, 64))
    y = J.forward(g, x, [0])[0]
    assert np.allclose(y[16:80], x.sum(axis=1), rtol=0, atol=1e-12)


@pytest.mark.parametrize("theta", [0.2, 0.7, math.pi / 4, 1.3, 2.5])
def test_constant_image_gives_slab_chord(theta):
    n = 40
    g = _geom(n, n, [theta], 9, ds=1.0)
    y = J.forward(g, np.ones((n, n)), [0])[0]
    c, s = abs(math.cos(theta)), abs(math.sin(theta))
    m, t = max(c, s), min(c, s)
    # a ray whose interpolation point stays within the outer pixel centres on every
    # dominant-axis line has taps summing to 1 on each line: chord = n*delta/m
    half = (n - 1) / 2.0
    inside = np.abs(g.bins()) / m + half * t / m <= half
    assert inside.sum() >= 1
    assert np.allclose(y[inside], n / m, rtol=0, atol=1e-12)
    assert np.all(y[~inside] < n / m + 1e-12)


def _disc_image(n, r_frac, sub=16):
    """Disc of radius r_frac*n/2 (pixel units), area-sampled with sub x sub points per pixel."""
    c = (np.arange(n * sub) + 0.5) / sub - n / 2.0
    X, Y = np.meshgrid(c, c)
    inside = (X * X + Y * Y <= (r_frac * n / 2.0) ** 2).astype(float)
    return inside.reshape(n, sub, n, sub).mean(axis=(1, 3))


def test_disc_projection_converges_to_chord():
    """Radon transform of a disc of radius r: 2 sqrt(r^2 - s^2) (checked away from the
    tangent rays, where the partial-volume edge dominates)."""
    errs = []
    for n in (32, 64, 128, 256):
        g = _geom(n, n, [0.0, 0.37, 1.0], n, ds=1.0)
        y = J.forward(g, _disc_image(n, 0.6), g.all_angles())
        r = 0.6 * n / 2.0
        s = g.bins()
        sel = np.abs(s) < 0.8 * r
        chord = 2.0 * np.sqrt(r * r - s[sel] ** 2)
        errs.append(np.linalg.norm(y[:, sel] - chord[None, :]) / (np.linalg.norm(chord) * np.sqrt(3)))
    assert errs[0] > errs[1] and errs[2] > errs[3]
    assert errs[3] < 1e-3


def test_smooth_bump_second_order():
    """f = (1 - rho^2/r^2)^2 on rho < r has Radon transform (16/15) (r^2 - s^2)^(5/2) / r^4;
    Joseph (linear interpolation + uniform steps) converges at second order for it."""
    errs = []
    for n in (32, 64, 128):
        c = np.arange(n) - (n - 1) / 2.0
        X, Y = np.meshgrid(c, c)
        r = 0.6 * n / 2.0
        img = np.maximum(1.0 - (X * X + Y * Y) / (r * r), 0.0) ** 2
        g = _geom(n, n, [0.0, 0.37, 1.0, math.pi / 4, 2.2], n, ds=1.0)
        y = J.forward(g, img, g.all_angles())
        a2 = np.maximum(r * r - g.bins() ** 2, 0.0)
        ref = (16.0 / 15.0) * a2 ** 2.5 / r ** 4
        errs.append(np.linalg.norm(y - ref[None, :]) / (np.linalg.norm(ref) * np.sqrt(5)))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
    assert errs[2] < 5e-4


def test_sample_count_matches_dense_support():
    g = _geom(12, 10, ANGLE_SETS[0], 17)
    # every counted sample has a nonzero tap; count taps through the dense matrix row support
    n_samples = J.sample_count(g, g.all_angles())
    assert n_samples > 0
    A = J.dense_matrix(g).reshape(len(ANGLE_SETS[0]), 17, -1)
    # a ray has at most 2 nonzero taps per line, so nnz/2 <= samples <= nnz
    nnz = int(np.count_nonzero(A))
    assert nnz / 2 <= n_samples <= nnz
