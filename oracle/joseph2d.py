"""Ray-driven Joseph projector, 2D parallel beam, float64 (oracle).

The paper calls A "the discrete Radon transform" (Section 2.1) without naming a
discretisation; this library uses Joseph's method (linear interpolation along the axis
the ray is least aligned with).  Conventions (pixel size delta, centred grids):

  pixel (ix, iy) centre  (x_c, y_c) = ((ix-(nx-1)/2) delta, (iy-(ny-1)/2) delta)
  bin j position         s_j = (j-(nb-1)/2) ds
  ray (theta, j)         {x cos(theta) + y sin(theta) = s_j}

A ray with |cos theta| >= |sin theta| is marched row by row (y dominant; a tie goes to y):
on row iy it meets x = (s_j - y_c sin)/cos, which is linearly interpolated between the two
nearest pixel centres of that row; each row contributes delta/|cos theta|.  Otherwise the
ray is marched column by column with the roles of x and y swapped.  Taps outside the
image are zero.  The dominant-axis test is taken in float64 from math.cos/math.sin of the
float64 angle.

forward() applies A to an image; adjoint() applies A^T by scattering the same taps
(the literal transpose of the same loop).  dense_matrix() builds A column by column, and
closed_form_matrix() evaluates the entry formula
    A[(theta, j), (ix, iy)] = (delta/m) * max(0, 1 - |s_j - s_c|/(delta m)),
    m = max(|cos|, |sin|),  s_c = x_c cos + y_c sin,
which the tests use to pin the ray-driven loop.
"""
from __future__ import annotations

import math

import numpy as np


class Geometry2D:
    """Oracle-side description of a 2D parallel-beam acquisition with N staggered subsets."""

    def __init__(self, nx, ny, pixel, angles, n_bins, bin_spacing, n_subsets):
        self.nx, self.ny = int(nx), int(ny)
        self.pixel = float(pixel)
        self.angles = np.asarray(angles, dtype=np.float64)
        self.n_bins = int(n_bins)
        self.bin_spacing = float(bin_spacing)
        self.n_subsets = int(n_subsets)

    @classmethod
    def from_spec(cls, spec):
        return cls(spec.nx, spec.ny, spec.pixel, spec.angles, spec.n_bins, spec.bin_spacing, spec.n_subsets)

    @property
    def n(self):
        return self.nx * self.ny

    @property
    def n_angles(self):
        return len(self.angles)

    @property
    def m(self):
        return self.n_angles * self.n_bins

    def bins(self):
        return (np.arange(self.n_bins) - (self.n_bins - 1) / 2.0) * self.bin_spacing

    def subset(self, i):
        """Staggered subset i: angles {i, i+N, i+2N, ...} (Fig. 1 caption)."""
        return np.arange(i, self.n_angles, self.n_subsets)

    def all_angles(self):
        return np.arange(self.n_angles)

    def trig(self, a):
        th = float(self.angles[a])
        return math.cos(th), math.sin(th)


def _gather(line, idx, w):
    ok = (idx >= 0) & (idx < line.shape[0])
    out = np.zeros_like(w)
    out[ok] = w[ok] * line[idx[ok]]
    return out


def _scatter(line, idx, vals):
    ok = (idx >= 0) & (idx < line.shape[0])
    np.add.at(line, idx[ok], vals[ok])


def _taps(g, c, s, line_index):
    """Interpolation taps of every bin's ray on one dominant-axis line.

    Returns (i0, f, weight): taps i0 (weight 1-f) and i0+1 (weight f) along the line,
    and the per-line length factor delta/m.
    """
    sj = g.bins()
    if abs(c) >= abs(s):       # rows
        y = (line_index - (g.ny - 1) / 2.0) * g.pixel
        xs = (sj - y * s) / c
        u = xs / g.pixel + (g.nx - 1) / 2.0
        scale = g.pixel / abs(c)
    else:                       # columns
        x = (line_index - (g.nx - 1) / 2.0) * g.pixel
        ys = (sj - x * c) / s
        u = ys / g.pixel + (g.ny - 1) / 2.0
        scale = g.pixel / abs(s)
    i0 = np.floor(u).astype(np.int64)
    return i0, u - i0, scale


def forward(g: Geometry2D, x, angle_ids) -> np.ndarray:
    """Rows of A x for the given angle indices: array [len(angle_ids)][n_bins]."""
    img = np.asarray(x, dtype=np.float64).reshape(g.ny, g.nx)
    out = np.zeros((len(angle_ids), g.n_bins))
    for r, a in enumerate(angle_ids):
        c, s = g.trig(a)
        rows = abs(c) >= abs(s)
        n_lines = g.ny if rows else g.nx
        acc = np.zeros(g.n_bins)
        for l in range(n_lines):
            i0, f, scale = _taps(g, c, s, l)
            line = img[l, :] if rows else img[:, l]
            acc += _gather(line, i0, 1.0 - f) + _gather(line, i0 + 1, f)
        out[r] = acc * scale
    return out


def adjoint(g: Geometry2D, r, angle_ids) -> np.ndarray:
    """A^T r for rows r[len(angle_ids)][n_bins]: image [ny][nx] (scatter of the forward taps)."""
    r = np.asarray(r, dtype=np.float64).reshape(len(angle_ids), g.n_bins)
    img = np.zeros((g.ny, g.nx))
    for row, a in enumerate(angle_ids):
        c, s = g.trig(a)
        rows = abs(c) >= abs(s)
        n_lines = g.ny if rows else g.nx
        for l in range(n_lines):
            i0, f, scale = _taps(g, c, s, l)
            line = img[l, :] if rows else img[:, l]      # views: scatter lands in img
            _scatter(line, i0, (1.0 - f) * r[row] * scale)
            _scatter(line, i0 + 1, f * r[row] * scale)
    return img


def dense_matrix(g: Geometry2D, angle_ids=None) -> np.ndarray:
    """A as a dense [m_sub][n] matrix, one forward projection per unit image."""
    ids = g.all_angles() if angle_ids is None else angle_ids
    A = np.zeros((len(ids) * g.n_bins, g.n))
    for col in range(g.n):
        e = np.zeros(g.n)
        e[col] = 1.0
        A[:, col] = forward(g, e, ids).reshape(-1)
    return A


def dense_adjoint_matrix(g: Geometry2D, angle_ids=None) -> np.ndarray:
    """A^T as a dense [n][m_sub] matrix, one back projection per unit sinogram."""
    ids = g.all_angles() if angle_ids is None else angle_ids
    m = len(ids) * g.n_bins
    B = np.zeros((g.n, m))
    for col in range(m):
        e = np.zeros(m)
        e[col] = 1.0
        B[:, col] = adjoint(g, e, ids).reshape(-1)
    return B


def closed_form_matrix(g: Geometry2D, angle_ids=None) -> np.ndarray:
    """A from the entry formula (delta/m) max(0, 1 - |s_j - s_c|/(delta m))."""
    ids = g.all_angles() if angle_ids is None else angle_ids
    xc = (np.arange(g.nx) - (g.nx - 1) / 2.0) * g.pixel
    yc = (np.arange(g.ny) - (g.ny - 1) / 2.0) * g.pixel
    XC, YC = np.meshgrid(xc, yc)            # [ny][nx]
    sj = g.bins()
    A = np.zeros((len(ids), g.n_bins, g.n))
    for r, a in enumerate(ids):
        c, s = g.trig(a)
        mth = max(abs(c), abs(s))
        sc = (XC * c + YC * s).reshape(-1)
        A[r] = (g.pixel / mth) * np.maximum(0.0, 1.0 - np.abs(sj[:, None] - sc[None, :]) / (g.pixel * mth))
    return A.reshape(len(ids) * g.n_bins, g.n)


def sample_count(g: Geometry2D, angle_ids) -> int:
    """Number of Joseph samples (ray, dominant-axis line) with at least one tap inside the image."""
    total = 0
    for a in angle_ids:
        c, s = g.trig(a)
        rows = abs(c) >= abs(s)
        n_lines = g.ny if rows else g.nx
        n_cols = g.nx if rows else g.ny
        for l in range(n_lines):
            i0, f, _ = _taps(g, c, s, l)
            total += int(np.count_nonzero((i0 >= -1) & (i0 <= n_cols - 1) & ~((i0 == -1) & (f == 0.0))))
    return total
