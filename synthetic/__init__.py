"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the reconstruction method's arithmetic. It only makes the
inputs a reconstruction starts from:

* random ellipse (2D) and ellipsoid (3D) phantoms, drawn with numpy's PCG64 generator;
* closed-form line integrals of those phantoms (the "analytic projection data" the paper
  uses for its simulated experiment, Section 2.2), so that the measured data are not made
  with the projector under test;
* measurement noise: Gaussian, or Poisson photon counts followed by the log transform.

Geometry conventions (shared statement of the acquisition set-up, Section 2.1 "discrete
Radon transform"; the paper fixes none of them):

* 2D parallel beam: pixel (ix, iy) has its centre at ((ix-(nx-1)/2)*pixel,
  (iy-(ny-1)/2)*pixel); detector bin j sits at s_j = (j-(nb-1)/2)*bin_spacing; the ray of
  angle theta and bin j is the line {x cos(theta) + y sin(theta) = s_j}.  Images are
  stored row-major [ny][nx], sinograms [n_angles][nb].
* 3D circular cone beam: source S = SOD*(cos b, sin b, 0); detector centre
  -(SDD-SOD)*(cos b, sin b, 0); detector axes e_u = (-sin b, cos b, 0), e_v = (0, 0, 1);
  pixel (iu, iv) centre at (iu-(nu-1)/2)*du, (iv-(nv-1)/2)*dv.  Volumes are stored
  [nz][ny][nx], projections [n_views][nv][nu].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Par2DSpec", "Cone3DSpec", "Problem2D", "Problem3D",
    "random_ellipses", "rasterize_ellipses", "ellipse_sinogram",
    "random_ellipsoids", "rasterize_ellipsoids", "ellipsoid_cone_projections",
    "gaussian_noise", "poisson_log_noise", "make_problem_2d", "make_problem_3d",
    "WORKLOADS_2D", "WORKLOADS_3D", "uniform_angles",
]


# --------------------------------------------------------------------------- geometry specs
@dataclass(frozen=True)
class Par2DSpec:
    nx: int
    ny: int
    pixel: float
    angles: np.ndarray          # radians, float64
    n_bins: int
    bin_spacing: float
    n_subsets: int

    def bin_centers(self) -> np.ndarray:
        return (np.arange(self.n_bins) - (self.n_bins - 1) / 2.0) * self.bin_spacing


@dataclass(frozen=True)
class Cone3DSpec:
    nx: int
    ny: int
    nz: int
    voxel: float
    betas: np.ndarray           # source angles, radians, float64
    nu: int
    nv: int
    du: float
    dv: float
    sod: float
    sdd: float
    n_subsets: int


def uniform_angles(n: int, span: float) -> np.ndarray:
    """n angles a*span/n, a = 0..n-1 (span = pi for [0, 180) degrees, 2*pi for a full turn)."""
    return np.array([a * span / n for a in range(n)], dtype=np.float64)


# --------------------------------------------------------------------------- 2D phantoms
def random_ellipses(n_ellipses: int, fov_radius: float, rng: np.random.Generator) -> np.ndarray:
    """Rows (cx, cy, a, b, phi, intensity).

    Centres uniform in the disc of radius 0.5*R, semi-axes U[0.05, 0.35]*R, rotation
    U[0, pi), intensity U[0, 1]; the ellipses add up where they overlap.
    """
    out = np.empty((n_ellipses, 6))
    for e in range(n_ellipses):
        r = 0.5 * fov_radius * math.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * math.pi)
        out[e, 0] = r * math.cos(ang)
        out[e, 1] = r * math.sin(ang)
        out[e, 2] = rng.uniform(0.05, 0.35) * fov_radius
        out[e, 3] = rng.uniform(0.05, 0.35) * fov_radius
        out[e, 4] = rng.uniform(0.0, math.pi)
        out[e, 5] = rng.uniform(0.0, 1.0)
    return out


def rasterize_ellipses(ell: np.ndarray, nx: int, ny: int, pixel: float) -> np.ndarray:
    """Ground-truth image: each pixel takes the summed intensity of the ellipses holding its centre."""
    xs = (np.arange(nx) - (nx - 1) / 2.0) * pixel
    ys = (np.arange(ny) - (ny - 1) / 2.0) * pixel
    X, Y = np.meshgrid(xs, ys)
    img = np.zeros((ny, nx))
    for cx, cy, a, b, phi, mu in ell:
        c, s = math.cos(phi), math.sin(phi)
        xr = (X - cx) * c + (Y - cy) * s
        yr = -(X - cx) * s + (Y - cy) * c
        img += mu * ((xr / a) ** 2 + (yr / b) ** 2 <= 1.0)
    return img


def ellipse_sinogram(ell: np.ndarray, angles: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Closed-form line integrals of a sum of ellipses (textbook Radon transform of an ellipse).

    For an ellipse with semi-axes a, b rotated by phi and centred at c, the line
    x cos t + y sin t = s has chord 2ab*sqrt(r2 - (s - c.(cos t, sin t))^2)/r2 where
    r2 = a^2 cos^2(t - phi) + b^2 sin^2(t - phi) (zero when the root is imaginary).
    """
    sino = np.zeros((len(angles), len(s)))
    for ia, t in enumerate(angles):
        ct, st = math.cos(t), math.sin(t)
        for cx, cy, a, b, phi, mu in ell:
            r2 = (a * math.cos(t - phi)) ** 2 + (b * math.sin(t - phi)) ** 2
            ds = s - (cx * ct + cy * st)
            q = r2 - ds * ds
            sino[ia] += mu * np.where(q > 0, 2.0 * a * b * np.sqrt(np.maximum(q, 0.0)) / r2, 0.0)
    return sino


# --------------------------------------------------------------------------- 3D phantoms
def _rotation(a1: float, a2: float, a3: float) -> np.ndarray:
    """Rotation matrix Rz(a1) @ Ry(a2) @ Rz(a3)."""
    def rz(t):
        c, s = math.cos(t), math.sin(t)
        return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])

    def ry(t):
        c, s = math.cos(t), math.sin(t)
        return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])

    return rz(a1) @ ry(a2) @ rz(a3)


def random_ellipsoids(n: int, radius: float, rng: np.random.Generator) -> list:
    """List of (centre[3], semi_axes[3], rotation[3x3], intensity).

    Centres uniform in the ball of radius 0.5*R, semi-axes U[0.05, 0.35]*R, random Euler
    angles, intensity U[0, 1]. Every ellipsoid stays inside the ball of radius 0.85*R.
    """
    out = []
    for _ in range(n):
        while True:
            c = rng.uniform(-1.0, 1.0, 3)
            if c @ c <= 1.0:
                break
        c = 0.5 * radius * c
        ax = rng.uniform(0.05, 0.35, 3) * radius
        R = _rotation(rng.uniform(0, 2 * math.pi), rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi))
        out.append((c, ax, R, float(rng.uniform(0.0, 1.0))))
    return out


def rasterize_ellipsoids(ells: list, nx: int, ny: int, nz: int, voxel: float) -> np.ndarray:
    xs = (np.arange(nx) - (nx - 1) / 2.0) * voxel
    ys = (np.arange(ny) - (ny - 1) / 2.0) * voxel
    zs = (np.arange(nz) - (nz - 1) / 2.0) * voxel
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    vol = np.zeros((nz, ny, nx))
    for c, ax, R, mu in ells:
        P = np.stack([X - c[0], Y - c[1], Z - c[2]], axis=-1) @ R   # body-frame coordinates
        vol += mu * (((P / ax) ** 2).sum(-1) <= 1.0)
    return vol


def _cone_rays(spec: Cone3DSpec, view: int):
    b = spec.betas[view]
    cb, sb = math.cos(b), math.sin(b)
    S = np.array([spec.sod * cb, spec.sod * sb, 0.0])
    D0 = -(spec.sdd - spec.sod) * np.array([cb, sb, 0.0])
    eu = np.array([-sb, cb, 0.0])
    u = (np.arange(spec.nu) - (spec.nu - 1) / 2.0) * spec.du
    v = (np.arange(spec.nv) - (spec.nv - 1) / 2.0) * spec.dv
    P = D0[None, None, :] + u[None, :, None] * eu[None, None, :]
    P = P + np.zeros((spec.nv, 1, 1))
    P[..., 2] = v[:, None]
    return S, P - S[None, None, :]


def ellipsoid_cone_projections(ells: list, spec: Cone3DSpec) -> np.ndarray:
    """Closed-form line integrals of a sum of ellipsoids along every source-to-pixel segment.

    In the ellipsoid's scaled body frame the ray becomes p + t q and meets the unit sphere
    where |p + t q|^2 = 1; the chord is (t2 - t1)*|d| with t in units of the segment S->P.
    """
    out = np.zeros((len(spec.betas), spec.nv, spec.nu))
    for view in range(len(spec.betas)):
        S, d = _cone_rays(spec, view)
        dn = np.linalg.norm(d, axis=-1)
        for c, ax, R, mu in ells:
            p = ((S - c) @ R) / ax
            q = (d @ R) / ax
            qa = (q * q).sum(-1)
            qb = 2.0 * (q @ p)
            qc = p @ p - 1.0
            disc = qb * qb - 4.0 * qa * qc
            chord = np.where(disc > 0, np.sqrt(np.maximum(disc, 0.0)) / qa, 0.0)
            out[view] += mu * chord * dn
    return out


# --------------------------------------------------------------------------- noise
def gaussian_noise(clean: np.ndarray, rel_sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Additive Gaussian noise with sigma = rel_sigma * max(clean)."""
    sigma = rel_sigma * float(np.max(clean))
    return clean + sigma * rng.standard_normal(clean.shape)


def poisson_log_noise(clean: np.ndarray, photons: float, rng: np.random.Generator) -> np.ndarray:
    """Transmission data: counts ~ Poisson(I0 exp(-clean)), counts >= 1, b = -log(counts / I0)."""
    counts = rng.poisson(photons * np.exp(-clean)).astype(np.float64)
    counts = np.maximum(counts, 1.0)
    return -np.log(counts / photons)


# --------------------------------------------------------------------------- workloads
@dataclass
class Problem2D:
    spec: Par2DSpec
    b: np.ndarray               # float64 [n_angles][n_bins]
    truth: np.ndarray           # float64 [ny][nx]
    alpha: float
    meta: dict = field(default_factory=dict)


@dataclass
class Problem3D:
    spec: Cone3DSpec
    b: np.ndarray               # float64 [n_views][nv][nu]
    truth: np.ndarray | None    # float64 [nz][ny][nx] (None when not rasterised)
    alpha: float
    meta: dict = field(default_factory=dict)


# Paper-shaped 2D workloads: (side, angles, bins, subsets, noise)
WORKLOADS_2D = {
    # 64^2, 90 angles over [0,180), 96 unit bins, 10 subsets, Gaussian 1 %
    "par2d_64": dict(n=64, n_angles=90, n_bins=96, n_subsets=10, noise="gauss", alpha=0.01),
    # 512^2, 720 angles, 768 bins, 20 subsets, Poisson I0 = 1e4 with max clean line integral 4
    "par2d_512": dict(n=512, n_angles=720, n_bins=768, n_subsets=20, noise="poisson", alpha=1.0),
}

WORKLOADS_3D = {
    # 256^3 voxels of 0.5, 360 views over 360 deg, 384^2 detector of pixel 1, SOD 500, SDD 1000
    "cone3d_256": dict(n=256, voxel=0.5, n_views=360, det=384, d=1.0, sod=500.0, sdd=1000.0,
                       n_subsets=30, alpha=0.01),
}


def make_problem_2d(n: int, n_angles: int, n_bins: int, n_subsets: int, seed: int,
                    noise: str = "gauss", alpha: float = 0.01, pixel: float = 1.0,
                    bin_spacing: float = 1.0, n_ellipses: int = 10, truth: bool = True) -> Problem2D:
    """A seeded 2D parallel-beam problem: ellipse phantom, analytic sinogram, noise."""
    rng = np.random.default_rng(seed)
    spec = Par2DSpec(nx=n, ny=n, pixel=pixel, angles=uniform_angles(n_angles, math.pi),
                     n_bins=n_bins, bin_spacing=bin_spacing, n_subsets=n_subsets)
    ell = random_ellipses(n_ellipses, fov_radius=n * pixel / 2.0, rng=rng)
    clean = ellipse_sinogram(ell, spec.angles, spec.bin_centers())
    meta = {"seed": seed, "noise": noise}
    if noise == "gauss":
        b = gaussian_noise(clean, 0.01, rng)
        scale = 1.0
    elif noise == "poisson":
        scale = 4.0 / float(np.max(clean))      # max clean line integral = 4 (transmission >= e^-4)
        b = poisson_log_noise(clean * scale, 1.0e4, rng)
    elif noise == "none":
        b, scale = clean, 1.0
    else:
        raise ValueError(noise)
    ell = ell.copy()
    ell[:, 5] *= scale
    meta["intensity_scale"] = scale
    img = rasterize_ellipses(ell, n, n, pixel) if truth else None
    return Problem2D(spec=spec, b=b, truth=img, alpha=alpha, meta=meta)


def make_problem_3d(n: int, voxel: float, n_views: int, det: int, d: float, sod: float, sdd: float,
                    n_subsets: int, seed: int, alpha: float = 0.01, noise: str = "gauss",
                    n_ellipsoids: int = 10, truth: bool = False) -> Problem3D:
    """A seeded 3D circular cone-beam problem: ellipsoid phantom, analytic projections, noise."""
    rng = np.random.default_rng(seed)
    spec = Cone3DSpec(nx=n, ny=n, nz=n, voxel=voxel, betas=uniform_angles(n_views, 2.0 * math.pi),
                      nu=det, nv=det, du=d, dv=d, sod=sod, sdd=sdd, n_subsets=n_subsets)
    ells = random_ellipsoids(n_ellipsoids, radius=n * voxel / 2.0, rng=rng)
    clean = ellipsoid_cone_projections(ells, spec)
    if noise == "gauss":
        b = gaussian_noise(clean, 0.01, rng)
    elif noise == "none":
        b = clean
    else:
        raise ValueError(noise)
    vol = rasterize_ellipsoids(ells, n, n, n, voxel) if truth else None
    return Problem3D(spec=spec, b=b, truth=vol, alpha=alpha, meta={"seed": seed, "noise": noise})
