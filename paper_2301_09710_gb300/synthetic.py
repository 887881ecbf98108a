"""Seeded synthetic inputs shaped like the paper's SPECT workloads.

This module is shared by the CUDA path's tests/benchmark and by the oracle's
tests.  It holds none of the projector's or EM's arithmetic: it only draws
phantoms, attenuation maps, PSF stacks and noise.  The XCAT and virtual
patient phantoms of the paper (Section II-C) are not available; ellipsoid
phantoms with the same sizes and value ranges stand in for them.

All arrays are numpy float32 in the library's layouts:
  x, mu : (nz, ny, nx)            x(i,j,k) = x[k, j, i]
  psf   : (nview_psf, ny, pz, px) p(a,b,j,l) = psf[l, j, b, a]
  fx    : (nview_psf, ny, px), fz : (nview_psf, ny, pz)  separable factors
  v, y  : (nview, nz, nx)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FWHM_TO_SIGMA = 1.0 / (2.0 * np.sqrt(2.0 * np.log(2.0)))


def _grid(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i.astype(np.float64), j.astype(np.float64), k.astype(np.float64)


def ellipsoid_mask(shape, centre, semi, phi=0.0):
    """Voxel-centre inclusion test for an ellipsoid turned by phi about z."""
    nz, ny, nx = shape
    i, j, k = _grid(nx, ny, nz)
    di, dj, dk = i - centre[0], j - centre[1], k - centre[2]
    c, s = np.cos(phi), np.sin(phi)
    u = c * di + s * dj
    w = -s * di + c * dj
    return (u / semi[0]) ** 2 + (w / semi[1]) ** 2 + (dk / semi[2]) ** 2 <= 1.0


def _random_centre(rng, n, nz, rmax_frac, semi_xy):
    """Centre whose in-plane extent stays inside radius rmax_frac * n of the axis."""
    c = 0.5 * (n - 1)
    rlim = max(rmax_frac * n - semi_xy, 0.0)
    r = rlim * np.sqrt(rng.uniform())
    a = rng.uniform(0, 2 * np.pi)
    return (c + r * np.cos(a), c + r * np.sin(a), rng.uniform(0.25, 0.75) * (nz - 1))


def gaussian_factor(size: int, fwhm: float) -> np.ndarray:
    """Odd-length sampled Gaussian, truncated and normalised to unit sum."""
    assert size % 2 == 1
    c = (size - 1) // 2
    sig = fwhm * FWHM_TO_SIGMA
    t = np.arange(size) - c
    g = np.exp(-0.5 * (t / sig) ** 2)
    return g / g.sum()


@dataclass
class Problem:
    """One synthetic projection problem (all float32 numpy)."""
    x: np.ndarray
    mu: np.ndarray
    dy: float
    fx: np.ndarray
    fz: np.ndarray
    nview: int
    psf: np.ndarray | None = None        # full stack, built from fx/fz on request
    body: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.x.shape

    def full_psf(self) -> np.ndarray:
        """Full PSF stack p = fx (x) fz, rounded to float32 (an input in its own right)."""
        if self.psf is None:
            self.psf = (self.fz[..., :, None].astype(np.float64) *
                        self.fx[..., None, :].astype(np.float64)).astype(np.float32)
        return self.psf


def depth_psf_factors(ny: int, px: int, pz: int, fwhm_x_near: float, fwhm_x_far: float,
                      aniso: bool, nview_psf: int = 1, orbit_gap=None):
    """Depth-dependent Gaussian PSF factors.

    FWHM grows linearly with distance from the detector (plane ny-1 nearest).
    With ``aniso`` the z-FWHM is 0.8 * FWHM_x + 0.3 clamped to [near, far].
    ``orbit_gap`` (nview_psf values, in voxels) adds a per-view distance,
    standing in for a non-circular orbit.
    """
    fx = np.empty((nview_psf, ny, px), np.float32)
    fz = np.empty((nview_psf, ny, pz), np.float32)
    for l in range(nview_psf):
        gap = 0.0 if orbit_gap is None else float(orbit_gap[l])
        for j in range(ny):
            dist = (ny - 1 - j + gap) / max(ny - 1 + (0.0 if orbit_gap is None else max(orbit_gap)), 1)
            fwx = fwhm_x_near + (fwhm_x_far - fwhm_x_near) * dist
            fwz = np.clip(0.8 * fwx + 0.3, fwhm_x_near, fwhm_x_far) if aniso else fwx
            fx[l, j] = gaussian_factor(px, fwx)
            fz[l, j] = gaussian_factor(pz, fwz)
    return fx, fz


def small_phantom(nx: int, nz: int, seed: int, n_blobs: int = 6):
    """Config-1 style activity and mu: ellipsoids on a zero background, mu per voxel."""
    rng = np.random.default_rng(seed)
    shape = (nz, nx, nx)
    x = np.zeros(shape, np.float64)
    for _ in range(n_blobs):
        semi = rng.uniform(0.06, 0.2, size=3) * np.array([nx, nx, nz])
        cen = _random_centre(rng, nx, nz, 0.45, max(semi[0], semi[1]))
        x += rng.uniform(0.5, 5.0) * ellipsoid_mask(shape, cen, semi, rng.uniform(0, np.pi))
    c = 0.5 * (nx - 1)
    body = ellipsoid_mask(shape, (c, c, 0.5 * (nz - 1)), (0.42 * nx, 0.32 * nx, 0.45 * nz + 0.5))
    mu = 0.012 * body
    bone_c = (c + 0.15 * nx, c - 0.05 * nx, 0.5 * (nz - 1))
    mu = np.where(ellipsoid_mask(shape, bone_c, (0.08 * nx, 0.08 * nx, 0.3 * nz)), 0.025, mu)
    return x.astype(np.float32), mu.astype(np.float32), body


def config1(seed: int = 0, nx: int = 64, nz: int = 32, nview: int = 64, psf_size: int = 11) -> Problem:
    """64x64x32, 64 views, 11x11 isotropic depth-dependent Gaussian PSF (FWHM 1 -> 4)."""
    x, mu, body = small_phantom(nx, nz, seed)
    fx, fz = depth_psf_factors(nx, psf_size, psf_size, 1.0, 4.0, aniso=False)
    return Problem(x=x, mu=mu, dy=1.0, fx=fx, fz=fz, nview=nview, body=body,
                   meta={"workload": f"{nx}x{nx}x{nz}, {nview} views, {psf_size}x{psf_size} PSF"})


def xcat_like_phantom(nx: int, nz: int, seed: int, n_organs: int = 20, n_lesions: int = 3):
    """Config-2 style: body at activity 1, organs U[0.3,3], 3 hot spherical lesions (4-8x)."""
    rng = np.random.default_rng(seed)
    shape = (nz, nx, nx)
    c = 0.5 * (nx - 1)
    body = ellipsoid_mask(shape, (c, c, 0.5 * (nz - 1)), (0.42 * nx, 0.30 * nx, 0.55 * nz))
    x = body.astype(np.float64)
    for _ in range(n_organs):
        semi = rng.uniform(0.05, 0.16, size=3) * np.array([nx, nx, nz])
        cen = _random_centre(rng, nx, nz, 0.40, max(semi[0], semi[1]))
        m = ellipsoid_mask(shape, cen, semi, rng.uniform(0, np.pi)) & body
        x[m] = rng.uniform(0.3, 3.0)
    for _ in range(n_lesions):
        r = rng.uniform(2.2, 6.0)
        cen = _random_centre(rng, nx, nz, 0.35, r)
        m = ellipsoid_mask(shape, cen, (r, r, r)) & body
        x[m] = rng.uniform(4.0, 8.0)
    mu = 0.0150 * body
    for side in (-1, 1):  # lung-like regions
        m = ellipsoid_mask(shape, (c + side * 0.2 * nx, c - 0.02 * nx, 0.7 * (nz - 1)),
                           (0.12 * nx, 0.14 * nx, 0.25 * nz))
        mu = np.where(m & body, 0.005, mu)
    spine = ellipsoid_mask(shape, (c, c + 0.2 * nx, 0.5 * (nz - 1)), (0.05 * nx, 0.05 * nx, 0.6 * nz))
    mu = np.where(spine & body, 0.030, mu)
    return x.astype(np.float32), mu.astype(np.float32), body


def config2(seed: int = 0, nx: int = 128, nz: int = 80, nview: int = 128, psf_size: int = 37,
            per_view_orbit: bool = False) -> Problem:
    """128x128x80, 128 views, 37x37 anisotropic depth-dependent Gaussians (FWHM 1.5 -> 9).

    mu in mm^-1 with voxel size dy = 4.8 mm (the paper's 4.8 mm voxels).  With
    ``per_view_orbit`` every view gets its own PSF stack (gap 4 + 6|sin theta|).
    """
    x, mu, body = xcat_like_phantom(nx, nz, seed)
    nvp = 1
    gap = None
    if per_view_orbit:
        nvp = nview
        th = 2 * np.pi * np.arange(nview) / nview
        gap = 4.0 + 6.0 * np.abs(np.sin(th))
    fx, fz = depth_psf_factors(nx, psf_size, psf_size, 1.5, 9.0, aniso=True, nview_psf=nvp, orbit_gap=gap)
    return Problem(x=x, mu=mu, dy=4.8, fx=fx, fz=fz, nview=nview, body=body,
                   meta={"workload": f"{nx}x{nx}x{nz}, {nview} views, {psf_size}x{psf_size} PSF"})


def random_problem(seed: int, nx: int, nz: int, nview: int, px: int, pz: int,
                   nview_psf: int = 1, symmetric: bool = False, mu_scale: float = 0.05) -> Problem:
    """Unstructured random inputs (non-negative x, mu, PSF) for operator tests.

    With ``symmetric`` the full PSF is symmetric in a and in b (the paper's
    adjoint-test setting); otherwise it is a generic non-separable array.
    Separable factors are also drawn, for the separable path.
    """
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (nz, nx, nx)).astype(np.float32)
    mu = (mu_scale * rng.uniform(0, 1, (nz, nx, nx))).astype(np.float32)
    p = rng.uniform(0, 1, (nview_psf, nx, pz, px))
    if symmetric:
        p = p + p[..., ::-1, :]
        p = p + p[..., :, ::-1]
    p = p / p.sum(axis=(2, 3), keepdims=True)
    fx = rng.uniform(0, 1, (nview_psf, nx, px))
    fz = rng.uniform(0, 1, (nview_psf, nx, pz))
    fx /= fx.sum(-1, keepdims=True)
    fz /= fz.sum(-1, keepdims=True)
    return Problem(x=x, mu=mu, dy=1.0, fx=fx.astype(np.float32), fz=fz.astype(np.float32), nview=nview,
                   psf=p.astype(np.float32), meta={"workload": "random"})


def blur_views(v: np.ndarray, sigma: float) -> np.ndarray:
    """Per-view 2D Gaussian blur (reflect edges) of projections (nview, nz, nx).

    Used only to shape a smooth background r = scatter-like copy of the
    projections; it is not part of the projector.
    """
    from scipy.ndimage import gaussian_filter
    return np.stack([gaussian_filter(np.asarray(p, np.float64), sigma, mode="reflect") for p in v])


def poisson_counts(mean: np.ndarray, seed: int) -> np.ndarray:
    """y ~ Poisson(mean), as float32."""
    rng = np.random.default_rng(seed + 1000)
    return rng.poisson(np.clip(np.asarray(mean, np.float64), 0, None)).astype(np.float32)


def background_from(primary: np.ndarray, fraction: float = 0.1, sigma: float = 8.0) -> np.ndarray:
    """Smoothed background with total = fraction * total(primary)."""
    g = blur_views(primary, sigma)
    return (fraction * primary.sum() / max(g.sum(), 1e-30) * g).astype(np.float32)
