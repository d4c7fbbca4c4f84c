"""Seeded synthetic permittivity fields, evaluated per finest cell at the
cell centroid (inputs only).

The paper's target (an irregular body with a surface layer and voids,
Sec. III) exists only as a figure, so these seeded fields stand in for it:
a background value, a thin surface layer, random elliptical voids and
inclusions, and, in 2D, smoothed multiplicative noise.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import ndimage

from .meshes import ELLIPSOID_AXES, NestedMesh, asteroid_radius, centroids


def rng_for(config: int, instance: int = 0) -> np.random.Generator:
    """numpy PCG64 stream with seed 1000*config + instance."""
    return np.random.Generator(np.random.PCG64(1000 * config + instance))


def square_disc_eps(mesh: NestedMesh, background=4.0, inner=6.0,
                    centre=(0.2, -0.1), radius=0.3) -> np.ndarray:
    """eps = background with one disc of value ``inner``."""
    c = centroids(mesh)
    r = np.hypot(c[:, 0] - centre[0], c[:, 1] - centre[1])
    eps = np.full(c.shape[0], background)
    eps[r < radius] = inner
    return eps


def _random_rotation_2d(rng):
    a = rng.uniform(0.0, 2.0 * math.pi)
    return np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])


def _random_rotation_3d(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def smoothed_noise_2d(points: np.ndarray, rng, sigma=0.05, spacing=0.01,
                      extent=1.4) -> np.ndarray:
    """i.i.d. N(0,1) on a regular grid of the given spacing over
    [-extent, extent]^2, Gaussian-smoothed (std ``sigma``, truncated at
    3 sigma), sampled at ``points`` by bilinear interpolation and scaled so
    that max |.| over the points is 1."""
    n = int(round(2 * extent / spacing)) + 1
    g = rng.standard_normal((n, n))
    g = ndimage.gaussian_filter(g, sigma=sigma / spacing, truncate=3.0,
                                mode="constant")
    u = (points[:, 0] + extent) / spacing
    v = (points[:, 1] + extent) / spacing
    vals = ndimage.map_coordinates(g, np.stack([u, v]), order=1, mode="nearest")
    return vals / np.abs(vals).max()


def asteroid_eps(mesh: NestedMesh, seed_config: int, instance: int = 0,
                 rotation: float = 0.0, scale: float = 1.0, n_ellipses=6,
                 layer=0.05, noise=0.05) -> np.ndarray:
    """2D asteroid permittivity: eps=4 background, ``n_ellipses`` random
    ellipses (centre uniform by area in rho<0.7, semi-axes U[0.05,0.2],
    uniform rotation, eps in {1,8} with p=1/2, later ones overwrite earlier
    ones), then a surface layer eps=3 where r(theta)-|x| < ``layer``, then
    eps <- eps (1 + noise * n) with n the smoothed noise field."""
    rng = rng_for(seed_config, instance)
    c = centroids(mesh)
    # body frame: undo the instance rotation and scale
    ca, sa = math.cos(-rotation), math.sin(-rotation)
    b = np.stack([ca * c[:, 0] - sa * c[:, 1], sa * c[:, 0] + ca * c[:, 1]], 1) / scale
    th = np.arctan2(b[:, 1], b[:, 0])
    R = asteroid_radius(th)
    rad = np.hypot(b[:, 0], b[:, 1])
    eps = np.full(c.shape[0], 4.0)
    for _ in range(n_ellipses):
        rho = 0.7 * math.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * math.pi)
        ctr = rho * float(asteroid_radius(phi)) * np.array([math.cos(phi), math.sin(phi)])
        ax = rng.uniform(0.05, 0.2, size=2)
        Q = _random_rotation_2d(rng)
        val = 1.0 if rng.uniform() < 0.5 else 8.0
        loc = (b - ctr[None, :]) @ Q
        inside = (loc[:, 0] / ax[0]) ** 2 + (loc[:, 1] / ax[1]) ** 2 < 1.0
        eps[inside] = val
    eps[(R - rad) < layer] = 3.0
    if noise:
        eps = eps * (1.0 + noise * smoothed_noise_2d(b, rng))
    return eps


def ellipsoid_eps(mesh: NestedMesh, seed_config: int, instance: int = 0,
                  n_bodies=10, layer=0.05, axes=ELLIPSOID_AXES) -> np.ndarray:
    """3D permittivity: eps=4 background, ``n_bodies`` random ellipsoidal
    voids/inclusions (centre uniform by volume in ellipsoidal radius < 0.7,
    semi-axes U[0.05,0.2], uniform rotation, eps in {1,8}), then a surface
    layer eps=3 where the radial depth (1-rho)|x|/rho < ``layer``."""
    rng = rng_for(seed_config, instance)
    c = centroids(mesh)
    A = np.asarray(axes)
    eps = np.full(c.shape[0], 4.0)
    for _ in range(n_bodies):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        ctr = 0.7 * rng.uniform() ** (1.0 / 3.0) * d * A
        ax = rng.uniform(0.05, 0.2, size=3)
        Q = _random_rotation_3d(rng)
        val = 1.0 if rng.uniform() < 0.5 else 8.0
        loc = (c - ctr[None, :]) @ Q
        inside = ((loc / ax[None, :]) ** 2).sum(1) < 1.0
        eps[inside] = val
    rho = np.sqrt(((c / A[None, :]) ** 2).sum(1))
    rad = np.linalg.norm(c, axis=1)
    depth = np.where(rho > 0, (1.0 - rho) * rad / np.where(rho > 0, rho, 1.0), 1.0)
    eps[depth < layer] = 3.0
    return eps
