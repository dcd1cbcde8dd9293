"""Seeded synthetic inputs: ellipse phantoms and low-dose sinogram noise.

This module holds none of the reconstruction method's arithmetic (no system
matrix, no projection, no QR).  It draws the images and the noise that both
the CUDA path and the CPU oracle consume, so that both see identical inputs.

The inputs stand in for the paper's CT slices (COVID-CT-MD, DICOM-CT-PD,
Sec. 3.1 and 3.2), which are not available: attenuation-like values in
[0, 1] with zero-valued air around the object, many slices per geometry, and
Poisson counting noise for the low-dose case (Sec. 3.2 simulates low dose by
adding Poisson noise to the projections).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1234


def ellipse_phantom(n_side: int, n_ellipses: int, seed: int) -> np.ndarray:
    """One n_side x n_side phantom, returned flattened with pixel index
    j = iy*n_side + ix (iy grows with +y).

    Ellipses are painted in order (a later ellipse overwrites an earlier one):
    centre ~ U(-0.6, 0.6)^2, semi-axes ~ U(0.05, 0.4), rotation ~ U(0, pi),
    value ~ U(0, 1), in normalised coordinates [-1, 1]^2 sampled at pixel
    centres; pixels outside the unit disk are 0 (air)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cx = rng.uniform(-0.6, 0.6, n_ellipses)
    cy = rng.uniform(-0.6, 0.6, n_ellipses)
    ax = rng.uniform(0.05, 0.4, n_ellipses)
    ay = rng.uniform(0.05, 0.4, n_ellipses)
    rot = rng.uniform(0.0, np.pi, n_ellipses)
    val = rng.uniform(0.0, 1.0, n_ellipses)
    centres = (np.arange(n_side, dtype=np.float64) + 0.5) * (2.0 / n_side) - 1.0
    X, Y = np.meshgrid(centres, centres, indexing="xy")  # Y[iy, ix], X[iy, ix]
    img = np.zeros((n_side, n_side), np.float64)
    for e in range(n_ellipses):
        c, s = np.cos(rot[e]), np.sin(rot[e])
        u = (X - cx[e]) * c + (Y - cy[e]) * s
        v = -(X - cx[e]) * s + (Y - cy[e]) * c
        inside = (u / ax[e]) ** 2 + (v / ay[e]) ** 2 <= 1.0
        img[inside] = val[e]
    img[X * X + Y * Y > 1.0] = 0.0
    return img.reshape(-1)


def phantom_batch(n_side: int, k: int, n_ellipses: int, first_seed: int = BASE_SEED) -> np.ndarray:
    """k phantoms as the columns of an (n_side^2 x k) Fortran-ordered array;
    slice s uses seed first_seed + s."""
    out = np.empty((n_side * n_side, k), np.float64, order="F")
    for s in range(k):
        out[:, s] = ellipse_phantom(n_side, n_ellipses, first_seed + s)
    return out


def poisson_sinogram(p: np.ndarray, n_side: int, i0: float, seed: int) -> np.ndarray:
    """Low-dose measurement model for noiseless line integrals p (pixel units).

    Physical line integral p*w with w = 2/n_side (the image spans 2 units);
    counts N ~ Poisson(i0 * exp(-p*w)), clamped to >= 1; measured line
    integral -ln(N/i0)/w, returned in pixel units like p."""
    w = 2.0 / n_side
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = i0 * np.exp(-np.asarray(p, np.float64) * w)
    counts = np.maximum(rng.poisson(lam), 1).astype(np.float64)
    out = -np.log(counts / i0) / w
    return np.asfortranarray(out)
