"""Seeded synthetic voxel microstructures (host numpy, float64).

This module holds only input generation -- geometry and random numbers -- and
none of the solver's arithmetic.  Both the CUDA path and the CPU test oracle
consume the arrays it returns.

All arrays have shape (Nz, Ny, Nx), C order, x fastest; the unit cube is
discretised into voxels and a voxel belongs to an inclusion iff its centre lies
inside it (the rule the paper states for its centre-ball experiment, Sec. 4.1).
"""
from __future__ import annotations

import numpy as np


def voxel_centres(n):
    """Voxel-centre coordinates (k + 1/2) / n along one axis of the unit cube."""
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def centre_ball(n, kappa_inc, kappa_matrix=1.0, radius=0.25):
    """Ball of radius 1/4 at the cube centre (Sec. 4.1, Table 3 geometry)."""
    c = voxel_centres(n) - 0.5
    r2 = c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2
    return np.where(r2 <= radius * radius, float(kappa_inc), float(kappa_matrix))


def random_spheres(shape, radius_range, volume_fraction, seed, kappa_matrix=1.0,
                   kappa_inclusion=10.0, max_attempts=1_000_000):
    """Random non-overlapping spheres by random sequential addition.

    Radii (in voxels) are uniform in ``radius_range``; centres are uniform over
    the box (spheres may be cut by the boundary); a candidate is accepted if its
    centre is at least r1 + r2 from every accepted centre.  Addition stops once
    the voxel fraction inside spheres reaches ``volume_fraction`` or after
    ``max_attempts`` candidates.  Returns (kappa, info) with the achieved
    fraction and the sphere list in ``info``.
    """
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    phase = np.zeros(shape, dtype=bool)
    total = nz * ny * nx
    centres = np.empty((0, 3))
    radii = np.empty(0)
    filled = 0
    attempts = 0
    batch = 256
    while filled < volume_fraction * total and attempts < max_attempts:
        cand_r = rng.uniform(radius_range[0], radius_range[1], batch)
        cand_c = rng.uniform(0.0, 1.0, (batch, 3)) * np.array([nx, ny, nz])
        for c, r in zip(cand_c, cand_r):
            attempts += 1
            if radii.size:
                d2 = ((centres - c) ** 2).sum(axis=1)
                if np.any(d2 < (radii + r) ** 2):
                    continue
            centres = np.vstack([centres, c])
            radii = np.append(radii, r)
            lo = np.maximum(np.floor(c - r).astype(int), 0)
            hi = np.minimum(np.ceil(c + r).astype(int) + 1, [nx, ny, nz])
            xs = np.arange(lo[0], hi[0]) + 0.5 - c[0]
            ys = np.arange(lo[1], hi[1]) + 0.5 - c[1]
            zs = np.arange(lo[2], hi[2]) + 0.5 - c[2]
            inside = (zs[:, None, None] ** 2 + ys[None, :, None] ** 2
                      + xs[None, None, :] ** 2) <= r * r
            sub = phase[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
            filled += int(np.count_nonzero(inside & ~sub))
            sub |= inside
            if filled >= volume_fraction * total or attempts >= max_attempts:
                break
    kappa = np.where(phase, float(kappa_inclusion), float(kappa_matrix))
    info = {"fraction": filled / total, "spheres": len(radii), "attempts": attempts,
            "centres": centres, "radii": radii}
    return kappa, info


def series_laminate(shape, values, axis):
    """Layers normal to ``axis`` (0=x, 1=y, 2=z); layer l takes values[l % len]."""
    nz, ny, nx = shape
    n = (nx, ny, nz)[axis]
    prof = np.asarray([values[l % len(values)] for l in range(n)], dtype=np.float64)
    view = [1, 1, 1]
    view[2 - axis] = n
    return np.broadcast_to(prof.reshape(view), shape).copy()


def random_field(shape, seed, lo=0.5, hi=2.0):
    """Independent uniform voxel values in [lo, hi) (unit tests only)."""
    return np.random.default_rng(seed).uniform(lo, hi, shape)


def two_phase_random(shape, seed, fraction=0.3, kappa_matrix=1.0, kappa_inclusion=10.0):
    """Independent Bernoulli voxels (a cheap two-phase medium for tests)."""
    mask = np.random.default_rng(seed).random(shape) < fraction
    return np.where(mask, float(kappa_inclusion), float(kappa_matrix))
