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


def lognormal_field(shape, correlation_length, sigma, seed):
    """kappa = exp(g), g a zero-mean Gaussian field with covariance
    sigma^2 exp(-r / l) (r, l in voxels), by spectral synthesis on the periodic
    box: white noise filtered by the square root of the exponential-covariance
    spectral density, proportional to l^3 / (1 + |k|^2 l^2)^2 in 3-D; the sample
    is then shifted and scaled to mean 0 and standard deviation sigma."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    kz = 2.0 * np.pi * np.fft.fftfreq(nz)[:, None, None]
    ky = 2.0 * np.pi * np.fft.fftfreq(ny)[None, :, None]
    kx = 2.0 * np.pi * np.fft.rfftfreq(nx)[None, None, :]
    l = float(correlation_length)
    amp = np.sqrt(l ** 3 / (1.0 + (kx ** 2 + ky ** 2 + kz ** 2) * l * l) ** 2)
    g = np.fft.irfftn(np.fft.rfftn(noise) * amp, s=shape, axes=(0, 1, 2))
    g -= g.mean()
    g *= sigma / g.std()
    return np.exp(g)


def random_ellipsoids(shape, semi_axes_range, fractions, kappas, seed, max_attempts=200_000):
    """Multi-phase medium of randomly oriented ellipsoids.

    Phase 0 (kappas[0]) is the matrix.  Ellipsoids of phases 1, 2, ... are
    added in turn (semi-axes uniform in ``semi_axes_range`` voxels, centres
    uniform over the box, orientation a uniformly random rotation) until each
    phase p reaches voxel fraction fractions[p-1]; a voxel keeps the first phase
    that covers it.  Returns (kappa, info) with the achieved fractions.
    """
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    label = np.zeros(shape, dtype=np.int8)
    total = nz * ny * nx
    filled = [0] * len(fractions)
    attempts = 0
    active = [p for p in range(len(fractions)) if fractions[p] > 0]
    while active and attempts < max_attempts:
        for p in list(active):
            attempts += 1
            ax = rng.uniform(semi_axes_range[0], semi_axes_range[1], 3)
            q, rmat = np.linalg.qr(rng.standard_normal((3, 3)))
            q = q * np.sign(np.diag(rmat))
            c = rng.uniform(0.0, 1.0, 3) * np.array([nx, ny, nz])
            r = ax.max()
            lo = np.maximum(np.floor(c - r).astype(int), 0)
            hi = np.minimum(np.ceil(c + r).astype(int) + 1, [nx, ny, nz])
            X = np.arange(lo[0], hi[0]) + 0.5 - c[0]
            Y = np.arange(lo[1], hi[1]) + 0.5 - c[1]
            Z = np.arange(lo[2], hi[2]) + 0.5 - c[2]
            pts = np.stack(np.meshgrid(Z, Y, X, indexing="ij")[::-1], axis=-1)  # (..., xyz)
            loc = pts @ q  # coordinates in the ellipsoid's frame
            inside = ((loc / ax) ** 2).sum(axis=-1) <= 1.0
            sub = label[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
            new = inside & (sub == 0)
            sub[new] = p + 1
            filled[p] += int(np.count_nonzero(new))
            if filled[p] >= fractions[p] * total:
                active.remove(p)
    kappa = np.asarray(kappas, dtype=np.float64)[label]
    info = {"fractions": [f / total for f in filled], "attempts": attempts}
    return kappa, info


def batched_sphere_member(i, seed0=4001):
    """Member i of the seeded batch of uneven RVEs: N from {64, 96, 128, 160,
    192}, spheres with radius U[N/32, N/12] at fraction U[0.1, 0.4], inclusion
    contrast log-uniform in [10, 1000].  Returns (N, fraction, contrast, kappa)."""
    rng = np.random.default_rng(seed0 + i)
    n = int(rng.choice([64, 96, 128, 160, 192]))
    phi = rng.uniform(0.1, 0.4)
    contrast = float(np.exp(rng.uniform(np.log(10.0), np.log(1000.0))))
    mask, _ = random_spheres((n, n, n), (n / 32, n / 12), phi, seed0 + i, 0.0, 1.0)
    return n, phi, contrast, 1.0 + (contrast - 1.0) * mask


def smooth_problem(n):
    """Data of the smooth test of Sec. 4.1 (Table 2) on an n^3 grid of the unit cube.

    K = diag(cos(pi y) + 2, 2 e^z, 3 cos(pi x) + 4) and exact solution
    p = cos(pi x) cos(pi y) e^z, so the source is f = -div(K grad p) =
    cos(pi x) cos(pi y) [(cos(pi y) + 2) pi^2 e^z + 2 pi^2 e^{2z} - (3 cos(pi x) + 4) e^z]
    (homogeneous Neumann data hold on the x and y faces).  Returns
    (kx, ky, kz, p_in face values on z = 0, p_out face values on z = 1,
    source at the voxel centres, exact p at the voxel centres).
    """
    c = voxel_centres(n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    cx, cy = np.cos(np.pi * x), np.cos(np.pi * y)
    kx = cy + 2.0
    ky = 2.0 * np.exp(z)
    kz = 3.0 * cx + 4.0
    exact = cx * cy * np.exp(z)
    src = cx * cy * ((cy + 2.0) * np.pi ** 2 * np.exp(z) + 2.0 * np.pi ** 2 * np.exp(2.0 * z)
                     - (3.0 * cx + 4.0) * np.exp(z))
    fy, fx = np.meshgrid(c, c, indexing="ij")
    face = np.cos(np.pi * fx) * np.cos(np.pi * fy)
    return kx, ky, kz, face, np.e * face, src, exact


def channel_lattice(n, cells, psi):
    """Anisotropic channel lattice of Sec. 4.4: the periodic cell has three
    orthogonal channels (cross-section (3/8, 5/8)^2) with K = diag(2^psi, 5^psi,
    10^psi), elsewhere diag(0.01, 0.1, 1); the RVE repeats the cell `cells` times
    per axis.  Returns (kx, ky, kz)."""
    c = np.modf(voxel_centres(n) * cells)[0]
    inside = (c > 3.0 / 8.0) & (c < 5.0 / 8.0)
    iz, iy, ix = np.meshgrid(inside, inside, inside, indexing="ij")
    chan = (iy & iz) | (ix & iz) | (ix & iy)
    kx = np.where(chan, 2.0 ** psi, 0.01)
    ky = np.where(chan, 5.0 ** psi, 0.1)
    kz = np.where(chan, 10.0 ** psi, 1.0)
    return kx, ky, kz
