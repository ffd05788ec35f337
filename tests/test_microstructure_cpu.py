"""The seeded input generators against the recipes they implement.

The oracle and the CUDA path read the same arrays, so a generator bug would
not show up as a parity failure; these tests check each recipe directly.
"""
import math

import numpy as np
import pytest

from paper_2404_02433_b300 import microstructure as M


def test_random_spheres_follow_the_recipe():
    shape = (30, 36, 40)
    k, info = M.random_spheres(shape, (3.0, 6.0), 0.3, 17, 1.0, 10.0)
    k2, info2 = M.random_spheres(shape, (3.0, 6.0), 0.3, 17, 1.0, 10.0)
    assert np.array_equal(k, k2) and info["spheres"] == info2["spheres"]
    c, r = info["centres"], info["radii"]
    assert np.all((r >= 3.0) & (r <= 6.0))
    # non-overlapping: centres at least r1 + r2 apart
    d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    iu = np.triu_indices(len(r), 1)
    assert np.all(d[iu] >= (r[:, None] + r[None, :])[iu])
    # a voxel is an inclusion iff its centre lies in some sphere (brute force)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                          indexing="ij")
    inside = np.zeros(shape, dtype=bool)
    for (cx, cy, cz), rr in zip(c, r):
        inside |= (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= rr * rr
    assert np.array_equal(k == 10.0, inside)
    assert set(np.unique(k)) == {1.0, 10.0}
    # addition stops at the first sphere that reaches the fraction
    frac = inside.mean()
    assert frac == pytest.approx(info["fraction"], abs=0)
    assert 0.3 <= frac < 0.3 + (4.0 / 3.0) * math.pi * 6.0 ** 3 / inside.size


@pytest.mark.parametrize("ell", [4.0, 8.0])
def test_lognormal_field_statistics(ell):
    # lags of at least l/2: the lattice cuts the spectrum off at the Nyquist
    # frequency, which rounds the cusp of exp(-r/l) at r = 0 (lag-1 correlation
    # 0.85 against 0.78 at l = 4), as any voxel sampling of this covariance does
    sigma = 1.5
    rho = {lag: [] for lag in (int(ell // 2), int(ell), int(2 * ell))}
    for seed in (1, 2, 3):
        g = np.log(M.lognormal_field((64, 64, 64), ell, sigma, seed))
        assert abs(g.mean()) < 1e-12 and g.std() == pytest.approx(sigma, rel=1e-12)
        for lag in rho:
            rho[lag].append(np.mean([(g * np.roll(g, lag, axis=a)).mean() / g.var()
                                     for a in range(3)]))
    # sample correlation against the exponential covariance exp(-r / l)
    for lag, vals in rho.items():
        assert np.mean(vals) == pytest.approx(math.exp(-lag / ell), abs=0.05), lag


def test_random_ellipsoids_reach_their_fractions():
    kappas = (1.0, 20.0, 500.0)
    k, info = M.random_ellipsoids((32, 32, 32), (3.0, 6.0), (0.15, 0.15), kappas, 3002)
    assert set(np.unique(k)) <= set(kappas)
    for p, target in ((1, 0.15), (2, 0.15)):
        frac = float(np.mean(k == kappas[p]))
        assert frac == pytest.approx(info["fractions"][p - 1], abs=0)
        assert target <= frac < target + (4.0 / 3.0) * math.pi * 6.0 ** 3 / k.size
    k2, _ = M.random_ellipsoids((32, 32, 32), (3.0, 6.0), (0.15, 0.15), kappas, 3002)
    assert np.array_equal(k, k2)


def test_batch_members_draw_from_the_stated_ranges():
    sizes = set()
    for i in range(6):
        n, phi, contrast, kappa = M.batched_sphere_member(i)
        sizes.add(n)
        assert n in (64, 96, 128, 160, 192) and kappa.shape == (n, n, n)
        assert 0.1 <= phi <= 0.4 and 10.0 <= contrast <= 1000.0
        assert set(np.unique(kappa)) == {1.0, contrast}
        assert np.mean(kappa == contrast) >= phi
    assert len(sizes) > 1


def test_channel_lattice_cell_fraction():
    # three orthogonal channels of cross-section (1/4)^2 in a unit cell:
    # 3/16 of the cell minus twice the shared central cube (1/4)^3
    kx, ky, kz = M.channel_lattice(64, 4, 2)
    chan = kx == 4.0
    assert chan.mean() == pytest.approx(3.0 / 16.0 - 2.0 / 64.0, abs=1e-15)
    assert np.array_equal(chan, ky == 25.0) and np.array_equal(chan, kz == 100.0)
    assert np.all(kx[~chan] == 0.01) and np.all(ky[~chan] == 0.1) and np.all(kz[~chan] == 1.0)


def test_centre_ball_volume():
    k = M.centre_ball(96, 5.0)
    assert np.mean(k == 5.0) == pytest.approx(4.0 / 3.0 * math.pi / 64.0, rel=0.02)
    # symmetric under every axis reflection and permutation
    assert np.array_equal(k, k[::-1]) and np.array_equal(k, k.transpose(2, 1, 0))
