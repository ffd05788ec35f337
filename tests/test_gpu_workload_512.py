"""The benchmark workload at full size, through the C ABI, by properties.

512^3 random spheres (radius 8-20 voxels, fraction 0.25, seed 2001), inclusions
1000 times the matrix, load along z, rtol 1e-8, FP64 and mixed precision --
one of the six solves bench.py times, in the same launch configuration.  The
oracle cannot solve this size in a test, so the GPU solution is checked where
the oracle can compute one value at a time, and by properties that hold at
any size:
* the TPFA balance (Sec. 2.2) evaluated cell by cell from the oracle's face
  formula at 4096 sampled cells, interior and on both Dirichlet planes: its
  RMS, scaled to the whole grid, is a residual estimate independent of the
  library's own;
* the discrete maximum principle (A is an M-matrix, b >= 0): p_out <= p <= p_in;
* inflow = outflow (conservation, to the solve's accuracy);
* Reuss <= kappa_eff <= Voigt;
* the mixed path within 3e-6 of FP64.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etc_oracle as O
from paper_2404_02433_b300 import binding as B
from paper_2404_02433_b300 import microstructure as M

pytestmark = pytest.mark.gpu

N = 512
CONTRAST = 1000.0


def sampled_balance(kap, p, cells, p_in, p_out):
    """TPFA residual (A p - b)_c at the given cells, in kappa~ units."""
    n = kap.shape[0]
    ks = O.scaled_conductivity(kap, 1.0 / n)  # unit cube: h = 1/n on every axis
    out = np.empty(len(cells))
    for m, (k, j, i) in enumerate(cells):
        r = 0.0
        for dk, dj, di in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            kk, jj, ii = k + dk, j + dj, i + di
            if 0 <= kk < n and 0 <= jj < n and 0 <= ii < n:
                r += O.harmonic_face(ks[k, j, i], ks[kk, jj, ii]) * (p[k, j, i] - p[kk, jj, ii])
        if k == 0:
            r += 2.0 * ks[k, j, i] * (p[k, j, i] - p_in)
        if k == n - 1:
            r += 2.0 * ks[k, j, i] * (p[k, j, i] - p_out)
        out[m] = r
    return out


def test_benchmark_rve_512_load_z_by_properties():
    mask, info = M.random_spheres((N, N, N), (8.0, 20.0), 0.25, 2001, 0.0, 1.0)
    kap = 1.0 + (CONTRAST - 1.0) * mask
    rve = B.RVE(torch.from_numpy(kap).cuda())
    try:
        k64, inf64 = rve.solve(2, rtol=1e-8)
        p = rve.solution(2).cpu().numpy()
        kmx, infmx = rve.solve(2, rtol=1e-8, precision=B.ETC_PREC_MIXED)
    finally:
        rve.close()
    assert inf64["status"] == B.ETC_OK and infmx["status"] == B.ETC_OK
    assert inf64["relres"] <= 1e-8 and 0 <= inf64["true_relres"] < 2e-8
    # residual at sampled cells, scaled to an estimate of ||b - A p|| / ||b||
    rng = np.random.default_rng(7)
    interior = [tuple(v) for v in rng.integers(0, N, (3072, 3))]
    planes = [(k, int(j), int(i)) for k in (0, N - 1)
              for j, i in rng.integers(0, N, (512, 2))]
    ks0 = O.scaled_conductivity(kap[0], 1.0 / N)
    bnorm = float(np.linalg.norm(2.0 * ks0 * 1.0))  # b on plane 0 (p_in = 1, p_out = 0)
    for cells in (interior, planes):
        r = sampled_balance(kap, p, cells, 1.0, 0.0)
        est = math.sqrt(float(np.mean(r * r)) * kap.size) / bnorm
        assert est < 1e-6, est
    # maximum principle, conservation, bounds, mixed against FP64
    assert p.min() >= -1e-6 and p.max() <= 1.0 + 1e-6
    assert abs(inf64["kappa_in"] - k64) <= 1e-4 * k64
    reuss = 1.0 / float(np.mean(1.0 / kap))
    voigt = float(np.mean(kap))
    assert reuss <= k64 <= voigt
    assert abs(kmx - k64) <= 3e-6 * k64
