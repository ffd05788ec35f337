"""The face conductance of the TPFA scheme against its correctly rounded value.

Sec. 2.2 gives an internal face between cells of conductivities a and b the
harmonic mean 2 / (1/a + 1/b) = 2ab / (a + b).  The face assembly forms
2ab * (1/(a+b)) with the reciprocal taken from the FP32 hardware approximation
and refined by two Newton-Raphson steps in FP64; sums outside the binary32
normal range (1e-30 .. 1e30) divide instead.  A medium of two columns of cells
with h = 1 makes the operator return that face exactly: with w = 1 on the
first column and 0 on the second, (A w) on the second column is -T, with no
other term (every other neighbour difference is 0).  The exact value
2ab/(a+b) is formed in rational arithmetic and rounded once.
"""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2404_02433_b300 import binding as B

pytestmark = pytest.mark.gpu


def exact_harmonic(a, b):
    """2ab/(a+b), correctly rounded to binary64 (exact rationals, one rounding)."""
    return np.array([float(Fraction(2) * Fraction(x) * Fraction(y) / (Fraction(x) + Fraction(y)))
                     for x, y in zip(a.tolist(), b.tolist())])


def faces_on_gpu(a, b):
    """-(A w) on the second column of a medium whose rows hold the pairs (a, b).

    The pairs fill a (nz, ny) grid of rows (an axis holds at most 8192
    voxels); rows are coupled along y and z by faces of value 1, which carry
    no flux because w is the same in every row.
    """
    m = a.size
    ny = min(m, 400)
    nz = m // ny
    assert ny * nz == m
    kx = np.empty((nz, ny, 2))
    kx[:, :, 0], kx[:, :, 1] = a.reshape(nz, ny), b.reshape(nz, ny)
    ones = np.ones_like(kx)
    dev = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    # lengths equal to the voxel counts: h = 1 on every axis, kappa~ = kappa
    rve = B.RVE(dev(kx), dev(ones), dev(ones), lengths=(2.0, float(ny), float(nz)))
    w = np.zeros((nz, ny, 2))
    w[:, :, 0] = 1.0
    q = torch.empty((nz, ny, 2), dtype=torch.float64, device="cuda")
    B.etc_apply_operator(rve.h, 2, dev(w), q)
    out = -q.cpu().numpy()[:, :, 1].ravel()
    rve.close()
    return out


def test_harmonic_face_within_two_units_of_correct_rounding():
    rng = np.random.default_rng(2404)
    m = 60000
    # contrasts up to 1e8 around 1, and a lognormal spread (log-sd 6, about
    # 1e-10 .. 1e10) wider than that of the sigma = 1.5 benchmark field
    a = np.concatenate([10.0 ** rng.uniform(-4, 4, m), np.exp(6.0 * rng.standard_normal(m))])
    b = np.concatenate([10.0 ** rng.uniform(-4, 4, m), np.exp(6.0 * rng.standard_normal(m))])
    # equal values (T = a exactly) and powers of two
    a[:64] = b[:64] = 2.0 ** np.arange(-32, 32)
    got = faces_on_gpu(a, b)
    ref = exact_harmonic(a, b)
    rel = np.abs(got - ref) / ref
    assert rel.max() <= 2.0 ** -51, (rel.max() / 2.0 ** -53, a[rel.argmax()], b[rel.argmax()])
    assert np.array_equal(got[:64], a[:64])


def test_harmonic_face_both_sides_of_the_guard():
    # a + b below 1e-30 or above 1e30 (binary32 reciprocal out of range): the
    # division path 2 (a b) / (a + b), three roundings (sum, product,
    # quotient), so at most 1.5 units of 2^-52; just inside the limits: the
    # Newton-Raphson path
    rng = np.random.default_rng(7)
    m = 4000
    lo = 10.0 ** rng.uniform(-36, -31, (2, m))          # sums < 1e-30
    hi = 10.0 ** rng.uniform(30.5, 35, (2, m))          # sums > 1e30
    in_lo = 10.0 ** rng.uniform(-29.5, -28, (2, m))     # sums just above 1e-30
    in_hi = 10.0 ** rng.uniform(27, 29.5, (2, m))       # sums just below 1e30
    for (a, b), bound in ((lo, 1.5 * 2.0 ** -52), (hi, 1.5 * 2.0 ** -52), (in_lo, 2.0 ** -51),
                          (in_hi, 2.0 ** -51)):
        got = faces_on_gpu(a, b)
        ref = exact_harmonic(a, b)
        assert (np.abs(got - ref) / ref).max() <= bound
