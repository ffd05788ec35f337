"""Block-floating-point transforms of the FP64 path against the oracle.

The FP64 path may run its cosine transforms (Eq. (forward DCT), Eq. (backward
DCT), Sec. 3.2) in 64-bit fixed point with one exponent per line, for the
register-resident lengths 32..1024 (tiles -3/-4 on axis 0, -3 on axis 1, and
-4 on axis 1 for the three-stage kernels of n1 = 256, 512, 1024; chosen by the
autotuner or forced through ETC_FORCE_TILES).  These tests force them on
every such length, on each axis alone and on both, and compare with the
oracle's direct O(n^2) transforms and its reference inverse (Algorithm 3):
  * the 2-D transform pair within 1e-14 and the preconditioner within 2e-14
    (max norm): the error of FP64 transforms (1e-15 and 2e-15 measured at
    n = 512, fixed point and floating point alike), with margin, and 100 times
    inside the FP64 kernels' bars;
  * planes scaled by 10^-300 .. 10^200 in one array, each within 1e-14 of the
    oracle relative to its own size (one exponent per line, not per array),
    a zero plane staying zero;
  * a NaN in one plane turns that plane, and only that plane, into NaN, and
    an output above the binary64 range becomes an infinity;
  * lines at the growth bounds of the arithmetic (constant, alternating, a
    spike; backward, one dominant coefficient) within tolerances derived from
    the per-line quantisation;
  * a whole solve with the forced tiles reaches the oracle's kappa_eff.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etc_oracle as O
from paper_2404_02433_b300 import binding as B
from paper_2404_02433_b300 import microstructure as M

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def relmax(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# [n2][n1][n0]: every length of these kernels (32..1024; radices 2, 3, 5 and
# the non-power-of-two backward scale) on axis 0 and on axis 1 with ragged
# partners, and pairs of them on both axes including the benchmark length
SHAPES = [(3, 40, 32), (3, 32, 40), (2, 24, 64), (2, 64, 24), (2, 20, 96), (2, 96, 20),
          (3, 20, 128), (3, 128, 20), (2, 12, 160), (2, 160, 12), (2, 10, 192), (2, 192, 10),
          (2, 12, 256), (2, 256, 12), (2, 6, 384), (2, 384, 6), (2, 6, 512), (2, 512, 6),
          (2, 3, 1024), (2, 1024, 3), (2, 96, 160), (2, 384, 192), (2, 64, 512), (2, 512, 256)]
# forced (axis-0 forward, axis-0 backward, axis 1); 1 and 2 are generic
# floating-point tiles, used where the other axis has no fixed-point kernel
FIXED = [(-3, -3, -3), (-4, -4, -3), (-3, -4, 1), (-4, -3, 1), (1, 1, -3), (2, 2, -3),
         (1, 1, -4), (-3, -3, -4)]  # -4 on axis 1: the three-stage kernels (n1 = 256..1024)


def forced(monkeypatch, tiles):
    monkeypatch.setenv("ETC_FORCE_TILES", ",".join(map(str, tiles)))


def medium(shape, seed):
    rng = np.random.default_rng(seed)
    kx, ky, kz = (rng.uniform(0.2, 5.0, shape) for _ in range(3))
    return B.RVE(dev(kx), dev(ky), dev(kz)), rng


@pytest.mark.parametrize("shape", SHAPES)
def test_fixed_point_transforms_match_oracle(shape, monkeypatch):
    rve, rng = medium(shape, 7 * sum(shape))
    ku = [0.7, 1.9, 3.1, 0.4, 2.2]
    rve.set_reference(2, B.ETC_REF_USER, ku)
    r = rng.standard_normal(shape)
    zo = O.apply_reference_inverse(r, ku)
    rhat = O.dct_forward(O.dct_forward(r, 2), 1)
    z = torch.empty(shape, dtype=torch.float64, device="cuda")
    out = torch.empty_like(z)
    ran = 0
    for tiles in FIXED:
        forced(monkeypatch, tiles)
        try:
            B.etc_apply_preconditioner(rve.h, 2, B.ETC_PREC_FP64, dev(r), z)
        except B.EtcError as e:  # the other axis has no such kernel
            assert e.status == B.ETC_EINVAL and "ETC_FORCE_TILES" in str(e)
            continue
        ran += 1
        assert relmax(host(z), zo) < 2e-14, tiles
        B.etc_dct_planes(rve.h, 2, 0, dev(r), out)
        assert relmax(host(out), rhat) < 1e-14, tiles
        B.etc_dct_planes(rve.h, 2, 1, dev(rhat), out)
        assert relmax(host(out), r) < 1e-14, tiles
        # the mixed forms have no fixed-point kernels
        with pytest.raises(B.EtcError):
            B.etc_apply_preconditioner(rve.h, 2, B.ETC_PREC_MIXED, dev(r), z)
    assert ran >= 2
    rve.close()


@pytest.mark.parametrize("tiles", [(-3, -3, -3), (-4, -4, -3)])
def test_fixed_point_dynamic_range_per_line(tiles, monkeypatch):
    shape = (6, 64, 128)
    rve, rng = medium(shape, 11)
    forced(monkeypatch, tiles)
    scales = np.array([1e-200, 1.0, 0.0, 3e150, 1e-300, 7e200])
    u = rng.standard_normal(shape)
    u[1, :, :5] *= 1e-12  # a line with a wide range inside it
    u *= scales[:, None, None]
    # exact zeros and subnormals inside rows and columns of normal range (the
    # conversions' short path for such lines, against their full path)
    u[1, :, 7:9] = 0.0
    u[1, 20:22, :] = 0.0
    u[1, 3, 10], u[1, 30, 40], u[3, 5, 6], u[3, 6, 6] = 5e-324, -2.2e-310, 1e-320, -0.0
    ref = O.dct_forward(O.dct_forward(u, 2), 1)
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    B.etc_dct_planes(rve.h, 2, 0, dev(u), out)
    got = host(out)
    back = torch.empty_like(out)
    B.etc_dct_planes(rve.h, 2, 1, dev(ref), back)
    gb = host(back)
    for k in range(shape[0]):
        if scales[k] == 0.0:
            assert not got[k].any() and not gb[k].any()
            continue
        assert relmax(got[k], ref[k]) < 1e-14, k
        assert relmax(gb[k], u[k]) < 1e-14, k
    rve.close()


def test_fixed_point_overflow_gives_infinities(monkeypatch):
    # a constant line near the top of the binary64 range: its zero-frequency
    # output (n times the value) overflows to an infinity of the right sign,
    # as in floating point; the other outputs stay finite
    shape = (2, 4, 64)
    rve, _ = medium(shape, 19)
    forced(monkeypatch, (-3, -3, 1))
    u = np.full(shape, 1e307)
    u[1] *= -1.0
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    B.etc_dct_planes(rve.h, 2, 0, dev(u), out)
    got = host(out)
    assert got[0, 0, 0] == np.inf and got[1, 0, 0] == -np.inf
    assert np.isfinite(got[:, :, 1:]).all()
    rve.close()


def test_fixed_point_nan_stays_in_its_plane(monkeypatch):
    shape = (4, 32, 64)
    rve, rng = medium(shape, 13)
    forced(monkeypatch, (-3, -3, -3))
    u = rng.standard_normal(shape)
    u[2, 5, 7] = np.nan
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    B.etc_dct_planes(rve.h, 2, 0, dev(u), out)
    got = host(out)
    assert np.isnan(got[2]).all()
    assert np.isfinite(got[[0, 1, 3]]).all()
    rve.close()


@pytest.mark.parametrize("tiles", [(-3, -3, -3), (-4, -4, -3)])
def test_fixed_point_solve_matches_oracle(tiles, monkeypatch):
    k, _ = M.random_spheres((32, 64, 64), (3, 6), 0.3, 31, 1.0, 50.0)
    ref = O.solve_direction(k, k, k, 2, rtol=1e-10)
    forced(monkeypatch, tiles)
    rve = B.RVE(torch.from_numpy(k).cuda())
    kap, inf = rve.solve(2, rtol=1e-10)
    assert inf["status"] == B.ETC_OK
    assert abs(kap - ref.kappa_eff) <= 1e-9 * ref.kappa_eff, (kap, ref.kappa_eff)
    assert abs(inf["iters"] - ref.iters) <= 1, (inf["iters"], ref.iters)
    rve.close()


@pytest.mark.parametrize("shape,ytile", [((5, 4, 512), -3), ((5, 512, 4), -3), ((5, 512, 4), -4),
                                         ((5, 4, 1024), -3), ((5, 1024, 4), -4),
                                         ((5, 4, 192), -3)])
def test_fixed_point_worst_case_growth(shape, ytile, monkeypatch):
    # lines that drive the transforms to their bounds: all equal (the whole line
    # lands in the zero-frequency output), alternating signs (the highest
    # frequency), one spike over a tiny background, and, backward, spectra of
    # equal coefficients; each within 1e-14 of the oracle relative to its line
    n2, n1, n0 = shape
    rve, rng = medium(shape, 17)
    tiles = (-3, -3, 1) if n1 == 4 else (1, 1, ytile)  # the long axis in fixed point
    forced(monkeypatch, tiles)
    axis_len = n0 if n1 == 4 else n1
    idx = np.arange(axis_len)
    lines = [np.full(axis_len, 1.0), np.where(idx % 2 == 0, 1.0, -1.0),
             np.where(idx == 7, 1.0, 1e-9 * rng.standard_normal(axis_len)),
             -np.full(axis_len, 3.5e10)]
    u = np.zeros(shape)
    for k in range(n2):
        line = lines[k % len(lines)] * (1.0 + 0.001 * k)
        if n1 == 4:
            u[k, :, :] = line[None, :]
        else:
            u[k, :, :] = line[:, None]
    # bits kept for a line's largest value: forward min(53, 61 - ceil(log2 n)),
    # backward min(53, 60 - ceil(log2 (n/2))) (the growth bounds of the
    # arithmetic); a value is quantised to units of 2^-(bits-1) of the line's
    # largest, and n such roundings add up in each forward output as a random
    # walk: about sqrt(n) units of the largest output (4 sqrt(n) allowed)
    lg = int(np.ceil(np.log2(axis_len)))
    bits_f, bits_b = min(53, 61 - lg), min(53, 61 - lg)
    tol_f = 4.0 * np.sqrt(axis_len) * 2.0 ** -(bits_f - 1)
    ref = O.dct_forward(O.dct_forward(u, 2), 1)
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    B.etc_dct_planes(rve.h, 2, 0, dev(u), out)
    got = host(out)
    for k in range(n2):
        assert relmax(got[k], ref[k]) < tol_f, (shape, k)
    # backward of spectra of equal coefficients, and of the forward results:
    # a constant line's spectrum is one coefficient n max|u| over the oracle's
    # rounding noise, which block floating point quantises to units of
    # 2^-(bits-1) of the largest coefficient (FP64 keeps each to 2^-53 of
    # itself); the output, of size max|X| / n, then carries up to n such units
    # of itself (3.4e-14 measured at n = 512, against 1e-16 for FP64
    # transforms: where these transforms trail FP64, inside the 1e-12 bar)
    spec = np.ones(shape) * (1.0 + np.arange(n2))[:, None, None]
    tol_b = axis_len * 2.0 ** -(bits_b - 1)
    for X in (spec, ref):
        back = torch.empty_like(out)
        B.etc_dct_planes(rve.h, 2, 1, dev(X), back)
        want = O.dct_backward(O.dct_backward(X, 1), 2)
        gb = host(back)
        for k in range(n2):
            assert relmax(gb[k], want[k]) < tol_b, (shape, k)
    rve.close()


@pytest.mark.parametrize("tiles", [(-3, -3, 1), (-4, -4, 2)])
def test_fixed_point_axis0_with_generic_axis1_in_a_solve(tiles, monkeypatch):
    # load z on a 37 x 100 x 96 box: axis 0 (n0 = 96, the radix-3 length) in
    # block floating point, axis 1 (n1 = 100, no such kernel) generic, in one
    # solve; kappa_eff and iterations against the oracle
    k, _ = M.random_spheres((37, 100, 96), (3, 7), 0.3, 51, 1.0, 80.0)
    ref = O.solve_direction(k, k, k, 2, rtol=1e-10)
    forced(monkeypatch, tiles)
    rve = B.RVE(torch.from_numpy(k).cuda())
    kap, inf = rve.solve(2, rtol=1e-10)
    assert B.etc_transform_tiles(rve.h, 2, B.ETC_PREC_FP64) == list(tiles)
    rve.close()
    assert inf["status"] == B.ETC_OK
    assert abs(kap - ref.kappa_eff) <= 1e-9 * ref.kappa_eff, (kap, ref.kappa_eff, tiles)
    assert abs(inf["iters"] - ref.iters) <= 1, (inf["iters"], ref.iters)
