"""General face data and source term on the GPU (etc_solve_general): the smooth
test of Table 2 (Sec. 4.1) up to 512^3, parity with the oracle, and the
"one" vs LP reference parameters on the channel lattice of Sec. 4.4."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etc_oracle as O
from paper_2404_02433_b300 import binding as B
from paper_2404_02433_b300 import microstructure as M

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def table2():
    rows = {}
    with open(os.path.join(GOLDEN, "table2_smooth.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                r, n, e, it = line.split()
                rows[(float(r), int(n))] = (float(e), int(it))
    return rows


def gpu_smooth(n, rtol, precision=B.ETC_PREC_FP64):
    kx, ky, kz, pin, pout, src, exact = M.smooth_problem(n)
    rve = B.RVE(dev(kx), dev(ky), dev(kz))
    info = rve.solve_general(2, dev(pin), dev(pout), dev(src), rtol=rtol, precision=precision)
    p = rve.solution(2).cpu().numpy()
    rve.close()
    return p, exact, info


def test_smooth_32_matches_oracle():
    kx, ky, kz, pin, pout, src, exact = M.smooth_problem(32)
    po, it_o = O.solve_general(kx, ky, kz, pin, pout, src, rtol=1e-12)
    p, _, info = gpu_smooth(32, 1e-12)
    assert np.abs(p - po).max() <= 1e-10 * np.abs(po).max()
    assert abs(info["iters"] - it_o) <= 1
    assert info["true_relres"] < 1e-11


@pytest.mark.parametrize("n,rtol", [(32, 1e-9), (64, 1e-9), (128, 1e-9), (128, 1e-8),
                                    (512, 1e-9), (512, 1e-8)])
def test_table2_on_gpu(n, rtol):
    err, iters = table2()[(rtol, n)]
    p, exact, info = gpu_smooth(n, rtol)
    l2 = np.sqrt(((p - exact) ** 2).sum() / n ** 3)
    assert abs(l2 - err) / err < 0.01
    assert abs(info["iters"] - iters) <= 1


@pytest.mark.parametrize("n", [64, 96])
def test_table2_mixed_precision(n):
    # general face data and source through the mixed path (FP32 preconditioner,
    # double-float vectors): the L2 error of Table 2's converged rows
    kx, ky, kz, pin, pout, src, exact = M.smooth_problem(n)
    p64, _, i64 = gpu_smooth(n, 1e-10)
    pm, _, im = gpu_smooth(n, 1e-10, precision=B.ETC_PREC_MIXED)
    assert np.abs(pm - p64).max() <= 1e-7 * np.abs(p64).max()
    assert im["true_relres"] < 2e-10
    l2 = lambda p: np.sqrt(((p - exact) ** 2).sum() / n ** 3)
    assert abs(l2(pm) - l2(p64)) <= 1e-3 * l2(p64)


def test_general_data_in_x_direction_matches_oracle():
    shape = (10, 12, 14)
    rng = np.random.default_rng(9)
    kx, ky, kz = (rng.uniform(0.5, 3.0, shape) for _ in range(3))
    src = rng.standard_normal(shape)
    rve = B.RVE(dev(kx), dev(ky), dev(kz))
    n0, n1, n2 = rve.loading_dims(0)
    pin = rng.standard_normal((n1, n0))
    pout = rng.standard_normal((n1, n0))
    info = rve.solve_general(0, dev(pin), dev(pout), dev(src), rtol=1e-12)
    p = rve.solution(0).cpu().numpy()
    (k0, k1, k2), lens = O.permute_medium(kx, ky, kz, (1.0, 1.0, 1.0), 0)
    srcp = O.permute_medium(src, src, src, (1.0, 1.0, 1.0), 0)[0][0]
    po, _ = O.solve_general(k0, k1, k2, pin, pout, srcp, lens, rtol=1e-12)
    po = O.unpermute_field(po, 0)
    assert np.abs(p - po).max() <= 1e-10 * np.abs(po).max()


@pytest.mark.parametrize("psi", [2, 3])
def test_channel_lattice_lp_beats_ones(psi):
    # Sec. 4.4: for the anisotropic channel lattice the LP reference parameters
    # converge clearly faster than all-ones for psi = 2, 3 (paper: Fig. 10).
    kx, ky, kz = M.channel_lattice(256, 32, psi)
    rve = B.RVE(dev(kx), dev(ky), dev(kz))
    iters = {}
    for name, mode in (("ones", B.ETC_REF_ONES), ("lp", B.ETC_REF_LP)):
        rve.set_reference(2, mode)
        kap, info = rve.solve(2, rtol=1e-8, maxit=5000, precision=B.ETC_PREC_MIXED)
        iters[name] = info["iters"]
        assert info["status"] == B.ETC_OK
    assert iters["lp"] < 0.8 * iters["ones"]
