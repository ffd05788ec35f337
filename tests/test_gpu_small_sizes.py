"""Exhaustive small sizes against the oracle.

Every pair of transform-axis lengths n0, n1 in 1..17 (odd lengths take the
direct-sum transforms; even ones the half-length FFT with m = n/2 of radices 2,
3, 4, 5 and 8, or the direct sum for m = 7; n0 a multiple of 4 also takes the
bulk-tensor matvec and tridiagonal kernels of the mixed path) for the operator
of Eq. (scaled bilinear forms) and the reference inverse of Algorithm 3 in FP64
and FP32, and the 3x3 tensor with each axis of the box swept over 1..17.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etc_oracle as O
from paper_2404_02433_b300 import binding as B

pytestmark = pytest.mark.gpu

N = range(1, 18)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def relmax(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("n1", N)
def test_operator_and_preconditioner_every_small_length(n1):
    ku = [0.7, 1.9, 3.1, 0.4, 2.2]
    for n0 in N:
        n2 = 1 + (n0 + n1) % 5  # 1..5 planes
        shape = (n2, n1, n0)
        rng = np.random.default_rng(1000 * n0 + n1)
        kx, ky, kz = (rng.uniform(0.2, 5.0, shape) for _ in range(3))
        rve = B.RVE(dev(kx), dev(ky), dev(kz), lengths=(1.0, 1.3, 0.7))
        f = O.face_conductances(kx, ky, kz, (1.0, 1.3, 0.7))
        w = rng.standard_normal(shape)
        q = torch.empty(shape, dtype=torch.float64, device="cuda")
        B.etc_apply_operator(rve.h, 2, dev(w), q)
        assert relmax(q.cpu().numpy(), O.apply_operator(f, w)) < 1e-12, shape
        rve.set_reference(2, B.ETC_REF_USER, ku)
        zo = O.apply_reference_inverse(w, ku)
        for prec, tol in ((B.ETC_PREC_FP64, 1e-11), (B.ETC_PREC_MIXED, 2e-5),
                          (B.ETC_PREC_MIXED_F64, 2e-5)):
            B.etc_apply_preconditioner(rve.h, 2, prec, dev(w), q)
            assert relmax(q.cpu().numpy(), zo) < tol, (shape, prec)
        rve.close()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_tensor_every_small_length(axis):
    for n in N:
        dims = [5, 4, 6]  # x, y, z
        dims[axis] = n
        shape = (dims[2], dims[1], dims[0])
        rng = np.random.default_rng(77 * n + axis)
        kx = np.where(rng.random(shape) < 0.35, 20.0, 1.0)
        ky, kz = kx * rng.uniform(0.5, 2.0, shape), kx * rng.uniform(0.5, 2.0, shape)
        lengths = (1.0, 0.8, 1.5)
        K_o, res_o = O.effective_tensor(kx, ky, kz, lengths, rtol=1e-12)
        rve = B.RVE(dev(kx), dev(ky), dev(kz), lengths=lengths)
        K, infos, st = rve.tensor(rtol=1e-12)
        rve.close()
        K = np.array(K).reshape(3, 3)
        assert st == B.ETC_OK, n
        np.testing.assert_allclose(np.diag(K), np.diag(K_o), rtol=1e-10, err_msg=str(shape))
        assert np.abs(K - K_o).max() <= 1e-10 * np.abs(K_o).max(), shape
        # at rtol 1e-12 the last iterations sit near the rounding floor, where
        # the two implementations' residuals may cross the threshold a little
        # apart: 1 iteration, or 5 % of the count
        for d in range(3):
            assert abs(infos[d]["iters"] - res_o[d].iters) <= max(1, res_o[d].iters // 20), \
                (shape, d)
