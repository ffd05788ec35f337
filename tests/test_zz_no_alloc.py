"""The allocation-free preconditioner apply against the allocating one.

etc_apply_reference_inverse_static serves callers that cannot allocate device
memory (their GPU memory belongs to another allocator, or they cannot take the
synchronisation cudaFree may cause); it keeps its working memory in a fixed
array inside the library.  Two calls in a row, on different sizes and
parameters, must match etc_apply_preconditioner (FP64) to the tolerance of the
other preconditioner parity tests; sizes over the limit are refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2404_02433_b300 import binding as B

pytestmark = pytest.mark.gpu


def relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_static_scratch_matches_allocating_entry_point():
    stream = torch.cuda.current_stream().cuda_stream
    cases = [((18, 24, 20), [0.7, 1.9, 3.1, 0.4, 2.2]),
             ((12, 16, 33), [2.5, 0.3, 1.1, 4.0, 0.9])]
    for call, (shape, kref) in enumerate(cases):
        rng = np.random.default_rng(100 + call)
        kappa = torch.from_numpy(rng.uniform(0.5, 2.0, shape)).cuda()
        rve = B.RVE(kappa)
        rve.set_reference(2, B.ETC_REF_USER, kref)
        r = torch.from_numpy(rng.standard_normal(shape)).cuda()
        z_ref = torch.empty_like(r)
        B.etc_apply_preconditioner(rve.h, 2, B.ETC_PREC_FP64, r, z_ref)
        z = torch.full_like(r, float("nan"))
        n2, n1, n0 = shape
        st = B.etc_apply_reference_inverse_static(n0, n1, n2, kref, r, z, stream)
        assert st == B.ETC_OK
        torch.cuda.synchronize()
        assert relmax(z.cpu().numpy(), z_ref.cpu().numpy()) < 1e-12
        rve.close()


def test_static_scratch_refuses_oversized_problems():
    r = torch.zeros(8, device="cuda", dtype=torch.float64)
    z = torch.zeros(8, device="cuda", dtype=torch.float64)
    kref = [1.0] * 5
    assert B.etc_apply_reference_inverse_static(2049, 1, 1, kref, r, z) == B.ETC_EINVAL
    assert B.etc_apply_reference_inverse_static(1024, 1024, 2, kref, r, z) == B.ETC_EINVAL
    assert B.etc_apply_reference_inverse_static(2, 2, 2, [1, 1, -1, 1, 1], r, z) == B.ETC_EINVAL
