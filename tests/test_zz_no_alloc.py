"""The allocation-free preconditioner apply against the allocating one and the oracle.

etc_apply_reference_inverse_static serves callers that cannot allocate device
memory (their GPU memory belongs to another allocator, or they cannot take the
synchronisation cudaFree may cause); it keeps its working memory in a fixed
array inside the library.  Two calls in a row, on different sizes and
parameters, must match etc_apply_preconditioner (FP64) to the tolerance of the
other preconditioner parity tests; the CPU oracle's Algorithm 3 checks it at
the edges of its stated limits (an axis of 2048, exactly 2^20 cells), on odd
lengths (the direct-sum transforms) and on axes of one and two voxels, with
canary-padded buffers and on a side stream; sizes over the limit are refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etc_oracle as O
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


CANARY = np.frombuffer(np.uint64(0x7FF4DEADBEEFCAFE).tobytes(), dtype=np.float64)[0]
PAD = 64  # canary doubles on each side (512 bytes: the buffers stay 256-byte aligned)


@pytest.mark.parametrize("shape,side_stream", [
    ((1, 512, 2048), True),     # n0 at its limit, 2^20 cells, one plane
    ((1, 1024, 1024), False),   # 2^20 cells
    ((128, 4, 2048), True),     # n0 = 2048 with 128 planes: exactly 2^20 cells
    ((8, 2048, 4), False),      # n1 at its limit
    ((6, 10, 45), True),        # odd n0: direct-sum transform on axis 0
    ((5, 9, 1), False),         # n0 = 1, odd n1
    ((7, 15, 2), True),         # n0 = 2 (one complex point, no FFT stage), odd n1
])
def test_static_scratch_matches_oracle_at_its_limits(shape, side_stream):
    n2, n1, n0 = shape
    n = n0 * n1 * n2
    rng = np.random.default_rng(n0 * 7 + n1 * 3 + n2)
    kref = [0.7, 1.9, 3.1, 0.4, 2.2]
    r_np = rng.standard_normal(shape)
    zo = O.apply_reference_inverse(r_np, kref)
    rbuf = torch.full((n + 2 * PAD,), CANARY, dtype=torch.float64, device="cuda")
    zbuf = torch.full((n + 2 * PAD,), CANARY, dtype=torch.float64, device="cuda")
    rbuf[PAD:PAD + n] = torch.from_numpy(r_np.ravel()).cuda()
    r, z = rbuf[PAD:PAD + n], zbuf[PAD:PAD + n]
    s = torch.cuda.Stream() if side_stream else torch.cuda.current_stream()
    torch.cuda.synchronize()
    for _ in range(2):  # the second call finds the array holding the first call's values
        st = B.etc_apply_reference_inverse_static(n0, n1, n2, kref, r, z, s.cuda_stream)
        assert st == B.ETC_OK
        s.synchronize()
        assert relmax(z.cpu().numpy().reshape(shape), zo) < 1e-11
    zb, rb = zbuf.cpu().numpy(), rbuf.cpu().numpy()
    canary_bits = np.float64(CANARY).view(np.uint64)
    for buf in (zb, rb):
        assert np.all(buf[:PAD].view(np.uint64) == canary_bits)
        assert np.all(buf[PAD + n:].view(np.uint64) == canary_bits)
    assert np.array_equal(rb[PAD:PAD + n], r_np.ravel())


def test_static_scratch_refuses_oversized_problems():
    r = torch.zeros(8, device="cuda", dtype=torch.float64)
    z = torch.zeros(8, device="cuda", dtype=torch.float64)
    kref = [1.0] * 5
    assert B.etc_apply_reference_inverse_static(2049, 1, 1, kref, r, z) == B.ETC_EINVAL
    assert "2^20" in B.load_library().etc_last_error(None).decode()
    assert B.etc_apply_reference_inverse_static(1, 2049, 1, kref, r, z) == B.ETC_EINVAL
    assert B.etc_apply_reference_inverse_static(1024, 1024, 2, kref, r, z) == B.ETC_EINVAL
    assert B.etc_apply_reference_inverse_static(2, 2, 2, [1, 1, -1, 1, 1], r, z) == B.ETC_EINVAL
