"""Out-of-bounds writes into caller memory, caught by canaries.

Every caller-owned output of the C ABI (the operator, the preconditioner in
its three precisions, the plane transforms, the solution, the gradient, the
allocation-free preconditioner) is written into the middle of a larger device
buffer whose other elements hold a canary value; after the call the canaries
must be bit-for-bit intact, and so must the inputs (which the library only
reads).  The shapes leave partial tiles on every axis (rows per block, columns
per block, planes per chunk).  Each span starts 512 bytes into its buffer, so
its alignment is that of a fresh allocation.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2404_02433_b300 import binding as B

pytestmark = pytest.mark.gpu

CANARY = -3.0e300
PAD = 64  # doubles before and after each span


class Padded:
    def __init__(self, shape, fill=None):
        self.n = int(np.prod(shape))
        self.buf = torch.full((PAD + self.n + PAD,), CANARY, dtype=torch.float64, device="cuda")
        self.span = self.buf[PAD:PAD + self.n].view(shape)
        if fill is not None:
            self.span.copy_(torch.as_tensor(fill, dtype=torch.float64).reshape(shape))
        self.before = self.span.clone()

    def guards_intact(self):
        return bool((self.buf[:PAD] == CANARY).all()) and bool((self.buf[PAD + self.n:] == CANARY).all())

    def unchanged(self):
        return bool(torch.equal(self.span, self.before))


SHAPES = [(5, 7, 9), (13, 11, 3), (9, 37, 40), (33, 20, 18), (6, 64, 96)]


def medium(shape, seed):
    rng = np.random.default_rng(seed)
    return [torch.from_numpy(rng.uniform(0.3, 4.0, shape)).cuda() for _ in range(3)]


@pytest.mark.parametrize("shape", SHAPES)
def test_component_outputs_stay_in_bounds(shape):
    kx, ky, kz = medium(shape, sum(shape))
    rve = B.RVE(kx, ky, kz, lengths=(1.0, 1.2, 0.9))
    rng = np.random.default_rng(7)
    for d in range(3):
        fshape = tuple(reversed(rve.loading_dims(d)))
        src = Padded(fshape, rng.standard_normal(fshape))
        out = Padded(fshape)
        B.etc_apply_operator(rve.h, d, src.span, out.span)
        assert out.guards_intact() and src.guards_intact() and src.unchanged()
        for prec in (B.ETC_PREC_FP64, B.ETC_PREC_MIXED, B.ETC_PREC_MIXED_F64):
            out = Padded(fshape)
            B.etc_apply_preconditioner(rve.h, d, prec, src.span, out.span)
            assert out.guards_intact() and src.guards_intact() and src.unchanged()
        for inverse in (0, 1):
            out = Padded(fshape)
            B.etc_dct_planes(rve.h, d, inverse, src.span, out.span)
            assert out.guards_intact() and src.guards_intact() and src.unchanged()
    rve.close()


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_solution_and_gradient_stay_in_bounds(shape):
    kx, _, _ = medium(shape, 3 * sum(shape))
    k = Padded(shape, kx)
    rve = B.RVE(k.span)
    for d in range(3):
        for prec in (B.ETC_PREC_FP64, B.ETC_PREC_MIXED):
            rve.solve(d, rtol=1e-9, precision=prec)
            sol = Padded(shape)
            B.etc_get_solution(rve.h, d, sol.span)
            assert sol.guards_intact()
        for per_component in (0, 1):
            g = Padded(((3,) if per_component else ()) + shape)
            B.etc_gradient(rve.h, d, g.span, opts=B.make_opts(rtol=1e-10),
                           per_component=per_component)
            assert g.guards_intact()
    assert k.guards_intact() and k.unchanged()
    rve.close()


def test_allocation_free_apply_stays_in_bounds():
    shape = (9, 37, 40)
    rng = np.random.default_rng(5)
    r = Padded(shape, rng.standard_normal(shape))
    z = Padded(shape)
    st = B.etc_apply_reference_inverse_static(shape[2], shape[1], shape[0],
                                              [0.7, 1.9, 3.1, 0.4, 2.2], r.span, z.span,
                                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == B.ETC_OK
    assert z.guards_intact() and r.guards_intact() and r.unchanged()
