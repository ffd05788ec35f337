"""The CUDA path against the values the paper prints in Table 3 (Sec. 4.1).

Centre ball of radius 1/4 in the unit cube at 512^3, kappa_inc inside (voxel
centre rule) and 1 outside, loading along z.  The paper prints kappa_eff^z to
three decimals and states that it no longer changes for rtol <= 1e-5; each
row is solved here at rtol 1e-8 by the FP64 path and by the mixed path
(FP32 preconditioner, double-float vectors) and must round to the printed
value.  The iteration counts of the table depend on the LP vertex SciPy
returned (Algorithm 2 has no unique optimum) and are compared only loosely.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2404_02433_b300 import binding as B
from paper_2404_02433_b300 import microstructure as M

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows():
    rows = []
    with open(os.path.join(GOLDEN, "table3_centre_ball_512.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows.append((float(v[0]), float(v[1]), [int(x) for x in v[2:]]))
    return rows


@pytest.fixture(scope="module")
def ball_mask():
    inside = M.centre_ball(512, 2.0, 1.0) == 2.0
    return torch.from_numpy(inside).cuda()


@pytest.mark.parametrize("row", _rows(), ids=lambda r: f"kinc{r[0]:g}")
def test_table3_centre_ball_512(ball_mask, row):
    kinc, expect, iters_paper = row
    k = torch.where(ball_mask, torch.tensor(kinc, dtype=torch.float64, device="cuda"),
                    torch.tensor(1.0, dtype=torch.float64, device="cuda")).contiguous()
    rve = B.RVE(k)
    try:
        for precision in (B.ETC_PREC_FP64, B.ETC_PREC_MIXED):
            kap, inf = rve.solve(2, rtol=1e-8, precision=precision)
            assert inf["status"] == B.ETC_OK
            assert abs(kap - expect) <= 5e-4 + 1e-12, (precision, kap, expect)
            # soft: the paper's count at rtol 1e-8 came from another LP vertex
            assert inf["iters"] <= 3 * iters_paper[3] + 10, (precision, inf["iters"])
            print(f"kinc {kinc:g} prec {precision}: kappa_eff^z {kap:.6f} "
                  f"(paper {expect}), {inf['iters']} iterations (paper {iters_paper[3]})")
    finally:
        rve.close()
        del k
        torch.cuda.empty_cache()
