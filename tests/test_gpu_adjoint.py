"""Adjoint gradient d kappa_eff / d log kappa on the GPU (etc_gradient, autograd).

Checked against the oracle's adjoint (32^3 lognormal field, correlation length
8, sigma 1), central finite differences of GPU solves (16^3), the identities
the discrete system fixes (sum over voxels = kappa_eff by degree-1
homogeneity, non-negative entries), and, at 256^3, by the same identities.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etc_oracle as O
from paper_2404_02433_b300 import binding as B
from paper_2404_02433_b300 import microstructure as M
from paper_2404_02433_b300.autograd import effective_conductivity

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("direction", [0, 2])
def test_gradient_matches_oracle_adjoint(direction):
    k = M.lognormal_field((32, 32, 32), 8.0, 1.0, 5003)
    ky = k * 1.5
    G_o, kap_o, _, _ = O.adjoint_gradient(k, ky, k, direction, rtol=1e-12)
    rve = B.RVE(dev(k), dev(ky), dev(k))
    G, kap, infos = rve.gradient(direction, rtol=1e-12, per_component=True)
    G = G.cpu().numpy()
    assert kap == pytest.approx(kap_o, rel=1e-10)
    assert np.abs(G - G_o).max() <= 1e-8 * np.abs(G_o).max()
    Gs, _, _ = rve.gradient(direction, rtol=1e-12)
    assert np.abs(Gs.cpu().numpy() - G_o.sum(axis=0)).max() <= 1e-8 * np.abs(G_o).max()


def test_gradient_mixed_precision_matches_fp64():
    # both solves (state and adjoint) through the double-float vectors
    k = M.lognormal_field((32, 40, 24), 8.0, 1.0, 5004)
    rve = B.RVE(dev(k))
    G64, kap64, _ = rve.gradient(2, rtol=1e-10)
    Gm, kapm, infos = rve.gradient(2, rtol=1e-10, precision=B.ETC_PREC_MIXED)
    G64, Gm = G64.cpu().numpy(), Gm.cpu().numpy()
    assert kapm == pytest.approx(kap64, rel=1e-8)
    assert np.abs(Gm - G64).max() <= 1e-6 * np.abs(G64).max()
    assert all(i["status"] == B.ETC_OK and i["true_relres"] < 1e-9 for i in infos)


def test_gradient_central_differences():
    k = M.lognormal_field((16, 16, 16), 8.0, 1.0, 5002)
    rve = B.RVE(dev(k))
    G, kap, _ = rve.gradient(2, rtol=1e-13)
    G = G.cpu().numpy()
    eps = 1e-4
    for idx in [(0, 3, 5), (15, 8, 8), (7, 0, 15), (9, 9, 2), (4, 12, 11)]:
        kp = k.copy(); kp[idx] *= np.exp(eps)
        km = k.copy(); km[idx] *= np.exp(-eps)
        up, _ = B.RVE(dev(kp)).solve(2, rtol=1e-13)
        dn, _ = B.RVE(dev(km)).solve(2, rtol=1e-13)
        assert G[idx] == pytest.approx((up - dn) / (2 * eps), rel=1e-5, abs=1e-9 * kap)


def test_gradient_identities_and_autograd():
    k = M.lognormal_field((24, 20, 28), 6.0, 1.0, 7)
    logk = dev(np.log(k)).requires_grad_(True)
    y = effective_conductivity(logk, direction=1, rtol=1e-12)
    y.backward()
    g = logk.grad.cpu().numpy()
    assert g.sum() == pytest.approx(float(y.detach()), rel=1e-9)
    assert g.min() >= -1e-12 * float(y)
    # directional derivative against central differences through the Function
    v = np.random.default_rng(1).standard_normal(k.shape)
    eps = 1e-5
    with torch.no_grad():
        up = effective_conductivity(logk + eps * dev(v), direction=1, rtol=1e-13)
        dn = effective_conductivity(logk - eps * dev(v), direction=1, rtol=1e-13)
    assert float((up - dn) / (2 * eps)) == pytest.approx(float((g * v).sum()), rel=1e-5)


def test_autograd_forward_without_gradient_skips_the_adjoint():
    # without requires_grad (or under no_grad) the Function runs one PCG solve
    k = M.lognormal_field((20, 24, 16), 6.0, 1.0, 11)
    logk = dev(np.log(k))
    n0 = B.etc_kernel_launches()
    with torch.no_grad():
        y0 = effective_conductivity(logk.clone().requires_grad_(True), direction=0, rtol=1e-12)
    n1 = B.etc_kernel_launches()
    y1 = effective_conductivity(logk.clone().requires_grad_(True), direction=0, rtol=1e-12)
    n2 = B.etc_kernel_launches()
    assert float(y0) == pytest.approx(float(y1), rel=1e-12)
    assert (n1 - n0) < (n2 - n1)
    assert float(effective_conductivity(logk, direction=0, rtol=1e-12)) == float(y0)


def test_gradient_full_size_adjoint_config():
    # 256^3 lognormal (correlation length 8, sigma 1), FP64 forward and adjoint to 1e-10
    k = M.lognormal_field((256, 256, 256), 8.0, 1.0, 5001)
    rve = B.RVE(dev(k))
    G, kap, infos = rve.gradient(0, rtol=1e-10)
    assert infos[0]["status"] == B.ETC_OK and infos[1]["status"] == B.ETC_OK
    total = float(G.sum())
    assert total == pytest.approx(kap, rel=1e-6)
    assert float(G.min()) >= -1e-8 * float(G.max())
