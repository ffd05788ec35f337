"""Batched tensors in one CUDA graph (etc_batch_*) against individual solves
and the oracle, and the 64-RVE uneven batch of the batched workload."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etc_oracle as O
from paper_2404_02433_b300 import binding as B
from paper_2404_02433_b300 import microstructure as M

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def small_media():
    return [M.random_spheres((24, 24, 24), (2, 4), 0.3, 11, 1.0, 30.0)[0],
            M.random_spheres((20, 28, 32), (2, 5), 0.25, 12, 1.0, 200.0)[0],
            M.two_phase_random((11, 13, 17), 13, 0.3, 1.0, 8.0)]


@pytest.mark.parametrize("precision", [B.ETC_PREC_FP64, B.ETC_PREC_MIXED,
                                       B.ETC_PREC_MIXED_F64])
def test_batch_matches_individual_tensors(precision):
    media = small_media()
    rves = [B.RVE(dev(k)) for k in media]
    batch = B.Batch(rves, rtol=1e-10, maxit=400, precision=precision)
    Ks, infos, ms, st = batch.run()
    assert st == B.ETC_OK and ms > 0
    for i, rv in enumerate(rves):
        K1, inf1, st1 = rv.tensor(rtol=1e-10, maxit=400, precision=precision)
        np.testing.assert_allclose(Ks[i], K1, rtol=1e-12, atol=1e-13 * max(map(abs, K1)))
        for d in range(3):
            assert infos[3 * i + d]["iters"] == inf1[d]["iters"]
    # a second run of the same graph gives the same answer
    Ks2, _, _, _ = batch.run()
    assert Ks2 == Ks
    batch.close()


def test_batch_matches_oracle():
    media = small_media()
    rves = [B.RVE(dev(k)) for k in media]
    Ks, infos, ms, st = B.Batch(rves, rtol=1e-10, maxit=400).run()
    assert st == B.ETC_OK
    for i, k in enumerate(media):
        K_o, _ = O.effective_tensor(k, rtol=1e-10)
        K = np.array(Ks[i]).reshape(3, 3)
        np.testing.assert_allclose(np.diag(K), np.diag(K_o), rtol=1e-9)
        assert np.abs(K - K_o).max() <= 1e-9 * np.abs(K_o).max()


def test_batch_reports_noconv():
    k = M.random_spheres((24, 24, 24), (2, 4), 0.3, 11, 1.0, 1000.0)[0]
    Ks, infos, ms, st = B.Batch([B.RVE(dev(k))], rtol=1e-12, maxit=4).run()
    assert st == B.ETC_ENOCONV
    assert all(i["status"] == B.ETC_ENOCONV and i["iters"] == 4 for i in infos)


def batched_workload(count=64):
    return [M.batched_sphere_member(i) for i in range(count)]


@pytest.mark.parametrize("precision", [B.ETC_PREC_FP64, B.ETC_PREC_MIXED])
def test_batched_workload_64_uneven_rves(precision):
    media = batched_workload()
    rves = [B.RVE(dev(k)) for (_, _, _, k) in media]
    batch = B.Batch(rves, rtol=1e-8, precision=precision)
    Ks, infos, ms, st = batch.run()
    assert st == B.ETC_OK
    for i, (n, phi, c, k) in enumerate(media):
        K = np.array(Ks[i]).reshape(3, 3)
        voigt, reuss = k.mean(), 1.0 / (1.0 / k).mean()
        assert np.all(np.diag(K) > reuss * (1 - 1e-6)) and np.all(np.diag(K) < voigt * (1 + 1e-6))
        for d in range(3):
            assert infos[3 * i + d]["true_relres"] < 1e-7
    # two of the RVEs against individual FP64 solves
    for i in (0, 37):
        K1, _, _ = rves[i].tensor(rtol=1e-8)
        np.testing.assert_allclose(np.diag(np.array(Ks[i]).reshape(3, 3)),
                                   np.diag(np.array(K1).reshape(3, 3)), rtol=2e-6)
    batch.close()
