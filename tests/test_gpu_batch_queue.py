"""Batches whose iterations run as persistent launches over a device work queue.

Handles of equal sizes with register-resident transform lengths form a class:
per loading direction one graph WHILE loop serves all of them, each kernel of
the PCG iteration (Algorithm 1 with Algorithm 3) one persistent launch whose
blocks take (solve, block) items from the class's queue.  Checked against the
oracle, against the same batch on per-solve loops (the default batch form),
against individual solves, for repeatability, the iteration cap, and with a
handle of other sizes (its own loops) in the same graph.
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


def queue_media():
    # three 32^3 members (one class), one 64^3 (a class of one), two
    # 32 x 64 x 96 boxes (a non-cubic class: every frame has lengths 32..96),
    # and a 24^3 medium (not a register-resident length: its own loops)
    return [M.random_spheres((32, 32, 32), (2, 5), 0.3, 21, 1.0, 30.0)[0],
            M.random_spheres((32, 32, 32), (2, 5), 0.2, 22, 1.0, 300.0)[0],
            M.two_phase_random((32, 32, 32), 23, 0.35, 1.0, 12.0),
            M.random_spheres((64, 64, 64), (3, 8), 0.25, 24, 1.0, 100.0)[0],
            M.random_spheres((32, 64, 96), (3, 7), 0.25, 25, 1.0, 50.0)[0],
            M.random_spheres((32, 64, 96), (3, 7), 0.3, 26, 1.0, 8.0)[0],
            M.random_spheres((24, 24, 24), (2, 4), 0.3, 27, 1.0, 20.0)[0]]


@pytest.mark.parametrize("precision", [B.ETC_PREC_FP64, B.ETC_PREC_MIXED])
def test_queue_batch_matches_oracle_and_per_solve_loops(precision):
    media = queue_media()
    rves = [B.RVE(dev(k)) for k in media]
    # FP64 at the FP64 bar's rtol; the mixed form at 1e-9, where it holds 1e-6
    # against the converged value (at 1e-8 it stops about 1e-6 away, as FP64 does)
    rtol = 1e-10 if precision == B.ETC_PREC_FP64 else 1e-9
    batch = B.Batch(rves, rtol=rtol, precision=precision, queue=True)
    assert batch.queued() == 6  # all but the 24^3 handle
    Ks, infos, ms, st = batch.run()
    assert st == B.ETC_OK and ms > 0
    # the same graph again: bitwise the same (fixed-order reductions)
    Ks2, infos2, _, _ = batch.run()
    assert Ks2 == Ks and [i["iters"] for i in infos2] == [i["iters"] for i in infos]
    batch.close()
    ref = B.Batch(rves, rtol=rtol, precision=precision)
    assert ref.queued() == 0
    Kp, infp, _, stp = ref.run()
    ref.close()
    assert stp == B.ETC_OK
    tol = 1e-9 if precision == B.ETC_PREC_FP64 else 1e-6
    for i, k in enumerate(media):
        K = np.array(Ks[i]).reshape(3, 3)
        # the same solves on per-solve loops (tuned one-solve kernels)
        np.testing.assert_allclose(K, np.array(Kp[i]).reshape(3, 3), rtol=tol,
                                   atol=tol * np.abs(K).max())
        for d in range(3):
            assert abs(infos[3 * i + d]["iters"] - infp[3 * i + d]["iters"]) <= 1
            assert infos[3 * i + d]["status"] == B.ETC_OK
            assert infos[3 * i + d]["true_relres"] < 10 * rtol
        # the oracle (FP64 Algorithm 1 at rtol 1e-10)
        K_o, res_o = O.effective_tensor(k, rtol=1e-10)
        np.testing.assert_allclose(np.diag(K), np.diag(K_o), rtol=tol)
        assert np.abs(K - K_o).max() <= tol * np.abs(K_o).max()
        if precision == B.ETC_PREC_FP64:
            for d in range(3):
                assert abs(infos[3 * i + d]["iters"] - res_o[d].iters) <= 1


def test_queue_batch_matches_individual_solves():
    media = queue_media()[:4]
    rves = [B.RVE(dev(k)) for k in media]
    batch = B.Batch(rves, rtol=1e-10, precision=B.ETC_PREC_FP64, queue=True)
    assert batch.queued() == 4
    Ks, infos, _, st = batch.run()
    batch.close()
    assert st == B.ETC_OK
    for i, rv in enumerate(rves):
        K1, inf1, st1 = rv.tensor(rtol=1e-10)
        np.testing.assert_allclose(Ks[i], K1, rtol=1e-9, atol=1e-9 * max(map(abs, K1)))
        for d in range(3):
            assert abs(infos[3 * i + d]["iters"] - inf1[d]["iters"]) <= 1
        # the handle is usable after the batch: its solution of the last direction
        p = rv.solution(2).cpu().numpy()
        assert np.all(np.isfinite(p)) and p.min() >= -1e-9 and p.max() <= 1 + 1e-9


@pytest.mark.parametrize("precision", [B.ETC_PREC_FP64, B.ETC_PREC_MIXED])
def test_queue_batch_iteration_cap(precision):
    # maxit = 4 on a hard medium: every solve of the class stops at the cap
    media = [M.random_spheres((32, 32, 32), (2, 5), 0.3, 31 + s, 1.0, 1000.0)[0]
             for s in range(3)]
    rves = [B.RVE(dev(k)) for k in media]
    batch = B.Batch(rves, rtol=1e-12, maxit=4, precision=precision, queue=True)
    assert batch.queued() == 3
    Ks, infos, _, st = batch.run()
    batch.close()
    assert st == B.ETC_ENOCONV
    assert all(i["status"] == B.ETC_ENOCONV and i["iters"] == 4 for i in infos)
    assert all(np.all(np.isfinite(K)) for K in Ks)


def test_queue_batch_fp64_lengths_160_192():
    # lengths whose FP64 block-floating-point transforms take eight threads a
    # line (n = 160, 192: the second-stage DFTs go round-robin): a class of
    # two 32 x 96 x 160 boxes and a class of one 192 x 32 x 64 box, against
    # the oracle and the per-solve batch
    media = [M.random_spheres((32, 96, 160), (3, 7), 0.25, 41, 1.0, 60.0)[0],
             M.random_spheres((32, 96, 160), (3, 7), 0.3, 42, 1.0, 5.0)[0],
             M.random_spheres((192, 32, 64), (3, 7), 0.25, 43, 1.0, 200.0)[0]]
    rves = [B.RVE(dev(k)) for k in media]
    batch = B.Batch(rves, rtol=1e-10, precision=B.ETC_PREC_FP64, queue=True)
    assert batch.queued() == 3
    Ks, infos, _, st = batch.run()
    batch.close()
    assert st == B.ETC_OK
    ref = B.Batch(rves, rtol=1e-10, precision=B.ETC_PREC_FP64)
    Kp, infp, _, stp = ref.run()
    ref.close()
    assert stp == B.ETC_OK
    for i, k in enumerate(media):
        K = np.array(Ks[i]).reshape(3, 3)
        np.testing.assert_allclose(K, np.array(Kp[i]).reshape(3, 3), rtol=1e-9,
                                   atol=1e-9 * np.abs(K).max())
        K_o, res_o = O.effective_tensor(k, rtol=1e-10)
        np.testing.assert_allclose(np.diag(K), np.diag(K_o), rtol=1e-9)
        for d in range(3):
            assert infos[3 * i + d]["status"] == B.ETC_OK
            assert abs(infos[3 * i + d]["iters"] - res_o[d].iters) <= 1
