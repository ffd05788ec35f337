"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Kernel by kernel (operator, 2-D cosine transforms, preconditioner) and end to
end (kappa_eff, the solution field, the 3x3 tensor), on seeded inputs whose
sizes span several tiles, ragged tails, odd and mixed-radix lengths, and the
degenerate one-voxel axes.  Tolerances: 1e-12 relative (max norm) for FP64
kernels, 2e-5 for the FP32 preconditioner, 1e-9 relative on kappa_eff at
rtol 1e-10 (the FP64 bar), 1e-6 for the mixed path at rtol 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import etc_oracle as O
from paper_2404_02433_b300 import binding as B
from paper_2404_02433_b300 import microstructure as M
from closed_forms import checkerboard_closed_form

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def relmax(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def make(kx, ky=None, kz=None, lengths=(1.0, 1.0, 1.0)):
    return B.RVE(dev(kx), None if ky is None else dev(ky), None if kz is None else dev(kz),
                 lengths=lengths)


SHAPES = [(18, 20, 24), (11, 13, 17), (36, 48, 40), (5, 7, 1), (9, 1, 33), (1, 6, 4),
          (16, 16, 16), (12, 10, 30)]


def oracle_faces(kx, ky, kz, lengths, direction):
    (k0, k1, k2), lens = O.permute_medium(kx, ky, kz, lengths, direction)
    return O.face_conductances(k0, k1, k2, lens), (k0.shape)


# ------------------------------------------------------------------ kernels
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_operator_matches_oracle(shape, direction):
    rng = np.random.default_rng(hash((shape, direction)) % 2**32)
    kx, ky, kz = (rng.uniform(0.1, 10.0, shape) for _ in range(3))
    lengths = (1.0, 1.3, 0.7)
    rve = make(kx, ky, kz, lengths)
    f, fshape = oracle_faces(kx, ky, kz, lengths, direction)
    assert rve.loading_dims(direction) == tuple(reversed(fshape))
    w = rng.standard_normal(fshape)
    q = torch.empty(fshape, dtype=torch.float64, device="cuda")
    B.etc_apply_operator(rve.h, direction, dev(w), q)
    assert relmax(host(q), O.apply_operator(f, w)) < 1e-12


# The mixed path's double-float operator (FP32 search direction, faces as
# double-float pairs, the face-difference form summed by Sum2): both kernels,
# the bulk-tensor one (n0 a multiple of 4 in the loading frame) and the plain
# one, against the oracle's FP64 operator on the same FP32 w; and w.q, the
# denominator of alpha, as the kernel reduces it.
@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 10, 30), (11, 13, 17), (5, 7, 1),
                                   (8, 64, 96), (40, 36, 48)])
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_double_float_operator_matches_oracle(shape, direction):
    rng = np.random.default_rng(hash((shape, direction, "df")) % 2**32)
    kx, ky, kz = (rng.uniform(0.1, 10.0, shape) for _ in range(3))
    lengths = (1.0, 1.3, 0.7)
    rve = make(kx, ky, kz, lengths)
    f, fshape = oracle_faces(kx, ky, kz, lengths, direction)
    w = rng.standard_normal(fshape).astype(np.float32)
    w64 = w.astype(np.float64)
    q = torch.empty(fshape, dtype=torch.float64, device="cuda")
    wq = B.etc_apply_operator_df(rve.h, direction, torch.from_numpy(w).cuda(), q)
    qo = O.apply_operator(f, w64)
    # faces rounded to 48-bit pairs, exact differences, Sum2: a few units of 2^-47
    assert relmax(host(q), qo) < 1e-12, (shape, direction)
    wqo = float(np.dot(w64.ravel(), qo.ravel()))
    assert wqo > 0 and abs(wq - wqo) <= 1e-11 * wqo, (wq, wqo)
    rve.close()


@pytest.mark.parametrize("shape", SHAPES + [(8, 64, 96), (4, 160, 192), (3, 200, 50),
                                   (2, 1024, 32), (2, 96, 384)])
def test_dct_planes_match_oracle(shape):
    rng = np.random.default_rng(sum(shape))
    k = rng.uniform(1.0, 2.0, shape)
    rve = make(k)
    u = rng.standard_normal(shape)
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    B.etc_dct_planes(rve.h, 2, 0, dev(u), out)
    ref = O.dct_forward(O.dct_forward(u, 2), 1)
    assert relmax(host(out), ref) < 1e-12
    back = torch.empty_like(out)
    B.etc_dct_planes(rve.h, 2, 1, dev(ref), back)
    assert relmax(host(back), u) < 1e-12


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("direction", [0, 2])
def test_preconditioner_matches_oracle(shape, direction):
    rng = np.random.default_rng(7 + sum(shape) + direction)
    kx, ky, kz = (rng.uniform(0.2, 5.0, shape) for _ in range(3))
    rve = make(kx, ky, kz)
    f, fshape = oracle_faces(kx, ky, kz, (1.0, 1.0, 1.0), direction)
    kref_o = O.reference_parameters(O.group_extrema(f))
    kref_g = rve.set_reference(direction, B.ETC_REF_LP)
    np.testing.assert_allclose(kref_g, kref_o, rtol=1e-13)
    r = rng.standard_normal(fshape)
    z = torch.empty(fshape, dtype=torch.float64, device="cuda")
    B.etc_apply_preconditioner(rve.h, direction, B.ETC_PREC_FP64, dev(r), z)
    zo = O.apply_reference_inverse(r, kref_o)
    assert relmax(host(z), zo) < 1e-11
    # user-set parameters chosen by the test
    ku = [0.7, 1.9, 3.1, 0.4, 2.2]
    rve.set_reference(direction, B.ETC_REF_USER, ku)
    B.etc_apply_preconditioner(rve.h, direction, B.ETC_PREC_FP64, dev(r), z)
    assert relmax(host(z), O.apply_reference_inverse(r, ku)) < 1e-11
    # FP32 transforms and solves (mixed paths)
    for prec in (B.ETC_PREC_MIXED, B.ETC_PREC_MIXED_F64):
        B.etc_apply_preconditioner(rve.h, direction, prec, dev(r), z)
        assert relmax(host(z), O.apply_reference_inverse(r, ku)) < 2e-5


@pytest.mark.parametrize("shape", [(4, 96, 160), (3, 192, 384), (2, 32, 1024), (2, 1024, 64),
                                   (5, 64, 96)])
def test_preconditioner_register_resident_lengths(shape):
    # every line length of the register-resident transforms beyond the powers
    # of two (96, 160, 192, 384 and 1024 on both transform axes), FP64 and FP32
    rng = np.random.default_rng(3 * sum(shape))
    kx, ky, kz = (rng.uniform(0.2, 5.0, shape) for _ in range(3))
    rve = make(kx, ky, kz)
    ku = [0.7, 1.9, 3.1, 0.4, 2.2]
    rve.set_reference(2, B.ETC_REF_USER, ku)
    _, fshape = oracle_faces(kx, ky, kz, (1.0, 1.0, 1.0), 2)
    r = rng.standard_normal(fshape)
    zo = O.apply_reference_inverse(r, ku)
    z = torch.empty(fshape, dtype=torch.float64, device="cuda")
    B.etc_apply_preconditioner(rve.h, 2, B.ETC_PREC_FP64, dev(r), z)
    assert relmax(host(z), zo) < 1e-11
    B.etc_apply_preconditioner(rve.h, 2, B.ETC_PREC_MIXED, dev(r), z)
    assert relmax(host(z), zo) < 2e-5


# the benchmark's transform length (512) on axis 0, on axis 1, and on both;
# every tile the autotuner may pick is forced in turn (ETC_FORCE_TILES), so the
# kernels a 512^3 solve runs are compared with the oracle element by element
TILES_X = [-1, -2, -3, -4, 1, 2, 4, 8, 16, 32, 64]
TILES_Y = [-1, -3, -4, 1, 2, 4, 8, 16, 32]


@pytest.mark.parametrize("shape", [(4, 512, 512), (3, 96, 512), (3, 512, 96)])
def test_length_512_every_tile_matches_oracle(shape, monkeypatch):
    rng = np.random.default_rng(512 + sum(shape))
    kx, ky, kz = (rng.uniform(0.2, 5.0, shape) for _ in range(3))
    rve = make(kx, ky, kz)
    ku = [0.7, 1.9, 3.1, 0.4, 2.2]
    rve.set_reference(2, B.ETC_REF_USER, ku)
    r = rng.standard_normal(shape)
    zo = O.apply_reference_inverse(r, ku)
    rhat = O.dct_forward(O.dct_forward(r, 2), 1)
    z = torch.empty(shape, dtype=torch.float64, device="cuda")
    out = torch.empty_like(z)
    cands = [(t, t, -1) for t in TILES_X] + [(-1, -1, t) for t in TILES_Y[1:]]
    ran = {B.ETC_PREC_FP64: 0, B.ETC_PREC_MIXED: 0, B.ETC_PREC_MIXED_F64: 0}
    for tiles in cands:
        monkeypatch.setenv("ETC_FORCE_TILES", ",".join(map(str, tiles)))
        for prec, tol in ((B.ETC_PREC_FP64, 1e-11), (B.ETC_PREC_MIXED, 2e-5),
                          (B.ETC_PREC_MIXED_F64, 2e-5)):
            try:
                B.etc_apply_preconditioner(rve.h, 2, prec, dev(r), z)
            except B.EtcError as e:  # this tile is not available for the shape
                assert e.status == B.ETC_EINVAL and "ETC_FORCE_TILES" in str(e)
                continue
            assert relmax(host(z), zo) < tol, (tiles, prec)
            ran[prec] += 1
        try:
            B.etc_dct_planes(rve.h, 2, 0, dev(r), out)
        except B.EtcError as e:
            assert e.status == B.ETC_EINVAL
            continue
        assert relmax(host(out), rhat) < 1e-12, tiles
        B.etc_dct_planes(rve.h, 2, 1, dev(rhat), out)
        assert relmax(host(out), r) < 1e-12, tiles
    # the register-resident kernels and at least the small tiles ran everywhere
    assert min(ran.values()) >= 6, ran


@pytest.mark.parametrize("shape,ku", [
    ((129, 5, 7), [0.7, 1.9, 3.1, 0.4, 2.2]),
    ((200, 6, 10), [0.7, 1.9, 3.1, 0.4, 2.2]),
    ((600, 4, 6), [0.7, 1.9, 3.1, 0.4, 2.2]),
    ((1030, 3, 4), [0.7, 1.9, 3.1, 0.4, 2.2]),
    # kappa_ref^x,y << kappa_ref^z: every column has a small shift
    # s/kappa_ref^z, whose pivots converge slowly along the loading axis
    ((1030, 8, 8), [1e-4, 3e-4, 3.0, 0.4, 2.2]),
    ((600, 6, 5), [1e-6, 1e-6, 2.0, 1e-3, 5.0]),
])
def test_preconditioner_long_loading_axis(shape, ku):
    # long tridiagonal systems (up to 1030 planes) in FP64 and FP32
    rng = np.random.default_rng(sum(shape))
    kx, ky, kz = (rng.uniform(0.2, 5.0, shape) for _ in range(3))
    rve = make(kx, ky, kz)
    rve.set_reference(2, B.ETC_REF_USER, ku)
    _, fshape = oracle_faces(kx, ky, kz, (1.0, 1.0, 1.0), 2)
    r = rng.standard_normal(fshape)
    zo = O.apply_reference_inverse(r, ku)
    z = torch.empty(fshape, dtype=torch.float64, device="cuda")
    B.etc_apply_preconditioner(rve.h, 2, B.ETC_PREC_FP64, dev(r), z)
    assert relmax(host(z), zo) < 1e-11
    B.etc_apply_preconditioner(rve.h, 2, B.ETC_PREC_MIXED, dev(r), z)
    assert relmax(host(z), zo) < 2e-5


@pytest.mark.parametrize("shape", [
    (1, 40, 36),    # one plane: the middle row alone
    (2, 40, 36),    # one chunk, no bottom chain
    (9, 24, 20),    # two chunks, the second partial
    (17, 12, 16),   # three chunks: one more on top than below
    (24, 8, 12),    # three full chunks
    (33, 8, 8),     # five chunks, the last one plane
    (65, 4, 8),
    (9, 320, 512),  # 1280 blocks of columns: the one-ended kernels
])
def test_fp32_tridiagonal_forms_match_oracle(shape):
    # Sec. 3.2 solves along the loading axis in FP32: grids that fit in one wave
    # run the two-ended elimination (middle plane m, back-substitution outward),
    # larger ones the one-ended sweeps; both against the oracle's Algorithm 3
    rng = np.random.default_rng(17 + sum(shape))
    kx, ky, kz = (rng.uniform(0.2, 5.0, shape) for _ in range(3))
    rve = make(kx, ky, kz)
    for ku in ([0.7, 1.9, 3.1, 0.4, 2.2], [1e-4, 3e-4, 3.0, 0.4, 2.2]):
        rve.set_reference(2, B.ETC_REF_USER, ku)
        r = rng.standard_normal(shape)
        zo = O.apply_reference_inverse(r, ku)
        z = torch.empty(shape, dtype=torch.float64, device="cuda")
        B.etc_apply_preconditioner(rve.h, 2, B.ETC_PREC_MIXED, dev(r), z)
        assert relmax(host(z), zo) < 2e-5, ku


# ------------------------------------------------------------------ end to end
def test_config_32_spheres_direction_x():
    # 32^3 two-phase random spheres (radius 3-5, fraction 0.3, 1:10), rtol 1e-10, load x
    k, info = M.random_spheres((32, 32, 32), (3, 5), 0.3, 1001, 1.0, 10.0)
    ref = O.solve_direction(k, k, k, 0, rtol=1e-10)
    rve = make(k)
    kap, inf = rve.solve(0, rtol=1e-10)
    assert abs(kap - ref.kappa_eff) <= 1e-9 * ref.kappa_eff
    assert abs(inf["iters"] - ref.iters) <= 1
    assert inf["status"] == B.ETC_OK and inf["relres"] <= 1e-10
    assert inf["true_relres"] < 1e-9
    np.testing.assert_allclose(inf["kref"], ref.kref, rtol=1e-13)
    p = host(rve.solution(0))
    assert relmax(p, ref.p) < 1e-8


@pytest.mark.parametrize("precision", [B.ETC_PREC_FP64, B.ETC_PREC_MIXED, B.ETC_PREC_MIXED_F64])
def test_energy_form_of_kappa_eff(precision):
    # the energy identity (outflow = inflow = energy value at the exact
    # solution): at convergence it equals the oracle's outflow value; its
    # error is quadratic in the solve error, so early iterates are far closer
    # to the converged value than the outflow value; the energy is minimal at
    # the solution, so it never falls below the converged value
    k, _ = M.random_spheres((40, 36, 48), (3, 6), 0.3, 5, 1.0, 1000.0)
    ref = O.solve_direction(k, k, k, 2, rtol=1e-12)
    rve = make(k)
    kc, ic = rve.solve(2, rtol=1e-12)
    assert abs(kc - ref.kappa_eff) <= 1e-10 * ref.kappa_eff
    assert abs(ic["kappa_energy"] - ref.kappa_eff) <= 1e-10 * ref.kappa_eff
    rtol = 1e-6 if precision == B.ETC_PREC_FP64 else 1e-5
    kr, ir = rve.solve(2, rtol=rtol, precision=precision)
    err_out = abs(kr - kc) / kc
    err_en = abs(ir["kappa_energy"] - kc) / kc
    assert err_out > 1e-9
    # quadratic in the error: at least 20 times closer (measured 84 times for
    # the mixed forms at rtol 1e-5, more for FP64)
    assert err_en <= max(1e-10, 0.05 * err_out), (err_out, err_en)
    # E(x) - E(x*) = ||x - x*||_A^2 >= 0 (against the converged energy value)
    assert ir["kappa_energy"] >= ic["kappa_energy"] * (1.0 - 1e-13)
    _, i0 = rve.solve(2, rtol=1e-8, precision=precision, true_residual=0)
    assert i0["kappa_energy"] == -1.0


def test_residual_history_of_a_capped_solve():
    # ETC_ENOCONV after maxit iterations: the history holds iterations 0..maxit,
    # its last value is the reported relres
    k, _ = M.random_spheres((24, 24, 24), (3, 5), 0.3, 9, 1.0, 1000.0)
    rve = make(k)
    st, kap, info = B.etc_solve_direction(rve.h, 2, 1.0, 0.0, B.make_opts(rtol=1e-12, maxit=7))
    assert st == B.ETC_ENOCONV and info.iters == 7
    first, hist = rve.history()
    assert first == 0 and len(hist) == 8 and hist[0] == 1.0
    assert hist[-1] == pytest.approx(info.relres, rel=1e-14) and hist[-1] > 1e-12


def test_linear_initial_guess_in_batches():
    # the batch forms honour the initial guess: homogeneous media end with 0
    # iterations, a random medium matches the one-solve value
    media = [np.full((32, 32, 32), 2.5), M.random_spheres((32, 32, 32), (2, 5), 0.3, 21, 1.0, 30.0)[0]]
    rves = [make(k) for k in media]
    for queue in (False, True):
        b = B.Batch(rves, rtol=1e-10, queue=queue, init=B.ETC_INIT_LINEAR)
        assert b.queued() == (2 if queue else 0)
        Ks, infos, _, st = b.run()
        b.close()
        assert st == B.ETC_OK
        assert all(infos[d]["iters"] == 0 for d in range(3))
        assert all(Ks[0][4 * d] == pytest.approx(2.5, rel=1e-12) for d in range(3))
        for d in range(3):
            kap, inf = rves[1].solve(d, rtol=1e-10, init=B.ETC_INIT_LINEAR)
            assert abs(Ks[1][4 * d] - kap) <= 1e-9 * kap
            assert abs(infos[3 + d]["iters"] - inf["iters"]) <= 1


@pytest.mark.parametrize("direction", [0, 2])
def test_linear_initial_guess_matches_oracle(direction):
    # x0 = p_in + (p_out - p_in)(k + 1/2)/n2 along the loading axis: the
    # oracle's Algorithm 1 started from the same guess (the exit test stays
    # relative to ||b||, Eq. exit)
    k, _ = M.random_spheres((24, 20, 28), (3, 5), 0.3, 1001, 1.0, 10.0)
    (k0, k1, k2), lens = O.permute_medium(k, k, k, (1.0, 1.0, 1.0), direction)
    f = O.face_conductances(k0, k1, k2, lens)
    kref = O.reference_parameters(O.group_extrema(f))
    b = O.right_hand_side(f, 2.0, -1.0)
    nz = k0.shape[0]
    prof = 2.0 + (-1.0 - 2.0) * (np.arange(nz) + 0.5) / nz
    p0 = np.ascontiguousarray(np.broadcast_to(prof[:, None, None], k0.shape))
    res = O.pcg(f, b, kref, rtol=1e-10, p0=p0)
    kap_o = O.outflow_etc(f, res.p, lens, 2.0, -1.0)
    rve = make(k)
    kap, inf = rve.solve(direction, p_in=2.0, p_out=-1.0, rtol=1e-10, init=B.ETC_INIT_LINEAR)
    assert inf["status"] == B.ETC_OK
    assert abs(kap - kap_o) <= 1e-9 * kap_o
    assert abs(inf["iters"] - res.iters) <= 1
    _, hist = rve.history()
    assert hist[0] == pytest.approx(res.history[0], rel=1e-12) and hist[0] < 1.0
    assert relmax(host(rve.solution(direction)), O.unpermute_field(res.p, direction)) < 1e-8
    # the mixed forms start from the same guess
    for prec in (B.ETC_PREC_MIXED, B.ETC_PREC_MIXED_F64):
        km, im = rve.solve(direction, p_in=2.0, p_out=-1.0, rtol=1e-9, precision=prec,
                           init=B.ETC_INIT_LINEAR)
        assert im["status"] == B.ETC_OK and abs(km - kap_o) <= 1e-6 * kap_o


def test_linear_initial_guess_homogeneous_zero_iterations():
    # the guess is the solution of a homogeneous medium: no iteration at all
    shape = (10, 12, 14)
    comps = (np.full(shape, 2.0), np.full(shape, 3.5), np.full(shape, 0.7))
    rve = make(*comps)
    for prec in (B.ETC_PREC_FP64, B.ETC_PREC_MIXED, B.ETC_PREC_MIXED_F64):
        for d in range(3):
            kap, inf = rve.solve(d, p_in=2.0, p_out=-1.0, rtol=1e-12, precision=prec,
                                 init=B.ETC_INIT_LINEAR)
            assert inf["status"] == B.ETC_OK and inf["iters"] == 0
            assert kap == pytest.approx(comps[d][0, 0, 0], rel=1e-12)


def test_residual_history_matches_oracle():
    # ||r_i|| / ||b|| after every iteration (the convergence histories of
    # Sec. 4.2) against the oracle's Algorithm 1 on the same input
    k, _ = M.random_spheres((32, 32, 32), (3, 5), 0.3, 1001, 1.0, 10.0)
    (k0, k1, k2), lens = O.permute_medium(k, k, k, (1.0, 1.0, 1.0), 0)
    f = O.face_conductances(k0, k1, k2, lens)
    res = O.pcg(f, O.right_hand_side(f, 1.0, 0.0), O.reference_parameters(O.group_extrema(f)),
                rtol=1e-10)
    rve = make(k)
    kap, inf = rve.solve(0, rtol=1e-10)
    first, hist = rve.history()
    assert first == 0 and len(hist) == inf["iters"] + 1 == len(res.history)
    assert hist[0] == 1.0 and hist[-1] == pytest.approx(inf["relres"], rel=1e-14)
    np.testing.assert_allclose(hist, res.history, rtol=1e-6)
    # a short window: the last five iterations
    first5, hist5 = rve.history(cap=5)
    assert first5 == inf["iters"] - 4 and hist5 == hist[-5:]
    # the mixed path records its own iterations
    _, inf_m = rve.solve(0, rtol=1e-8, precision=B.ETC_PREC_MIXED)
    first_m, hist_m = rve.history()
    assert first_m == 0 and len(hist_m) == inf_m["iters"] + 1
    assert hist_m[-1] == pytest.approx(inf_m["relres"], rel=1e-14) and hist_m[-1] <= 1e-8


@pytest.mark.parametrize("shape", [(18, 20, 24), (11, 13, 17), (1, 6, 4), (7, 1, 9), (1, 1, 5),
                                   (6, 1, 1), (1, 1, 1)])
def test_tensor_matches_oracle(shape):
    rng = np.random.default_rng(sum(shape) * 3 + 1)
    kx = M.two_phase_random(shape, seed=sum(shape), fraction=0.35, kappa_inclusion=20.0)
    ky, kz = kx * rng.uniform(0.5, 2.0, shape), kx * rng.uniform(0.5, 2.0, shape)
    lengths = (1.0, 0.8, 1.5)
    # both sides solved to 1e-12, so that the comparison measures the
    # implementations and not where each stopped inside the 1e-10 ball
    K_o, res_o = O.effective_tensor(kx, ky, kz, lengths, rtol=1e-12)
    rve = make(kx, ky, kz, lengths)
    K, infos, st = rve.tensor(rtol=1e-12)
    K = np.array(K).reshape(3, 3)
    assert st == B.ETC_OK
    np.testing.assert_allclose(np.diag(K), np.diag(K_o), rtol=1e-10)
    assert np.abs(K - K_o).max() <= 1e-10 * np.abs(K_o).max()
    for d in range(3):
        assert abs(infos[d]["iters"] - res_o[d].iters) <= 1
        assert abs(infos[d]["kappa_in"] - res_o[d].kappa_eff) <= 1e-8 * res_o[d].kappa_eff


@pytest.mark.parametrize("ny,lengths", [(1, (1.0, 1.0, 1.0)), (3, (2.0, 0.5, 1.0))])
def test_checkerboard_off_diagonal_closed_form(ny, lengths):
    # 2 x 2 checkerboard [[a, b], [b, a]] in the x-z plane: nonzero K[x][z]
    # and K[z][x], solved by hand (half-turn symmetry, 2 x 2 system)
    a, b = 3.0, 0.7
    k = np.empty((2, ny, 2))
    k[0, :, 0], k[0, :, 1], k[1, :, 0], k[1, :, 1] = a, b, b, a
    lx, _, lz = lengths
    rve = make(k, lengths=lengths)
    K, _, st = rve.tensor(rtol=1e-12)
    K = np.array(K).reshape(3, 3)
    assert st == B.ETC_OK
    kxz, kzz = checkerboard_closed_form(a, b, lx, lz)
    kzx, kxx = checkerboard_closed_form(a, b, lz, lx)
    np.testing.assert_allclose([K[0, 2], K[2, 2], K[2, 0], K[0, 0], K[1, 1]],
                               [kxz, kzz, kzx, kxx, 0.5 * (a + b)], rtol=1e-10)
    assert max(abs(K[0, 1]), abs(K[1, 0]), abs(K[1, 2]), abs(K[2, 1])) < 1e-12


def test_homogeneous_one_iteration_exact():
    shape = (10, 12, 14)
    comps = (np.full(shape, 2.0), np.full(shape, 3.5), np.full(shape, 0.7))
    rve = make(*comps)
    for d in range(3):
        kap, inf = rve.solve(d, p_in=2.0, p_out=-1.0, rtol=1e-12)
        assert inf["iters"] == 1
        assert kap == pytest.approx(comps[d][0, 0, 0], rel=1e-12)


def test_series_laminate_harmonic_mean():
    vals = [1.0, 10.0, 3.0, 0.2, 7.0]
    k = M.series_laminate((20, 12, 11), vals, 2)
    rve = make(k)
    kap, inf = rve.solve(2, rtol=1e-12)
    layer = [vals[l % len(vals)] for l in range(20)]
    assert kap == pytest.approx(20 / sum(1 / v for v in layer), rel=1e-10)


@pytest.mark.parametrize("shape", [
    (40, 36, 48),  # loading axis 40 planes: whole chunks of the tridiagonal copies
    (37, 20, 22),  # 37 planes (a partial last chunk), plane 440 (a partial block of columns)
    (9, 12, 14),   # fewer planes than one chunk plus one, small tiles
])
@pytest.mark.parametrize("precision", [B.ETC_PREC_MIXED, B.ETC_PREC_MIXED_F64])
def test_mixed_precision_matches_fp64_oracle(precision, shape):
    # arrays are [z][y][x]: loading along z puts x (even here) on axis 0, so
    # both bulk-tensor kernels (matvec and tridiagonal) run
    k, _ = M.random_spheres(shape, (3, 6), 0.3, 77, 1.0, 100.0)
    ref = O.solve_direction(k, k, k, 2, rtol=1e-10)
    rve = make(k)
    kap, inf = rve.solve(2, rtol=1e-8, precision=precision)
    assert inf["status"] == B.ETC_OK
    assert abs(kap - ref.kappa_eff) <= 1e-6 * ref.kappa_eff
    assert inf["true_relres"] < 1e-7
    # the solution field too (each form returns x in FP64)
    p = host(rve.solution(2))
    assert relmax(p, ref.p) < 1e-5


def test_solution_unpermuted_each_direction():
    shape = (9, 10, 11)
    rng = np.random.default_rng(5)
    kx, ky, kz = (rng.uniform(0.5, 4.0, shape) for _ in range(3))
    rve = make(kx, ky, kz)
    for d in range(3):
        rve.solve(d, rtol=1e-11)
        ref = O.solve_direction(kx, ky, kz, d, rtol=1e-11)
        assert relmax(host(rve.solution(d)), ref.p) < 1e-8
        host_out = np.empty(shape)
        B.etc_get_solution(rve.h, d, host_out)
        assert relmax(host_out, ref.p) < 1e-8


# ------------------------------------------------------------------ errors & limits
def test_invalid_arguments():
    k = np.ones((4, 4, 4))
    rve = make(k)
    with pytest.raises(B.EtcError) as e:
        rve.solve(2, p_in=1.0, p_out=1.0)
    assert e.value.status == B.ETC_EINVAL
    with pytest.raises(B.EtcError):
        rve.solve(3)
    with pytest.raises(B.EtcError):
        rve.solve(0, rtol=-1.0)
    bad = k.copy(); bad[1, 2, 3] = 0.0
    with pytest.raises(B.EtcError) as e:
        make(bad)
    assert e.value.status == B.ETC_EINVAL
    bad[1, 2, 3] = np.nan
    with pytest.raises(B.EtcError):
        make(bad)
    with pytest.raises(B.EtcError) as e:
        B.etc_get_solution(rve.h, 1, torch.empty((4, 4, 4), dtype=torch.float64, device="cuda"))
    assert e.value.status == B.ETC_ESTATE


def test_maxit_reports_noconv_with_info():
    k, _ = M.random_spheres((24, 24, 24), (3, 5), 0.3, 9, 1.0, 1000.0)
    rve = make(k)
    opts = B.make_opts(rtol=1e-12, maxit=3)
    st, kap, info = B.etc_solve_direction(rve.h, 2, 1.0, 0.0, opts)
    assert st == B.ETC_ENOCONV
    assert info.iters == 3 and info.status == B.ETC_ENOCONV
    assert np.isfinite(kap) and kap > 0 and info.relres > 1e-12


@pytest.mark.parametrize("precision", [B.ETC_PREC_FP64, B.ETC_PREC_MIXED, B.ETC_PREC_MIXED_F64])
def test_deterministic_bitwise(precision):
    # fixed-order reductions, no float atomics: repeated solves are identical
    # (the mixed forms run the bulk-tensor matvec and tridiagonal kernels)
    k, _ = M.random_spheres((32, 32, 32), (3, 5), 0.3, 1001, 1.0, 10.0)
    rve = make(k)
    rtol = 1e-10 if precision == B.ETC_PREC_FP64 else 1e-8
    a, ia = rve.solve(1, rtol=rtol, precision=precision)
    pa = host(rve.solution(1)).copy()
    rve.solve(2, rtol=rtol, precision=precision)  # another frame in between
    b, ib = rve.solve(1, rtol=rtol, precision=precision)
    pb = host(rve.solution(1))
    assert a == b and ia["iters"] == ib["iters"]
    assert np.array_equal(pa, pb)


def test_host_pointer_input_equals_device_input():
    k, _ = M.random_spheres((20, 22, 24), (3, 5), 0.3, 3, 1.0, 10.0)
    h = B.etc_create_rve(24, 22, 20, 1.0, 1.0, 1.0, np.ascontiguousarray(k),
                         stream=torch.cuda.current_stream().cuda_stream)
    try:
        st, kap_h, _ = B.etc_solve_direction(h, 2, 1.0, 0.0, B.make_opts(rtol=1e-10))
    finally:
        B.etc_destroy_rve(h)
    kap_d, _ = make(k).solve(2, rtol=1e-10)
    assert kap_h == kap_d


# ------------------------------------------------------------------ conversions
def test_integer_pipe_conversions_are_exact():
    # widen: every binary32 pattern class (normal, subnormal, zero, inf, nan);
    # narrow: round to nearest even as IEEE-754 (numpy's float64 -> float32).
    rng = np.random.default_rng(42)
    bits32 = rng.integers(0, 2**32, 200_000, dtype=np.uint64).astype(np.uint32)
    special32 = np.array([0, 0x80000000, 1, 0x80000001, 0x7FFFFF, 0x800000, 0x7F7FFFFF,
                          0x7F800000, 0xFF800000, 0x3F800000, 0x00400000], dtype=np.uint32)
    f = np.concatenate([bits32, special32]).view(np.float32)
    bits64 = rng.integers(0, 2**63, f.size, dtype=np.uint64) | (
        rng.integers(0, 2, f.size, dtype=np.uint64) << np.uint64(63))
    d = bits64.view(np.float64).copy()
    # values near the binary32 range edges, ties, and subnormal results
    m = 20000
    d[:m] = rng.uniform(-1, 1, m) * np.exp2(rng.integers(-160, 130, m)).astype(np.float64)
    ties = (np.arange(1, 1001, dtype=np.float64) + 0.5) * 2.0 ** -23  # exact ties at 1..2
    d[m:m + ties.size] = 1.0 + ties
    d[-6:] = [0.0, -0.0, np.inf, -np.inf, 3.4028235677973366e38, 1e-46]
    fi, di = torch.from_numpy(f).cuda(), torch.from_numpy(d).cuda()
    do = torch.empty_like(di)
    fo = torch.empty_like(fi)
    B.etc_convert_check(fi, do, di, fo, torch.cuda.current_stream().cuda_stream)
    ref_w = f.astype(np.float64)
    got_w = host(do)
    nan = np.isnan(ref_w)
    assert np.array_equal(np.isnan(got_w), nan)
    assert np.array_equal(got_w[~nan].view(np.uint64), ref_w[~nan].view(np.uint64))
    with np.errstate(over="ignore"):
        ref_n = d.astype(np.float32)
    got_n = fo.cpu().numpy()
    nan = np.isnan(ref_n)
    assert np.array_equal(np.isnan(got_n), nan)
    assert np.array_equal(got_n[~nan].view(np.uint32), ref_n[~nan].view(np.uint32))


def test_double_float_split_is_exact():
    # hi = RN32(d), lo = RN32(d - hi) for the mixed matvec; lo = 0 below 2^-74
    # and where hi is not finite.
    rng = np.random.default_rng(7)
    m = 200_000
    d = rng.uniform(-1, 1, m) * np.exp2(rng.integers(-140, 140, m)).astype(np.float64)
    d[:1000] = 1.0 + (np.arange(1000) + 0.5) * 2.0 ** -23       # ties of hi
    d[1000:2000] = 1.0 + (np.arange(1000) + 0.25) * 2.0 ** -23   # remainders of both signs
    d[2000:2008] = [0.0, -0.0, np.inf, -np.inf, np.nan, 2.0 ** -74, 2.0 ** -75,
                    np.nextafter(2.0 ** 128, 0.0)]
    di = torch.from_numpy(d).cuda()
    hilo = torch.empty(2 * m, dtype=torch.float32, device="cuda")
    B.etc_split_check(di, hilo, torch.cuda.current_stream().cuda_stream)
    got = hilo.cpu().numpy().reshape(m, 2)
    with np.errstate(over="ignore", invalid="ignore"):
        hi = d.astype(np.float32)
        ok = np.isfinite(hi) & (np.abs(d) >= 2.0 ** -74)
        lo = np.where(ok, (d - hi.astype(np.float64)).astype(np.float32), np.float32(0))
    nan = np.isnan(hi)
    assert np.array_equal(np.isnan(got[:, 0]), nan)
    assert np.array_equal(got[~nan, 0].view(np.uint32), hi[~nan].view(np.uint32))
    assert np.array_equal(np.abs(got[:, 1]).view(np.uint32), np.abs(lo).view(np.uint32))
    assert np.array_equal(np.signbit(got[ok, 1]) | (got[ok, 1] == 0),
                          np.signbit(lo[ok]) | (lo[ok] == 0))
    # hi + lo carries 48 significant bits
    sel = ok & (d != 0)
    err = np.abs(got[sel, 0].astype(np.float64) + got[sel, 1] - d[sel]) / np.abs(d[sel])
    assert err.max() <= 2.0 ** -47


def test_bulk_copy_wait_runs_out_reports_ecuda_and_recovers():
    # ETC_TEST_TMA_TX_EXTRA=16 (read at create): every stage of the
    # bulk-tensor matvec expects 16 bytes that no copy delivers, so its bounded
    # waits (0.5 s) run out; no fault is involved.  The solve must end with
    # ETC_ECUDA and a message, and a new handle must solve normally.
    import os
    k, _ = M.random_spheres((16, 16, 32), (2, 4), 0.3, 5, 1.0, 10.0)
    os.environ["ETC_TEST_TMA_TX_EXTRA"] = "16"
    try:
        rve = make(k)
    finally:
        os.environ.pop("ETC_TEST_TMA_TX_EXTRA", None)
    with pytest.raises(B.EtcError) as e:
        rve.solve(2, rtol=1e-8, precision=B.ETC_PREC_MIXED)
    assert e.value.status == B.ETC_ECUDA and "wait for bulk-tensor copies ran out" in str(e.value)
    rve.close()
    rve2 = make(k)
    kap_m, info = rve2.solve(2, rtol=1e-8, precision=B.ETC_PREC_MIXED)
    kap_d, _ = rve2.solve(2, rtol=1e-10)
    assert info["status"] == B.ETC_OK and abs(kap_m - kap_d) <= 1e-6 * kap_d


def test_allocation_failure_reports_enomem_and_recovers():
    # ETC_FAIL_ALLOC_AFTER=k: the (k+1)-th device allocation of a handle fails;
    # creation must report ETC_ENOMEM and release what it took, and the next
    # handle must work
    import os
    k = np.ones((8, 8, 8))
    try:
        for budget in (0, 1, 5, 12, 20):
            os.environ["ETC_FAIL_ALLOC_AFTER"] = str(budget)
            with pytest.raises(B.EtcError) as e:
                make(k)
            assert e.value.status == B.ETC_ENOMEM
    finally:
        os.environ.pop("ETC_FAIL_ALLOC_AFTER", None)
    rve = make(k)
    kap, info = rve.solve(2, rtol=1e-12)
    assert kap == pytest.approx(1.0, rel=1e-12) and info["iters"] <= 2
