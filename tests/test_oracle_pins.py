"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle function to something other than itself: a library
routine for a special case, a closed form, an exact physical identity of the
discrete resistor network, an invariance, or a value printed in the paper.
"""
import math
import os

import numpy as np
import pytest
import scipy.fft

from oracle import etc_oracle as O
from paper_2404_02433_b300 import microstructure as M
from closed_forms import checkerboard_closed_form

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- DCT pins
@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 12, 17, 32])
def test_dct_forward_matches_scipy_type2(n):
    # Eq. (forward DCT) is half of SciPy's unnormalised DCT-II.
    u = np.random.default_rng(n).standard_normal((3, n))
    ours = O.dct_forward(u, 1)
    ref = scipy.fft.dct(u, type=2, axis=1) / 2.0
    np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-12 * max(1, n))


@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_dct_backward_inverts_forward(n):
    # Eq. (backward DCT) with 2/N and alpha_0 = 1/2 is the inverse of Eq. (forward DCT).
    u = np.random.default_rng(100 + n).standard_normal((n, 4))
    np.testing.assert_allclose(O.dct_backward(O.dct_forward(u, 0), 0), u, atol=1e-13)
    np.testing.assert_allclose(O.dct_forward(O.dct_backward(u, 0), 0), u, atol=1e-12 * n)


@pytest.mark.parametrize("n", [2, 5, 9, 16])
def test_neumann_eigenpairs(n):
    # Sec. 3.2: A v^k = 2(1 - cos(k pi/N)) v^k for the 1-D Neumann matrix, with
    # v^k.v^k = N/2 (k > 0) and N (k = 0).
    A = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    A[0, 0] = A[-1, -1] = 1.0
    for k in range(n):
        e = np.zeros(n); e[k] = 1.0
        v = O.dct_backward(e, 0)  # proportional to the cosine basis vector v^k
        lam = 2.0 * (1.0 - math.cos(k * math.pi / n))
        np.testing.assert_allclose(A @ v, lam * v, atol=1e-13)
        assert O.neumann_eigenvalue(k, n) == pytest.approx(lam, abs=1e-13)
        vk = np.cos(np.pi * (2 * np.arange(n) + 1) * k / (2 * n))
        assert vk @ vk == pytest.approx(n if k == 0 else n / 2)
        # forward transform of v^k is (v^k.v^k) e_k by orthogonality
        np.testing.assert_allclose(O.dct_forward(vk, 0), (vk @ vk) * e, atol=1e-12)


# ---------------------------------------------------------------- thomas / preconditioner
def test_thomas_matches_dense_solve():
    rng = np.random.default_rng(3)
    n, m = 9, 4
    sub = -rng.uniform(0.5, 1.0, (n - 1, m)); sup = sub.copy()
    diag = 3.0 + rng.uniform(0, 1, (n, m))
    rhs = rng.standard_normal((n, m))
    x = O.thomas(sub, diag, sup, rhs)
    for c in range(m):
        T = np.diag(diag[:, c]) + np.diag(sub[:, c], -1) + np.diag(sup[:, c], 1)
        np.testing.assert_allclose(x[:, c], np.linalg.solve(T, rhs[:, c]), atol=1e-13)


@pytest.mark.parametrize("shape", [(5, 4, 6), (1, 3, 2), (4, 1, 1), (7, 6, 5), (2, 2, 2)])
def test_reference_inverse_solves_reference_operator(shape):
    # Algorithm 3 output z must satisfy A_ref z = r, with A_ref applied as the
    # homogeneous form of Eq. (refer bilinear forms) -- a different code path.
    rng = np.random.default_rng(sum(shape))
    kref = list(rng.uniform(0.3, 3.0, 5))
    r = rng.standard_normal(shape)
    z = O.apply_reference_inverse(r, kref)
    back = O.apply_operator(O.reference_operator_faces(kref, shape), z)
    np.testing.assert_allclose(back, r, atol=1e-11 * np.abs(r).max())


# ---------------------------------------------------------------- operator / PCG
def _dense(f, shape):
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n); e[c] = 1.0
        A[:, c] = O.apply_operator(f, e.reshape(shape)).ravel()
    return A


def _assembled(f, shape):
    # Element-by-face assembly of the same bilinear form: each internal face
    # adds t [[1,-1],[-1,1]] to its two cells; Dirichlet faces add to one cell.
    nz, ny, nx = shape
    idx = np.arange(nz * ny * nx).reshape(shape)
    A = np.zeros((idx.size, idx.size))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = idx[k, j, i]
                for t, nb in ((f.t0[k, j, i], (k, j, i - 1)), (f.t1[k, j, i], (k, j - 1, i)),
                              (f.t2[k, j, i], (k - 1, j, i))):
                    if min(nb) < 0:
                        continue
                    o = idx[nb]
                    A[c, c] += t; A[o, o] += t; A[c, o] -= t; A[o, c] -= t
                if k == 0:
                    A[c, c] += f.b_in[j, i]
                if k == nz - 1:
                    A[c, c] += f.b_out[j, i]
    return A


@pytest.mark.parametrize("shape", [(3, 4, 5), (1, 1, 4), (4, 1, 1), (2, 3, 1)])
def test_operator_symmetric_positive_definite_and_assembled(shape):
    rng = np.random.default_rng(7)
    kx, ky, kz = (rng.uniform(0.2, 5.0, shape) for _ in range(3))
    f = O.face_conductances(kx, ky, kz, (1.0, 2.0, 0.5))
    A = _dense(f, shape)
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    np.testing.assert_allclose(A, _assembled(f, shape), atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("direction", [0, 1, 2])
def test_pcg_reaches_dense_solution(direction):
    shape = (4, 3, 5)
    rng = np.random.default_rng(11 + direction)
    kx, ky, kz = (rng.uniform(0.1, 10.0, shape) for _ in range(3))
    (k0, k1, k2), lens = O.permute_medium(kx, ky, kz, (1.0, 1.5, 0.8), direction)
    f = O.face_conductances(k0, k1, k2, lens)
    b = O.right_hand_side(f, 2.0, -1.0)
    A = _dense(f, k0.shape)
    exact = np.linalg.solve(A, b.ravel()).reshape(k0.shape)
    kref = O.reference_parameters(O.group_extrema(f))
    res = O.pcg(f, b, kref, rtol=1e-13)
    assert res.converged
    np.testing.assert_allclose(res.p, exact, atol=1e-11)


# ---------------------------------------------------------------- physics closed forms
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_homogeneous_anisotropic_exact(direction):
    # Homogeneous medium: A_ref = A for the LP parameters, so PCG converges in
    # one iteration; the exact TPFA solution is linear and kappa_eff equals the
    # loading-axis component.
    shape = (6, 5, 7)
    comps = (np.full(shape, 2.0), np.full(shape, 3.5), np.full(shape, 0.7))
    r = O.solve_direction(*comps, direction, (1.0, 1.0, 1.0), p_in=3.0, p_out=1.0, rtol=1e-12)
    assert r.iters == 1
    assert r.kappa_eff == pytest.approx(comps[direction][0, 0, 0], rel=1e-12)
    n = shape[2 - direction]
    prof = 3.0 + (1.0 - 3.0) * (np.arange(n) + 0.5) / n
    view = [1, 1, 1]; view[2 - direction] = n
    np.testing.assert_allclose(r.p, np.broadcast_to(prof.reshape(view), shape), atol=1e-12)
    off = [a for a in range(3) if a != direction]
    np.testing.assert_allclose(r.column[off], 0.0, atol=1e-12)


def test_series_laminate_is_harmonic_mean():
    # Layers normal to the load: TPFA is a chain of resistors h/kappa_l, so the
    # effective value is exactly the harmonic mean of the layer values.
    vals = [1.0, 10.0, 3.0, 0.2, 7.0]
    for axis in range(3):
        k = M.series_laminate((10, 12, 11), vals, axis)
        n = k.shape[2 - axis]
        layer = [vals[l % len(vals)] for l in range(n)]
        r = O.solve_direction(k, k, k, axis, rtol=1e-13)
        assert r.kappa_eff == pytest.approx(n / sum(1.0 / v for v in layer), rel=1e-11)


def test_parallel_laminate_is_arithmetic_mean():
    # Layers parallel to the load: independent straight columns, exact
    # arithmetic mean, zero transverse mean flux.
    vals = [1.0, 10.0, 3.0, 0.2]
    k = M.series_laminate((9, 10, 8), vals, 0)  # varies along x
    for d in (1, 2):
        r = O.solve_direction(k, k, k, d, rtol=1e-13)
        layer = [vals[l % len(vals)] for l in range(8)]
        assert r.kappa_eff == pytest.approx(sum(layer) / 8, rel=1e-11)
        np.testing.assert_allclose(r.column[[a for a in range(3) if a != d]], 0.0, atol=1e-11)


def test_voigt_reuss_bounds_and_conservation():
    k = M.two_phase_random((10, 9, 8), seed=5, fraction=0.35, kappa_inclusion=50.0)
    r = O.solve_direction(k, k, k, 2, rtol=1e-13)
    voigt = k.mean()
    reuss = 1.0 / (1.0 / k).mean()
    assert reuss < r.kappa_eff < voigt
    # conservation: the same total flux crosses every plane of z faces
    (k0, k1, k2), lens = O.permute_medium(k, k, k, (1.0, 1.0, 1.0), 2)
    f = O.face_conductances(k0, k1, k2, lens)
    fl = O.plane_fluxes(f, r.p, lens, 1.0, 0.0)
    np.testing.assert_allclose(fl, fl[-1], rtol=1e-9)
    # inflow, outflow and energy formulas agree at convergence
    b = O.right_hand_side(f, 1.0, 0.0)
    assert O.inflow_etc(f, r.p, lens, 1.0, 0.0) == pytest.approx(r.kappa_eff, rel=1e-9)
    assert O.energy_etc(f, r.p, b, lens, 1.0, 0.0) == pytest.approx(r.kappa_eff, rel=1e-11)


def test_invariances():
    rng = np.random.default_rng(21)
    shape = (7, 6, 5)
    kx, ky, kz = (rng.uniform(0.5, 8.0, shape) for _ in range(3))
    K, _ = O.effective_tensor(kx, ky, kz, rtol=1e-12)
    # scaling kappa -> c kappa scales K
    K2, _ = O.effective_tensor(3.0 * kx, 3.0 * ky, 3.0 * kz, rtol=1e-12)
    np.testing.assert_allclose(K2, 3.0 * K, rtol=1e-9)
    # swapping the physical x and y axes of the medium swaps rows/cols of K
    sw = lambda a: np.ascontiguousarray(np.swapaxes(a, 1, 2))
    K3, _ = O.effective_tensor(sw(ky), sw(kx), sw(kz), rtol=1e-12)
    P = np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1]])
    np.testing.assert_allclose(K3, P @ K @ P.T, rtol=1e-8, atol=1e-10)
    # reflecting along the load with p_in <-> p_out leaves kappa_eff unchanged
    r1 = O.solve_direction(kx, ky, kz, 2, p_in=1.0, p_out=0.0, rtol=1e-12)
    fl = lambda a: np.ascontiguousarray(a[::-1])
    r2 = O.solve_direction(fl(kx), fl(ky), fl(kz), 2, p_in=0.0, p_out=1.0, rtol=1e-12)
    assert r2.kappa_eff == pytest.approx(r1.kappa_eff, rel=1e-9)
    # independent of the pressure drop and of a common shift
    r3 = O.solve_direction(kx, ky, kz, 2, p_in=7.0, p_out=2.5, rtol=1e-12)
    assert r3.kappa_eff == pytest.approx(r1.kappa_eff, rel=1e-9)


def test_mirror_symmetric_medium_has_zero_off_diagonals():
    k = M.centre_ball(12, 20.0)
    K, _ = O.effective_tensor(k, rtol=1e-12)
    np.testing.assert_allclose(K - np.diag(np.diag(K)), 0.0, atol=1e-10)
    np.testing.assert_allclose(np.diag(K), K[0, 0], rtol=1e-10)


@pytest.mark.parametrize("ny,lengths", [(1, (1.0, 1.0, 1.0)), (3, (2.0, 0.5, 1.0)),
                                        (2, (0.5, 1.0, 3.0))])
def test_checkerboard_off_diagonal_closed_form(ny, lengths):
    """Off-diagonal entries pinned to a hand-solved network (nonzero values).

    The medium has no mirror symmetry in x alone, so K[x][z] != 0.  Its value
    and sign, the h factors of a non-cubic box and the loading-frame
    permutation are all fixed by ``checkerboard_closed_form``; load x is the
    same checkerboard with the roles of x and z (and of L^x, L^z) swapped, and
    load y sees four identical parallel columns (arithmetic mean).
    """
    a, b = 3.0, 0.7
    k = np.empty((2, ny, 2))
    k[0, :, 0], k[0, :, 1], k[1, :, 0], k[1, :, 1] = a, b, b, a
    lx, ly, lz = lengths
    K, _ = O.effective_tensor(k, lengths=lengths, rtol=1e-13)
    kxz, kzz = checkerboard_closed_form(a, b, lx, lz)
    kzx, kxx = checkerboard_closed_form(a, b, lz, lx)
    assert abs(kxz) > 0.05
    np.testing.assert_allclose(K[0, 2], kxz, rtol=1e-10)
    np.testing.assert_allclose(K[2, 2], kzz, rtol=1e-10)
    np.testing.assert_allclose(K[2, 0], kzx, rtol=1e-10)
    np.testing.assert_allclose(K[0, 0], kxx, rtol=1e-10)
    np.testing.assert_allclose(K[1, 1], 0.5 * (a + b), rtol=1e-10)
    for i, j in ((0, 1), (1, 0), (1, 2), (2, 1)):
        assert abs(K[i, j]) < 1e-12


# ---------------------------------------------------------------- LP (Algorithm 2)
def test_centred_lp_point_is_optimal():
    rng = np.random.default_rng(4)
    for _ in range(20):
        ext = []
        for g in range(5):
            lo = math.exp(rng.uniform(-3, 3))
            ext.append((lo, lo * math.exp(rng.uniform(0, 4))))
        kc = O.reference_parameters(ext, "centred")
        kl = O.reference_parameters(ext, "linprog")
        # both optimal: the same Lambda''/Lambda' = max_g max/min
        best = max(hi / lo for lo, hi in ext)
        assert O.condition_bound(ext, kc) == pytest.approx(best, rel=1e-9)
        assert O.condition_bound(ext, kl) == pytest.approx(best, rel=1e-6)


def test_lp_brute_force_tiny():
    # 2 groups: a grid search over c_1 - c_0 cannot beat the closed form.
    ext = [(1.0, 4.0), (0.5, 8.0), None, (2.0, 3.0), (1.0, 1.0)]
    best = O.condition_bound(ext, O.reference_parameters(ext, "centred"))
    for t in np.linspace(-4, 4, 801):
        for u in np.linspace(-3, 3, 61):
            kref = [1.0, math.exp(t), 1.0, math.exp(u), 1.0]
            assert O.condition_bound(ext, kref) >= best * (1 - 1e-12)


def _brute_extrema(kx, ky, kz, lengths):
    # face by face: harmonic mean of kappa~ = kappa / h^2 of the two cells, over
    # internal faces of each axis; kappa~^z on the first and last z plane
    nz, ny, nx = kx.shape
    h = (lengths[0] / nx, lengths[1] / ny, lengths[2] / nz)
    groups = [[], [], [], [], []]
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for g, (comp, nb) in enumerate(((kx, (k, j, i + 1)), (ky, (k, j + 1, i)),
                                                (kz, (k + 1, j, i)))):
                    if nb[0] < nz and nb[1] < ny and nb[2] < nx:
                        a = comp[k, j, i] / h[g] ** 2
                        b = comp[nb] / h[g] ** 2
                        groups[g].append(2.0 / (1.0 / a + 1.0 / b))
                if k == 0:
                    groups[3].append(kz[k, j, i] / h[2] ** 2)
                if k == nz - 1:
                    groups[4].append(kz[k, j, i] / h[2] ** 2)
    return [(min(v), max(v)) if v else None for v in groups]


def _dense_of(f, shape):
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n); e[c] = 1.0
        A[:, c] = O.apply_operator(f, e.reshape(shape)).ravel()
    return A


@pytest.mark.parametrize("seed", [3, 11, 20, 38])
def test_lemma_3_1_spectral_bounds(seed):
    # Lemma 3.1: Lambda' <= p.Ap / p.A_ref p <= Lambda'' for every p, with
    # Lambda' = min_g min_g/kappa_ref^g and Lambda'' = max_g max_g/kappa_ref^g,
    # so every generalised eigenvalue of (A, A_ref) lies in [Lambda', Lambda''].
    import scipy.linalg
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in rng.integers(2, 5, 3))
    kx, ky, kz = (np.exp(rng.uniform(-2.0, 2.0, shape)) for _ in range(3))
    lengths = tuple(rng.uniform(0.5, 2.0, 3))
    f = O.face_conductances(kx, ky, kz, lengths)
    ext = O.group_extrema(f)
    np.testing.assert_allclose(np.array(ext), np.array(_brute_extrema(kx, ky, kz, lengths)),
                               rtol=1e-14)
    A = _dense_of(f, shape)
    for method in ("centred", "linprog"):
        kref = O.reference_parameters(ext, method)
        ev = scipy.linalg.eigh(A, _dense_of(O.reference_operator_faces(kref, shape), shape),
                               eigvals_only=True)
        lo = min(e[0] / k for e, k in zip(ext, kref))
        hi = max(e[1] / k for e, k in zip(ext, kref))
        assert ev.min() >= lo * (1 - 1e-10) and ev.max() <= hi * (1 + 1e-10)
        assert O.condition_bound(ext, kref) == pytest.approx(hi / lo, rel=1e-14)
        if seed == 20 and method == "centred":
            # the bound as printed (out group divided by kappa_ref^in) does not hold
            lo_p = min([e[0] / k for e, k in zip(ext[:4], kref[:4])] + [ext[4][0] / kref[3]])
            assert ev.min() < lo_p * (1 - 1e-6)


# ---------------------------------------------------------------- the paper's numbers
def _table3():
    rows = []
    with open(os.path.join(GOLDEN, "table3_centre_ball_512.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows.append((float(v[0]), float(v[1]), [int(x) for x in v[2:]]))
    return rows


@pytest.mark.slow
@pytest.mark.parametrize("row", _table3(), ids=lambda r: f"kinc{r[0]:g}")
def test_table3_centre_ball_512(row):
    # Table 3: kappa_eff^z to four significant digits at 512^3 (rtol 1e-5 suffices).
    kinc, expect, _ = row
    k = M.centre_ball(512, kinc)
    r = O.solve_direction(k, k, k, 2, rtol=1e-5)
    assert abs(r.kappa_eff - expect) <= 5e-4


# ---------------------------------------------------------------- planted mistakes
def test_planted_arithmetic_face_mean_breaks_series_pin(monkeypatch):
    monkeypatch.setattr(O, "harmonic_face", lambda a, b: 0.5 * (a + b))
    k = M.series_laminate((6, 5, 8), [1.0, 10.0], 2)
    r = O.solve_direction(k, k, k, 2, rtol=1e-12)
    assert abs(r.kappa_eff - 8 / (4 / 1.0 + 4 / 10.0)) > 1e-3


def test_planted_eigenvalue_error_breaks_preconditioner_pin(monkeypatch):
    monkeypatch.setattr(O, "neumann_eigenvalue",
                        lambda kp, n: 2.0 * (1.0 - np.cos(np.pi * np.asarray(kp, float) / (2 * n))))
    kref = [1.0, 2.0, 0.5, 1.5, 0.7]
    r = np.random.default_rng(0).standard_normal((4, 5, 6))
    z = O.apply_reference_inverse(r, kref)
    back = O.apply_operator(O.reference_operator_faces(kref, r.shape), z)
    assert np.abs(back - r).max() > 1e-3


# ---------------------------------------------------------------- adjoint pins
def _kappa_eff(kx, ky, kz, d, lengths=(1.0, 1.0, 1.0)):
    return O.solve_direction(kx, ky, kz, d, lengths, rtol=1e-13).kappa_eff


@pytest.mark.parametrize("direction", [0, 2])
def test_adjoint_gradient_matches_central_differences(direction):
    shape = (4, 5, 3)
    rng = np.random.default_rng(31 + direction)
    kx, ky, kz = (rng.uniform(0.3, 6.0, shape) for _ in range(3))
    lengths = (1.0, 1.2, 0.9)
    G, kap, _, _ = O.adjoint_gradient(kx, ky, kz, direction, lengths, rtol=1e-13)
    eps = 1e-4
    for comp in range(3):
        for idx in [(0, 0, 0), (3, 4, 2), (1, 2, 1), (2, 0, 2)]:
            ks = [kx.copy(), ky.copy(), kz.copy()]
            ks[comp][idx] *= np.exp(eps)
            up = _kappa_eff(*ks, direction, lengths)
            ks[comp][idx] *= np.exp(-2 * eps)
            dn = _kappa_eff(*ks, direction, lengths)
            fd = (up - dn) / (2 * eps)
            assert G[comp][idx] == pytest.approx(fd, rel=1e-6, abs=1e-10 * kap)


def test_adjoint_identities():
    k = M.two_phase_random((6, 5, 7), seed=3, fraction=0.4, kappa_inclusion=30.0)
    for d in range(3):
        G, kap, p, lam = O.adjoint_gradient(k, k, k, d, p_in=2.0, p_out=0.5, rtol=1e-13)
        # lambda = c (p_in - p) / (p_in - p_out): the constant field solves equal data
        (k0, _, _), lens = O.permute_medium(k, k, k, (1.0, 1.0, 1.0), d)
        nz, ny, nx = k0.shape
        c = lens[2] * (lens[2] / nz) / (nx * ny * 1.5)
        np.testing.assert_allclose(lam, c * (2.0 - p) / 1.5, atol=1e-10 * c)
        # more conductance never lowers the flux; degree-1 homogeneity: sum = kappa_eff
        assert G.min() > -1e-12 * kap
        assert G.sum() == pytest.approx(kap, rel=1e-9)


# ---------------------------------------------------------------- Table 2 (smooth problem)
def _table2():
    rows = []
    with open(os.path.join(GOLDEN, "table2_smooth.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                r, n, e, it = line.split()
                rows.append((float(r), int(n), float(e), int(it)))
    return rows


@pytest.mark.parametrize("row", [r for r in _table2() if r[1] in (32, 64) and r[0] <= 1e-8])
def test_table2_smooth_problem(row):
    # Sec. 4.1: L2 error (3 digits) and iteration count of the converged rows.
    rtol, n, err, iters = row
    kx, ky, kz, pin, pout, src, exact = M.smooth_problem(n)
    p, it = O.solve_general(kx, ky, kz, pin, pout, src, rtol=rtol)
    l2 = np.sqrt(((p - exact) ** 2).sum() / n ** 3)
    # three printed digits: within half a unit of the third digit (+ slack)
    assert abs(l2 - err) / err < 0.002
    assert abs(it - iters) <= 1


def test_smooth_problem_data_consistency():
    # The source and boundary data must make the exact field a solution of the
    # continuous problem: the TPFA residual of the exact centre values is O(1),
    # while the residual of a wrong-sign source would be O(n^2) larger.
    n = 24
    kx, ky, kz, pin, pout, src, exact = M.smooth_problem(n)
    f = O.face_conductances(kx, ky, kz, (1.0, 1.0, 1.0))
    b = O.general_right_hand_side(f, pin, pout, src)
    res = O.apply_operator(f, exact) - b
    bad = O.apply_operator(f, exact) - O.general_right_hand_side(f, pin, pout, -src)
    assert np.abs(res).max() < 0.05 * np.abs(bad).max()
