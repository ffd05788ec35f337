"""Plain CPU FP64 oracle for the TPFA + PCG effective-thermal-conductivity solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The CUDA product path never calls it, and it imports nothing from the
product package: it is a slow, obviously correct restatement of the method of
Ye, Fu & Chung, "A fast cosine transformation accelerated method for predicting
effective thermal conductivity" (arXiv 2404.02433), written in numpy float64.

Array convention: every voxel array has shape (Nz, Ny, Nx) in C order, so
``a[k, j, i]`` is voxel (i, j, k) of Sec. 2.2 and i (x) runs fastest.  The
loading (Dirichlet) direction is always the slowest axis k, as in Sec. 2.1;
other directions are handled by permuting the medium first (Sec. 2.1, the
remark that kappa_eff^x and kappa_eff^y follow by moving the Dirichlet faces).

Every function below names the passage of the paper it restates.  Readings of
places where the paper is garbled or silent:
  * Eq. (forward/backward DCT): the sums are printed up to N; they run to N-1.
  * Sec. 2.2, ghost cells: the index set printed as a product {-1,N^x} x ... is
    read as "any index outside I_h" (p = 0 there).
  * Eq. (effective formula): n.K grad p is negative for p_in > p_out; the
    discrete Eq. (effective formula dis) with v = -K grad p is used, which is
    positive.
  * Lemma 3.1 / Lambda' and Lambda'': the out-group term is printed divided by
    kappa_ref^in; it is divided by kappa_ref^out.
  * Algorithm 2: the LP optimum is not unique.  The centred optimal point
    kappa_ref^g = sqrt(min_g * max_g) is used by default (proved optimal in the
    docstring of ``reference_parameters``); ``method="linprog"`` calls SciPy
    as the paper did.
  * Algorithm 1: the initial guess is not stated; p = 0 is used.
  * Off-diagonal tensor entries are not defined by the paper (Sec. 2.1 defers
    to a citation); ``effective_tensor`` defines K[a][b] = L^b <v_a> / dp under
    load b, <v_a> the volume average of the cell-averaged a-face fluxes.
    The definition is a reading; the code that evaluates it is pinned by a
    hand-solved 2 x 2 checkerboard (nonzero K[x][z], non-cubic boxes), by
    zero entries for mirror-symmetric media and by the diagonal formula for
    a == b.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

AXIS_NAMES = ("x", "y", "z")


# --------------------------------------------------------------------------
# Loading direction: move the Dirichlet axis to the slowest position.
# --------------------------------------------------------------------------
def loading_frame(direction: int):
    """Axes (as x=0,y=1,z=2) of the permuted frame (fast, middle, slow).

    The loading axis becomes the slow axis k (Sec. 2.1 aligns Gamma_in and
    Gamma_out with z); the other two keep their original relative order, the
    originally slower one becoming the middle axis.
    """
    if direction == 2:
        return (0, 1, 2)
    if direction == 1:
        return (0, 2, 1)
    if direction == 0:
        return (1, 2, 0)
    raise ValueError("direction must be 0, 1 or 2")


def permute_medium(kx, ky, kz, lengths, direction):
    """Return (k_fast, k_mid, k_slow), (L_fast, L_mid, L_slow) in the loading frame."""
    frame = loading_frame(direction)
    comps = (kx, ky, kz)
    # numpy axis of physical axis a in a (Nz, Ny, Nx) array is 2 - a
    perm = tuple(2 - a for a in reversed(frame))  # new (slow, mid, fast) order
    out = tuple(np.ascontiguousarray(np.transpose(comps[a], perm)) for a in frame)
    lens = tuple(lengths[a] for a in frame)
    return out, lens


def unpermute_field(p, direction):
    """Inverse of the spatial transpose applied by ``permute_medium``."""
    frame = loading_frame(direction)
    perm = tuple(2 - a for a in reversed(frame))
    inv = np.argsort(perm)
    return np.ascontiguousarray(np.transpose(p, inv))


# --------------------------------------------------------------------------
# Sec. 2.2: TPFA discretisation.
# --------------------------------------------------------------------------
@dataclass
class Faces:
    """Face conductances of Eq. (scaled bilinear forms).

    t0[k,j,i] couples (i-1,j,k)-(i,j,k) (zero at i = 0, a Neumann face);
    t1[k,j,i] couples (i,j-1,k)-(i,j,k) (zero at j = 0);
    t2[k,j,i] couples (i,j,k-1)-(i,j,k) (zero at k = 0);
    b_in[j,i] = 2 kappa~^z_{i,j,0}, b_out[j,i] = 2 kappa~^z_{i,j,Nz-1}.
    """

    t0: np.ndarray
    t1: np.ndarray
    t2: np.ndarray
    b_in: np.ndarray
    b_out: np.ndarray
    ks2: np.ndarray  # kappa~ along the loading axis (needed by the extrema)


def scaled_conductivity(kappa, h):
    """kappa~ = kappa / h^2 (Sec. 2.2, just before Eq. (scaled bilinear forms))."""
    return np.asarray(kappa, dtype=np.float64) / (h * h)


def harmonic_face(a, b):
    """kappa_F = 2 / (1/kappa_a + 1/kappa_b) for an internal face (Sec. 2.2)."""
    return 2.0 / (1.0 / a + 1.0 / b)


def face_conductances(k0, k1, k2, lengths):
    """Build the face arrays of Eq. (scaled bilinear forms) in the loading frame."""
    nz, ny, nx = k0.shape
    h0, h1, h2 = lengths[0] / nx, lengths[1] / ny, lengths[2] / nz
    s0 = scaled_conductivity(k0, h0)
    s1 = scaled_conductivity(k1, h1)
    s2 = scaled_conductivity(k2, h2)
    t0 = np.zeros_like(s0)
    t1 = np.zeros_like(s1)
    t2 = np.zeros_like(s2)
    t0[:, :, 1:] = harmonic_face(s0[:, :, :-1], s0[:, :, 1:])
    t1[:, 1:, :] = harmonic_face(s1[:, :-1, :], s1[:, 1:, :])
    t2[1:, :, :] = harmonic_face(s2[:-1, :, :], s2[1:, :, :])
    # Dirichlet faces: kappa_F = 2 kappa^z of the cell that holds the face.
    return Faces(t0, t1, t2, 2.0 * s2[0].copy(), 2.0 * s2[-1].copy(), s2)


def apply_operator(f: Faces, p):
    """q = A p for the bilinear form a = a* + a^in + a^out (Eq. scaled bilinear forms).

    a(p, q) = sum over internal faces of kappa~_F (p_c - p_nb)(q_c - q_nb)
              + sum_{k=0} 2 kappa~^z p q + sum_{k=Nz-1} 2 kappa~^z p q,
    so (A p)_c gathers kappa~_F (p_c - p_nb) over the internal faces of c plus
    the Dirichlet terms on the two end planes.
    """
    q = np.zeros_like(p)
    d = f.t0[:, :, 1:] * (p[:, :, 1:] - p[:, :, :-1])
    q[:, :, 1:] += d
    q[:, :, :-1] -= d
    d = f.t1[:, 1:, :] * (p[:, 1:, :] - p[:, :-1, :])
    q[:, 1:, :] += d
    q[:, :-1, :] -= d
    d = f.t2[1:, :, :] * (p[1:, :, :] - p[:-1, :, :])
    q[1:, :, :] += d
    q[:-1, :, :] -= d
    q[0] += f.b_in * p[0]
    q[-1] += f.b_out * p[-1]
    return q


def right_hand_side(f: Faces, p_in, p_out):
    """b from Eq. (flux) with p~_F = -p_in on Gamma_in (k = 0) and p_out on Gamma_out.

    Substituting v_F = -kappa_F (p^delta_F + p~_F / h^z) into sum v_F q^delta_F = 0
    moves the p~ terms to the right: b.q = sum 2 kappa~^z_{.,.,0} p_in q_0 +
    sum 2 kappa~^z_{.,.,Nz-1} p_out q_{Nz-1}.
    """
    nz = f.t0.shape[0]
    b = np.zeros((nz,) + f.b_in.shape)
    b[0] += f.b_in * p_in
    b[-1] += f.b_out * p_out
    return b


# --------------------------------------------------------------------------
# Sec. 3.1: reference parameters (Eq. parameters for linear programming, Alg. 2).
# --------------------------------------------------------------------------
GROUPS = ("x", "y", "z", "in", "out")


def group_extrema(f: Faces):
    """(min, max) of each group of Eq. (parameters for linear programming).

    Groups x, y, z range over internal faces of the three axes of the loading
    frame; 'in' and 'out' over kappa~^z on the planes k = 0 and k = Nz-1.  A
    group with no internal face (N = 1 along that axis) is returned as None.
    """
    out = []
    for t, sl in ((f.t0, np.s_[:, :, 1:]), (f.t1, np.s_[:, 1:, :]), (f.t2, np.s_[1:, :, :])):
        v = t[sl]
        out.append((float(v.min()), float(v.max())) if v.size else None)
    out.append((float(f.ks2[0].min()), float(f.ks2[0].max())))
    out.append((float(f.ks2[-1].min()), float(f.ks2[-1].max())))
    return out


def reference_parameters(extrema, method="centred"):
    """kappa_ref = [x, y, z, in, out] from Algorithm 2.

    LP (Eq. linear programming): minimise l'' - l' subject to
    c_g + l' <= log min_g and c_g + l'' >= log max_g for the five groups.
    Optimal value: any feasible point has l'' - l' >= log(max_g/min_g) for each
    g, and c_g = (log min_g + log max_g)/2, l'' = -l' = D/2 with
    D = max_g log(max_g/min_g) is feasible and attains it.  ``centred`` returns
    that point, kappa_ref^g = sqrt(min_g max_g).  ``linprog`` solves the LP with
    SciPy (the paper's tool; its vertex is one of many optima).  A group with
    no faces gets kappa_ref = 1; it multiplies the zero eigenvalue only.
    """
    if method == "centred":
        return [1.0 if e is None else math.sqrt(e[0] * e[1]) for e in extrema]
    if method == "linprog":
        from scipy.optimize import linprog

        live = [g for g, e in enumerate(extrema) if e is not None]
        nv = len(live) + 2  # c_g..., l', l''
        A, ub = [], []
        for col, g in enumerate(live):
            lo, hi = extrema[g]
            row = np.zeros(nv); row[col] = 1.0; row[-2] = 1.0
            A.append(row); ub.append(math.log(lo))
            row = np.zeros(nv); row[col] = -1.0; row[-1] = -1.0
            A.append(row); ub.append(-math.log(hi))
        cost = np.zeros(nv); cost[-1] = 1.0; cost[-2] = -1.0
        res = linprog(cost, A_ub=np.array(A), b_ub=np.array(ub),
                      bounds=[(None, None)] * nv, method="highs")
        if not res.success:
            raise RuntimeError(res.message)
        kref = [1.0] * 5
        for col, g in enumerate(live):
            kref[g] = math.exp(res.x[col])
        return kref
    raise ValueError(method)


def condition_bound(extrema, kref):
    """Lambda''/Lambda' of Lemma 3.1 (out group divided by kappa_ref^out)."""
    lo = min(e[0] / k for e, k in zip(extrema, kref) if e is not None)
    hi = max(e[1] / k for e, k in zip(extrema, kref) if e is not None)
    return hi / lo


# --------------------------------------------------------------------------
# Sec. 3.2: DCT and the preconditioner solve (Definition 1D DCT, Alg. 3).
# --------------------------------------------------------------------------
def cosine_matrix(n):
    """C[i', i] = cos(pi (2i+1) i' / (2n)), the kernel of Eq. (forward DCT).

    The angle is reduced exactly in integers, m = (2i+1) i' mod 4n, before the
    cosine of pi m / (2n) is taken.
    """
    ip = np.arange(n, dtype=np.int64)[:, None]
    i = np.arange(n, dtype=np.int64)[None, :]
    m = ((2 * i + 1) * ip) % (4 * n)
    return np.cos(np.pi * m.astype(np.float64) / (2.0 * n))


def dct_forward(u, axis):
    """Eq. (forward DCT) along ``axis``: u^_{i'} = sum_{i<N} u_i cos(pi (2i+1) i' / 2N)."""
    n = u.shape[axis]
    c = cosine_matrix(n)
    return np.moveaxis(np.tensordot(c, np.moveaxis(u, axis, 0), axes=(1, 0)), 0, axis)


def dct_backward(uh, axis):
    """Eq. (backward DCT): u_i = (2/N) sum_{i'<N} alpha_{i'} u^_{i'} cos(...), alpha_0 = 1/2."""
    n = uh.shape[axis]
    c = cosine_matrix(n)
    alpha = np.ones(n); alpha[0] = 0.5
    w = (2.0 / n) * (c.T * alpha[None, :])
    return np.moveaxis(np.tensordot(w, np.moveaxis(uh, axis, 0), axes=(1, 0)), 0, axis)


def neumann_eigenvalue(kp, n):
    """lambda_k = 2 (1 - cos(k pi / N)) of the 1-D Neumann matrix in Sec. 3.2.

    Written as 4 sin^2(k pi / 2N), the same number without the cancellation of
    1 - cos for small k.
    """
    s = np.sin(np.pi * np.asarray(kp, dtype=np.float64) / (2.0 * n))
    return 4.0 * s * s


def thomas(sub, diag, sup, rhs):
    """Plain Thomas elimination for tridiagonal systems along axis 0.

    sub/sup have length n-1 along axis 0, diag and rhs length n; the trailing
    axes index independent systems.
    """
    n = diag.shape[0]
    c = np.zeros_like(rhs)
    d = np.zeros_like(rhs)
    denom = diag[0]
    c[0] = (sup[0] / denom) if n > 1 else 0.0
    d[0] = rhs[0] / denom
    for k in range(1, n):
        denom = diag[k] - sub[k - 1] * c[k - 1]
        if k < n - 1:
            c[k] = sup[k] / denom
        d[k] = (rhs[k] - sub[k - 1] * d[k - 1]) / denom
    x = np.zeros_like(rhs)
    x[n - 1] = d[n - 1]
    for k in range(n - 2, -1, -1):
        x[k] = d[k] - c[k] * x[k + 1]
    return x


def reference_tridiagonal(kref, nx, ny, nz):
    """Diagonal of T_{i',j'} (Sec. 3.2), shape (nz, ny, nx); off-diagonal is -kappa_ref^z."""
    kx, ky, kz, kin, kout = kref
    s = (neumann_eigenvalue(np.arange(nx), nx)[None, :] * kx
         + neumann_eigenvalue(np.arange(ny), ny)[:, None] * ky)
    diag = np.empty((nz, ny, nx))
    diag[:] = s[None] + 2.0 * kz
    if nz == 1:
        diag[0] = s + 2.0 * kin + 2.0 * kout
    else:
        diag[0] = s + kz + 2.0 * kin
        diag[-1] = s + kz + 2.0 * kout
    return diag


def apply_reference_inverse(r, kref):
    """z = A_ref^{-1} r by Algorithm 3.

    1) 2-D forward DCT in x and y for every k; 2) for each (i', j') solve
    T_{i',j'} z^ = r^ along k; 3) 2-D backward DCT in x and y.
    """
    nz, ny, nx = r.shape
    rh = dct_forward(dct_forward(r, 2), 1)
    diag = reference_tridiagonal(kref, nx, ny, nz)
    off = np.full((max(nz - 1, 0), ny, nx), -kref[2])
    zh = thomas(off, diag, off, rh)
    return dct_backward(dct_backward(zh, 1), 2)


def reference_operator_faces(kref, shape):
    """Faces of the homogeneous reference form a_ref (Eq. refer bilinear forms)."""
    nz, ny, nx = shape
    t0 = np.full(shape, kref[0]); t0[:, :, 0] = 0.0
    t1 = np.full(shape, kref[1]); t1[:, 0, :] = 0.0
    t2 = np.full(shape, kref[2]); t2[0] = 0.0
    return Faces(t0, t1, t2, np.full((ny, nx), 2.0 * kref[3]),
                 np.full((ny, nx), 2.0 * kref[4]), np.full(shape, np.nan))


# --------------------------------------------------------------------------
# Algorithm 1: PCG.
# --------------------------------------------------------------------------
@dataclass
class PcgResult:
    p: np.ndarray
    iters: int
    relres: float
    converged: bool
    history: list = field(default_factory=list)


def pcg(f: Faces, b, kref, rtol=1e-10, maxit=5000, p0=None, on_iterate=None):
    """Algorithm 1 with exit criterion ||r||_2 / ||b||_2 <= rtol (Eq. exit).

    The criterion is tested before each pass of the loop, so ``iters`` is the
    number of products with A after the initial residual.  ``on_iterate``, if
    given, is called as on_iterate(it, p, relres) after every pass; it only
    observes the iterate (the iterates are those of a run without it), so one
    run can report the solution at several exit thresholds.
    """
    p = np.zeros_like(b) if p0 is None else p0.copy()
    r = b - apply_operator(f, p)
    z = apply_reference_inverse(r, kref)
    w = z.copy()
    rho = float(np.vdot(r, z))
    bnorm = float(np.linalg.norm(b))
    hist = [float(np.linalg.norm(r)) / bnorm]
    it = 0
    while hist[-1] > rtol and it < maxit:
        z = apply_operator(f, w)
        alpha = rho / float(np.vdot(z, w))
        p = p + alpha * w
        r = r - alpha * z
        z = apply_reference_inverse(r, kref)
        rho_new = float(np.vdot(r, z))
        w = z + (rho_new / rho) * w
        rho = rho_new
        it += 1
        hist.append(float(np.linalg.norm(r)) / bnorm)
        if on_iterate is not None:
            on_iterate(it, p, hist[-1])
    return PcgResult(p, it, hist[-1], hist[-1] <= rtol, hist)


# --------------------------------------------------------------------------
# Post-processing: Eq. (flux) and Eq. (effective formula dis).
# --------------------------------------------------------------------------
def outflow_etc(f: Faces, p, lengths, p_in, p_out):
    """kappa_eff = L^z sum_ij v_{i,j,Nz-1/2} / (Nx Ny (p_in - p_out)).

    On Gamma_out, Eq. (flux) gives v = -kappa_F (p^delta + p_out / h^z) with
    kappa_F = 2 kappa^z_{i,j,Nz-1} and p^delta = (0 - p_{Nz-1}) / h^z, so
    v = 2 kappa^z (p_{Nz-1} - p_out) / h^z = b_out h^z (p_{Nz-1} - p_out).
    """
    nz, ny, nx = p.shape
    hz = lengths[2] / nz
    v = f.b_out * hz * (p[-1] - p_out)
    return lengths[2] * float(v.sum()) / (nx * ny * (p_in - p_out))


def inflow_etc(f: Faces, p, lengths, p_in, p_out):
    """Same as ``outflow_etc`` through Gamma_in: v = 2 kappa^z (p_in - p_0) / h^z."""
    nz, ny, nx = p.shape
    hz = lengths[2] / nz
    v = f.b_in * hz * (p_in - p[0])
    return lengths[2] * float(v.sum()) / (nx * ny * (p_in - p_out))


def energy_etc(f: Faces, p, b, lengths, p_in, p_out):
    """kappa_eff from the minimised energy (an identity of the discrete system).

    With E = p.Ap - 2 b.p + sum b_in p_in^2 + sum b_out p_out^2 (the quadratic
    form of all face fluxes, Dirichlet faces included), the total outflow of the
    exact solution is E / (h^z (p_in - p_out)) ... times the scaling of the
    flux formula; it agrees with ``outflow_etc`` up to the square of the solve
    error.
    """
    nz, ny, nx = p.shape
    hz = lengths[2] / nz
    e = (float(np.vdot(p, apply_operator(f, p))) - 2.0 * float(np.vdot(b, p))
         + float(f.b_in.sum()) * p_in * p_in + float(f.b_out.sum()) * p_out * p_out)
    dp = p_in - p_out
    return lengths[2] * hz * e / (nx * ny * dp * dp)


def plane_fluxes(f: Faces, p, lengths, p_in, p_out):
    """Total z-flux (times h^z) through every plane of z-faces, k = -1/2 .. Nz-1/2."""
    hz = lengths[2] / p.shape[0]
    out = [float((f.b_in * hz * (p_in - p[0])).sum())]
    for k in range(1, p.shape[0]):
        out.append(float((f.t2[k] * hz * (p[k - 1] - p[k])).sum()))
    out.append(float((f.b_out * hz * (p[-1] - p_out)).sum()))
    return np.array(out)


def mean_face_fluxes(f: Faces, p, lengths, p_in, p_out):
    """<v_a> for a = fast, mid, slow axes of the loading frame.

    Each cell averages its two a-faces (Neumann faces carry zero flux, Sec. 2.2);
    the volume average of that is the sum over internal faces plus half of each
    Dirichlet face, divided by the number of cells.
    """
    nz, ny, nx = p.shape
    n = p.size
    h = (lengths[0] / nx, lengths[1] / ny, lengths[2] / nz)
    v0 = float((f.t0[:, :, 1:] * h[0] * (p[:, :, :-1] - p[:, :, 1:])).sum())
    v1 = float((f.t1[:, 1:, :] * h[1] * (p[:, :-1, :] - p[:, 1:, :])).sum())
    v2 = float((f.t2[1:] * h[2] * (p[:-1] - p[1:])).sum())
    v2 += 0.5 * float((f.b_in * h[2] * (p_in - p[0])).sum())
    v2 += 0.5 * float((f.b_out * h[2] * (p[-1] - p_out)).sum())
    return np.array([v0, v1, v2]) / n


# --------------------------------------------------------------------------
# Whole routine (Sec. 2.2 closing paragraph) and the 3 x 3 tensor.
# --------------------------------------------------------------------------
@dataclass
class DirectionResult:
    kappa_eff: float
    iters: int
    relres: float
    converged: bool
    kref: list
    cond_bound: float
    p: np.ndarray          # solution in the ORIGINAL (Nz, Ny, Nx) frame
    column: np.ndarray     # K[:, direction] in original axes


def solve_direction(kx, ky, kz, direction, lengths=(1.0, 1.0, 1.0), p_in=1.0,
                    p_out=0.0, rtol=1e-10, maxit=5000, ref_method="centred", kref=None):
    """Solve A p = b for one loading direction and return kappa_eff (Sec. 2.2).

    Steps: permute so the load is along k; faces; reference parameters
    (Algorithm 2); PCG (Algorithm 1 with Algorithm 3); outflow formula.
    """
    if p_in == p_out:
        raise ValueError("p_in must differ from p_out (Sec. 2.1)")
    (k0, k1, k2), lens = permute_medium(kx, ky, kz, lengths, direction)
    f = face_conductances(k0, k1, k2, lens)
    ext = group_extrema(f)
    if kref is None:
        kref = reference_parameters(ext, ref_method)
    b = right_hand_side(f, p_in, p_out)
    res = pcg(f, b, kref, rtol=rtol, maxit=maxit)
    kap = outflow_etc(f, res.p, lens, p_in, p_out)
    vbar = mean_face_fluxes(f, res.p, lens, p_in, p_out)
    frame = loading_frame(direction)
    column = np.zeros(3)
    for local, axis in enumerate(frame):
        column[axis] = lengths[direction] * vbar[local] / (p_in - p_out)
    return DirectionResult(kap, res.iters, res.relres, res.converged, list(kref),
                           condition_bound(ext, kref), unpermute_field(res.p, direction),
                           column)


def effective_tensor(kx, ky=None, kz=None, lengths=(1.0, 1.0, 1.0), rtol=1e-10,
                     maxit=5000, ref_method="centred"):
    """K[a][b]: column b from the solve loaded along b (Sec. 2.1)."""
    ky = kx if ky is None else ky
    kz = kx if kz is None else kz
    K = np.zeros((3, 3))
    results = []
    for d in range(3):
        r = solve_direction(kx, ky, kz, d, lengths, rtol=rtol, maxit=maxit,
                            ref_method=ref_method)
        K[:, d] = r.column
        K[d, d] = r.kappa_eff
        results.append(r)
    return K, results


# --------------------------------------------------------------------------
# Adjoint gradient d kappa_eff / d log kappa (derived from Sec. 2.2; the
# paper has no adjoint).  J = kappa_eff of Eq. (effective formula dis).
# --------------------------------------------------------------------------
def adjoint_gradient(kx, ky, kz, direction, lengths=(1.0, 1.0, 1.0), p_in=1.0, p_out=0.0,
                     rtol=1e-12, maxit=5000):
    """Per-voxel dJ/d log kappa^a for a = x, y, z, shape (3, Nz, Ny, Nx).

    J = c sum_ij b_out (p_{Nz-1} - p_out), c = L^z h^z / (Nx Ny (p_in - p_out)),
    with A(kappa) p = b(kappa).  A is symmetric, so the adjoint lambda solves
    A lambda = dJ/dp = c b_out on the last plane -- the right-hand side of the
    same system with Dirichlet data (0, c).  Then
      dJ/dtheta = dJ/dtheta|explicit + lambda.(db/dtheta - dA/dtheta p),
    where, for theta = log kappa of one voxel and one component,
      internal face T = 2ab/(a+b):  dT/dlog a = T b/(a+b),
      Dirichlet faces b_in, b_out = 2 kappa~^z:  d/dlog = themselves,
      dA/dtheta p . lambda = sum_F dT_F (p_c - p_nb)(lambda_c - lambda_nb)
                              + d b_in p_0 lambda_0 + d b_out p_{Nz-1} lambda_{Nz-1},
      db/dtheta . lambda = d b_in p_in lambda_0 + d b_out p_out lambda_{Nz-1},
      dJ/dtheta|explicit = c d b_out (p_{Nz-1} - p_out).
    Returns (grad, kappa_eff, p, lambda) with p and lambda in the loading frame.
    """
    (k0, k1, k2), lens = permute_medium(kx, ky, kz, lengths, direction)
    nz, ny, nx = k0.shape
    f = face_conductances(k0, k1, k2, lens)
    kref = reference_parameters(group_extrema(f))
    b = right_hand_side(f, p_in, p_out)
    p = pcg(f, b, kref, rtol=rtol, maxit=maxit).p
    hz = lens[2] / nz
    c = lens[2] * hz / (nx * ny * (p_in - p_out))
    kap = outflow_etc(f, p, lens, p_in, p_out)
    lam = pcg(f, right_hand_side(f, 0.0, c), kref, rtol=rtol, maxit=maxit).p
    h = (lens[0] / nx, lens[1] / ny, lens[2] / nz)
    s = (scaled_conductivity(k0, h[0]), scaled_conductivity(k1, h[1]),
         scaled_conductivity(k2, h[2]))
    G = np.zeros((3,) + p.shape)
    for ax, t in enumerate((f.t0, f.t1, f.t2)):
        npax = 2 - ax
        hi = [slice(None)] * 3
        lo = [slice(None)] * 3
        hi[npax] = slice(1, None)
        lo[npax] = slice(None, -1)
        hi, lo = tuple(hi), tuple(lo)
        a, bb = s[ax][hi], s[ax][lo]
        tf = t[hi]
        prod = (p[hi] - p[lo]) * (lam[hi] - lam[lo])
        G[ax][hi] -= tf * bb / (a + bb) * prod
        G[ax][lo] -= tf * a / (a + bb) * prod
    G[2][0] += f.b_in * lam[0] * (p_in - p[0])
    G[2][-1] += c * f.b_out * (p[-1] - p_out) + f.b_out * lam[-1] * (p_out - p[-1])
    frame = loading_frame(direction)
    grad = np.zeros((3,) + kx.shape)
    for local, axis in enumerate(frame):
        grad[axis] = unpermute_field(G[local], direction)
    return grad, kap, p, lam


# --------------------------------------------------------------------------
# General data: spatially varying Dirichlet values and a source term
# (Sec. 4.1, the smooth test of Table 2).  Loading along z only.
# --------------------------------------------------------------------------
def general_right_hand_side(f: Faces, p_in_face, p_out_face, source):
    """b for -div(K grad p) = source with p = p_in(x, y) on z = 0, p_out(x, y) on z = L^z.

    Eq. (flux) with p~_F = -p_in(F) / p_out(F) gives the Dirichlet part as in
    ``right_hand_side`` with face values instead of constants; the second
    equation of the mixed system with div v = source adds the cell values of
    the source (the scaled system divides both sides by the cell volume).
    """
    b = source.astype(np.float64).copy()
    b[0] += f.b_in * p_in_face
    b[-1] += f.b_out * p_out_face
    return b


def solve_general(kx, ky, kz, p_in_face, p_out_face, source, lengths=(1.0, 1.0, 1.0),
                  rtol=1e-10, maxit=5000, kref=None):
    """Solution of the TPFA system with general data (load along z): (p, iters)."""
    f = face_conductances(kx, ky, kz, lengths)
    if kref is None:
        kref = reference_parameters(group_extrema(f))
    b = general_right_hand_side(f, p_in_face, p_out_face, source)
    res = pcg(f, b, kref, rtol=rtol, maxit=maxit)
    return res.p, res.iters
