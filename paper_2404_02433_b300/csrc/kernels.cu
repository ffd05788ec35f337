// CUDA kernels of the TPFA + PCG hot path and their host launchers.
//
// Per PCG iteration (Algorithm 1) the solver launches, in stream order:
//   matvec   w <- z + beta w_old ; q <- A w ; partial w.q   -> alpha  (last block)
//   fwd_x    x <- x + alpha w ; r <- r - alpha q ; ||r||^2 -> convergence (last block);
//            forward DCT of r along axis 0
//   fwd_y    forward DCT along axis 1                                  (Algorithm 3, step 1)
//   tridiag  T_{i'j'} z^ = r^ along axis 2 ; r.z in the transform domain -> beta
//                                                                       (Algorithm 3, step 2)
//   inv_y    backward DCT along axis 1                                 (Algorithm 3, step 3)
//   inv_x    backward DCT along axis 0 -> z (flexible PCG: z.q -> beta)
// Every kernel returns at entry once the device flag `done` is set, so the host
// may launch iterations ahead of the convergence test.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "dct_device.cuh"
#include "etc_internal.cuh"
#include "launchers.h"

namespace etc {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ long long gidx() {
  return (long long)blockIdx.x * blockDim.x + threadIdx.x;
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// ------------------------------------------------------------------ setup: checks
// min, max and count of non-finite or non-positive values of one input array.
__global__ void k_kappa_stats(const double* __restrict__ a, long long n, double* partials,
                              PcgState* st, int slot) {
  __shared__ int flag;
  double lo = INFINITY, hi = -INFINITY, bad = 0.0;
  for (long long c = gidx(); c < n; c += (long long)gridDim.x * blockDim.x) {
    const double v = a[c];
    if (!(v > 0.0) || !isfinite(v)) bad += 1.0;
    else { lo = fmin(lo, v); hi = fmax(hi, v); }
  }
  // block min / max / sum
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
    bad += __shfl_down_sync(0xffffffffu, bad, o);
  }
  __shared__ double wl[32], wh[32], wb[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) { wl[wid] = lo; wh[wid] = hi; wb[wid] = bad; }
  __syncthreads();
  double vals[3] = {INFINITY, -INFINITY, 0.0};
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) {
      vals[0] = fmin(vals[0], wl[w]); vals[1] = fmax(vals[1], wh[w]); vals[2] += wb[w];
    }
  if (publish_values(partials, 3, vals, 3, &st->cnt[kCntExt], &flag)) {
    // every thread a stride of blocks, then warps and block (min, max and the
    // integer-valued count do not depend on the order)
    double l2 = INFINITY, h2 = -INFINITY, b2 = 0.0;
    const unsigned int nb = nblocks();
    for (unsigned int b = threadIdx.x; b < nb; b += blockDim.x) {
      l2 = fmin(l2, __ldcg(partials + 3 * (size_t)b));
      h2 = fmax(h2, __ldcg(partials + 3 * (size_t)b + 1));
      b2 += __ldcg(partials + 3 * (size_t)b + 2);
    }
    for (int o = 16; o > 0; o >>= 1) {
      l2 = fmin(l2, __shfl_down_sync(0xffffffffu, l2, o));
      h2 = fmax(h2, __shfl_down_sync(0xffffffffu, h2, o));
      b2 += __shfl_down_sync(0xffffffffu, b2, o);
    }
    __syncthreads();
    if (lane == 0) { wl[wid] = l2; wh[wid] = h2; wb[wid] = b2; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < nw; ++w) { l2 = fmin(l2, wl[w]); h2 = fmax(h2, wh[w]); b2 += wb[w]; }
      st->ext[3 * slot] = l2; st->ext[3 * slot + 1] = h2; st->ext[3 * slot + 2] = b2;
      st->cnt[kCntExt] = 0;
    }
  }
}

// ------------------------------------------------------------------ setup: permutation
// out[o2][o1][o0] = in[o0*s0 + o1*s1 + o2*s2] (in dense, out dense).  When the
// input-contiguous axis is not o0 it is axis f (1 or 2) and a 32x32 shared
// tile makes both sides coalesced.
__global__ void k_permute_direct(const double* __restrict__ in, double* __restrict__ out, int d0,
                                 int d1, int d2, long long s1, long long s2) {
  const long long n = (long long)d0 * d1 * d2;
  for (long long o = gidx(); o < n; o += (long long)gridDim.x * blockDim.x) {
    const long long o0 = o % d0, r = o / d0, o1 = r % d1, o2 = r / d1;
    out[o] = in[o0 + o1 * s1 + o2 * s2];
  }
}

__global__ void k_permute_tile(const double* __restrict__ in, double* __restrict__ out, int d0,
                               int d1, int d2, long long s0, long long so, int f) {
  __shared__ double tile[32][33];
  const int df = (f == 1) ? d1 : d2;
  const int o0b = blockIdx.x * 32, ofb = blockIdx.y * 32, oo = blockIdx.z;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int rr = ty; rr < 32; rr += 8) {
    const int o0 = o0b + rr, of = ofb + tx;
    if (o0 < d0 && of < df) tile[rr][tx] = in[(long long)o0 * s0 + of + (long long)oo * so];
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8) {
    const int o0 = o0b + tx, of = ofb + rr;
    if (o0 < d0 && of < df) {
      const long long o1 = (f == 1) ? of : oo, o2 = (f == 1) ? oo : of;
      out[o0 + (long long)d0 * (o1 + (long long)d1 * o2)] = tile[tx][rr];
    }
  }
}

// ------------------------------------------------------------------ setup: faces
// 2ab/(a+b).  The reciprocal of s = a+b comes from the FP32 hardware
// approximation refined by two Newton-Raphson steps r <- r + r (1 - s r) in
// FP64 (each roughly doubles the correct bits: 2^-22 -> 2^-44 -> the FP64
// rounding), so the face is within about two units in the last place of the
// correctly rounded quotient, at 7 FP64 instructions per face instead of a
// full division: the face assembly is FP64-bound on this part (about 45 FP64
// instructions per cell with three divisions).  Sums outside the binary32
// normal range keep the division.
__device__ __forceinline__ double harmonic(double a, double b) {
  const double s = a + b;
  const float sf = narrow(s);
  if (!(sf > 1e-30f && sf < 1e30f)) return 2.0 * (a * b) / s;
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(sf));
  double r = widen(rf);
  r = fma(r, fma(-s, r, 1.0), r);
  r = fma(r, fma(-s, r, 1.0), r);
  return 2.0 * (a * b) * r;
}

// Face conductances of Eq. (scaled bilinear forms) in the loading frame, the
// diagonal D of A, the Dirichlet planes and the group extrema of
// Eq. (parameters for linear programming): res[0..9] = (min, max) of the x, y,
// z internal faces, kappa~^z on plane 0 and on plane n2-1.
__global__ void k_faces(Geometry g, double ih0, double ih1, double ih2,
                        const double* __restrict__ k0, const double* __restrict__ k1,
                        const double* __restrict__ k2, double* __restrict__ T0,
                        double* __restrict__ T1, double* __restrict__ T2, double* __restrict__ D,
                        double* __restrict__ Bin, double* __restrict__ Bout, double* partials,
                        PcgState* st) {
  __shared__ int flag;
  // Extrema of positive doubles (faces and kappa~ are > 0) kept as their bit
  // patterns: for non-negative IEEE values the unsigned-integer order is the
  // numeric order, so the integer pipe does the min/max (the FP64 pipe is
  // this kernel's bound).  Empty: lo = +inf bits, hi = 0.
  constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;
  unsigned long long lo[5], hi[5];
  for (int e = 0; e < 5; ++e) { lo[e] = kInfBits; hi[e] = 0ull; }
  auto note = [&](int e, double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    lo[e] = min(lo[e], b);
    hi[e] = max(hi[e], b);
  };
  // threads stride over the cells of a plane and blocks over the planes
  // (k = blockIdx.y + m gridDim.y): the three "minus" faces of each cell (each
  // face once; the diagonal follows in k_diag_split from the neighbours' faces)
  for (long long sidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; sidx < g.plane;
       sidx += (long long)gridDim.x * blockDim.x)
  for (int k = blockIdx.y; k < g.n2; k += gridDim.y) {
    const int j = (int)(sidx / g.n0), i = (int)(sidx - (long long)j * g.n0);
    const long long c = (long long)k * g.plane + sidx;
    const double s0 = k0[c] * ih0, s1 = k1[c] * ih1, s2 = k2[c] * ih2;
    const double t0 = (i > 0) ? harmonic(k0[c - 1] * ih0, s0) : 0.0;
    const double t1 = (j > 0) ? harmonic(k1[c - g.n0] * ih1, s1) : 0.0;
    const double t2 = (k > 0) ? harmonic(k2[c - g.plane] * ih2, s2) : 0.0;
    if (k == 0) { Bin[sidx] = 2.0 * s2; note(3, s2); }
    if (k == g.n2 - 1) { Bout[sidx] = 2.0 * s2; note(4, s2); }
    T0[c] = t0; T1[c] = t1; T2[c] = t2;
    if (i > 0) note(0, t0);
    if (j > 0) note(1, t1);
    if (k > 0) note(2, t2);
  }
  double ext[10];
  for (int e = 0; e < 5; ++e) {
    ext[2 * e] = __longlong_as_double((long long)lo[e]);
    ext[2 * e + 1] = lo[e] == kInfBits ? -INFINITY : __longlong_as_double((long long)hi[e]);
  }
  __shared__ double we[32][10];
  for (int o = 16; o > 0; o >>= 1)
    for (int e = 0; e < 10; e += 2) {
      ext[e] = fmin(ext[e], __shfl_down_sync(0xffffffffu, ext[e], o));
      ext[e + 1] = fmax(ext[e + 1], __shfl_down_sync(0xffffffffu, ext[e + 1], o));
    }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0)
    for (int e = 0; e < 10; ++e) we[wid][e] = ext[e];
  __syncthreads();
  double vals[10];
  if (threadIdx.x == 0) {
    for (int e = 0; e < 10; e += 2) { vals[e] = INFINITY; vals[e + 1] = -INFINITY; }
    for (int w = 0; w < nw; ++w)
      for (int e = 0; e < 10; e += 2) {
        vals[e] = fmin(vals[e], we[w][e]);
        vals[e + 1] = fmax(vals[e + 1], we[w][e + 1]);
      }
  }
  if (publish_values(partials, 10, vals, 10, &st->cnt[kCntExt], &flag)) {
    // min / max over the blocks' extrema: every thread a stride of blocks, then
    // the warps and the block (min and max do not depend on the order)
    double r[10];
    for (int e = 0; e < 10; e += 2) { r[e] = INFINITY; r[e + 1] = -INFINITY; }
    const unsigned int nb = nblocks();
    for (unsigned int b = threadIdx.x; b < nb; b += blockDim.x)
      for (int e = 0; e < 10; e += 2) {
        r[e] = fmin(r[e], __ldcg(partials + 10 * (size_t)b + e));
        r[e + 1] = fmax(r[e + 1], __ldcg(partials + 10 * (size_t)b + e + 1));
      }
    for (int o = 16; o > 0; o >>= 1)
      for (int e = 0; e < 10; e += 2) {
        r[e] = fmin(r[e], __shfl_down_sync(0xffffffffu, r[e], o));
        r[e + 1] = fmax(r[e + 1], __shfl_down_sync(0xffffffffu, r[e + 1], o));
      }
    __syncthreads();
    if (lane == 0)
      for (int e = 0; e < 10; ++e) we[wid][e] = r[e];
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < nw; ++w)
        for (int e = 0; e < 10; e += 2) {
          r[e] = fmin(r[e], we[w][e]);
          r[e + 1] = fmax(r[e + 1], we[w][e + 1]);
        }
      for (int e = 0; e < 10; ++e) st->ext[e] = r[e];
      // Algorithm 2, centred optimal point; a group without faces gets 1
      for (int gi = 0; gi < 5; ++gi) {
        const double lo = r[2 * gi], hi = r[2 * gi + 1];
        st->kref_lp[gi] = (isfinite(lo) && isfinite(hi) && lo > 0.0) ? sqrt(lo * hi) : 1.0;
      }
      st->cnt[kCntExt] = 0;
    }
  }
}

// ------------------------------------------------------------------ setup: pivots
// For every (i', j'): the LDL^T pivots of T_{i'j'} / kappa_ref^z (Sec. 3.2),
// stored as h_k = 1 / pivot_k in the layout of the transformed field.
template <typename R>
__global__ void k_pivots(Geometry g, const double* __restrict__ lam0,
                         const double* __restrict__ lam1, const double* kd, double kx, double ky,
                         double kz, double kin, double kout, R* __restrict__ h) {
  const long long s = gidx();
  if (s >= g.plane) return;
  if (kd) { kx = kd[0]; ky = kd[1]; kz = kd[2]; kin = kd[3]; kout = kd[4]; }
  const int i = (int)(s % g.n0), j = (int)(s / g.n0);
  const double sv = (lam0[i] * kx + lam1[j] * ky) / kz;
  const double a_in = 2.0 * kin / kz, a_out = 2.0 * kout / kz;
  if (g.n2 == 1) {
    h[s] = (R)(1.0 / (sv + a_in + a_out));
    return;
  }
  double hp = 1.0 / (sv + 1.0 + a_in);
  h[s] = (R)hp;
  for (int k = 1; k < g.n2; ++k) {
    const double dk = (k == g.n2 - 1) ? (sv + 1.0 + a_out) : (sv + 2.0);
    hp = 1.0 / (dk - hp);
    h[(long long)k * g.plane + s] = (R)hp;
  }
}

// kref = LP optimum, all ones, or user values (Algorithm 2 / the paper's "one").
__global__ void k_select_kref(PcgState* st, int mode, double u0, double u1, double u2, double u3,
                              double u4) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double u[5] = {u0, u1, u2, u3, u4};
  for (int gi = 0; gi < 5; ++gi)
    st->kref[gi] = (mode == 0) ? st->kref_lp[gi] : (mode == 1 ? 1.0 : u[gi]);
}

// Clear the PCG part of the state before a solve (extrema and kref are kept).
__global__ void k_state_reset(PcgState* st, int maxit) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->rho = 0.0; st->beta = 0.0; st->alpha[0] = 0.0; st->alpha[1] = 0.0;
  st->rr = 0.0; st->bb = 0.0; st->thresh2 = 0.0; st->dq = 0.0; st->zq = 0.0;
  for (int e = 0; e < 8; ++e) { st->res[e] = 0.0; st->cnt[e] = 0u; }
  st->iter = 0; st->maxit = maxit; st->done = 0; st->status = kOK; st->phase = 0;
  st->passes = 0;
  st->max_passes = maxit / 2 + 4;  // the loop body runs two iterations
  st->xpend = 0;
  st->bb_given = 0.0;
}

// End of one pass of a device-driven PCG loop (graph WHILE node): stop when
// the solve is done, or after max_passes passes whatever happened.
__global__ void k_loop_control(PcgState* st, cudaGraphConditionalHandle handle) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->passes += 1;
  if (!st->done && st->passes >= st->max_passes) {
    st->status = kENOCONV;
    st->done = 1;
  }
  if (st->done) cudaGraphSetConditional(handle, 0u);
}

// ------------------------------------------------------------------ init
// r = b, x = 0, w_old = 0.  b (Eq. flux): b_in p_in on plane 0 and b_out p_out
// on plane n2-1, with per-face values pin_f / pout_f (plane layout) when given,
// plus the source term src (loading-frame layout) when given.
__global__ void k_init(Geometry g, const double* __restrict__ Bin, const double* __restrict__ Bout,
                       double pin, double pout, const double* __restrict__ pin_f,
                       const double* __restrict__ pout_f, const double* __restrict__ src,
                       double* __restrict__ r, double* __restrict__ x, double* __restrict__ w0) {
  for (long long c = gidx(); c < g.n; c += (long long)gridDim.x * blockDim.x) {
    const long long k = c / g.plane, s = c - k * g.plane;
    double b = src ? src[c] : 0.0;
    if (k == 0) b += Bin[s] * (pin_f ? pin_f[s] : pin);
    if (k == g.n2 - 1) b += Bout[s] * (pout_f ? pout_f[s] : pout);
    r[c] = b;
    x[c] = 0.0;
    if (w0) w0[c] = 0.0;
  }
}

// Initial guess x0 of a homogeneous medium: the TPFA solution with constant
// conductivity is linear in k, half a cell from each Dirichlet face,
// x_c = p_in + (p_out - p_in) (k + 1/2) / n2.  Also ||b||^2 of r = b (last
// block: st->bb_given), for the exit test of Eq. (exit), which stays relative
// to ||b|| when r_0 = b - A x0 differs from b.
__global__ void k_init_linear(Geometry g, double pin, double pout, const double* __restrict__ r,
                              double* __restrict__ x, double* partials, PcgState* st) {
  __shared__ double sh[32];
  __shared__ int flag;
  double acc = 0.0;
  for (long long c = gidx(); c < g.n; c += (long long)gridDim.x * blockDim.x) {
    const long long k = c / g.plane;
    x[c] = pin + (pout - pin) * (((double)k + 0.5) / (double)g.n2);
    acc = fma(r[c], r[c], acc);
  }
  const double bs = block_sum(acc, sh);
  double v[1] = {bs};
  if (publish_values(partials, 1, v, 1, &st->cnt[kCntAux], &flag)) {
    const double bb = sum_partials(partials, (int)nblocks(), 1, sh);
    if (threadIdx.x == 0) {
      st->bb_given = bb;
      st->cnt[kCntAux] = 0;
    }
  }
}

// r <- r - q
__global__ void k_sub(long long n, double* __restrict__ r, const double* __restrict__ q) {
  for (long long c = gidx(); c < n; c += (long long)gridDim.x * blockDim.x) r[c] -= q[c];
}

// ------------------------------------------------------------------ matvec
// q_c = D_c w_c - sum_f T_f w_nb (Eq. scaled bilinear forms): one cell per
// thread, the six neighbours come through L1/L2 (each w value is used by seven
// cells; the z-neighbours one plane away stay resident in L2).  Neighbour
// indices are clamped at the domain edge, where the face value T is zero, so
// the loads stay in bounds without branches.  The "plus" faces T0[c+1],
// T1[c+n0], T2[c+plane] are read from arrays that carry one zero plane of
// padding.
// MODE 0: q = A w.  MODE 1: PCG step, also w.q -> alpha (last block).
// The body takes the block coordinates b (the hardware block, or a batch
// queue item standing for one block of this solve's launch).
template <int MODE>
__device__ __forceinline__ void matvec_body(const Blk& b, Geometry g, PcgState* st,
                                            const double* __restrict__ w,
                                            double* __restrict__ q,
                                            const double* __restrict__ T0,
                                            const double* __restrict__ T1,
                                            const double* __restrict__ T2,
                                            const double* __restrict__ D, double* partials,
                                            int par) {
  __shared__ double sh[32];
  __shared__ int flag;
  if (MODE == 1 && st->done) return;
  double dot = 0.0;
  const long long stride = (long long)b.nx * blockDim.x;
  for (long long c = (long long)b.x * blockDim.x + threadIdx.x; c < g.n; c += stride) {
    const int i = (int)(c % g.n0);
    const long long rem = c / g.n0;
    const int j = (int)(rem % g.n1);
    const int k = (int)(rem / g.n1);
    const long long cxm = (i > 0) ? c - 1 : c, cxp = (i < g.n0 - 1) ? c + 1 : c;
    const long long cym = (j > 0) ? c - g.n0 : c, cyp = (j < g.n1 - 1) ? c + g.n0 : c;
    const long long czm = (k > 0) ? c - g.plane : c, czp = (k < g.n2 - 1) ? c + g.plane : c;
    const double wc = w[c];
    double qv = D[c] * wc;
    qv = fma(-T0[c], w[cxm], qv);
    qv = fma(-T0[c + 1], w[cxp], qv);
    qv = fma(-T1[c], w[cym], qv);
    qv = fma(-T1[c + g.n0], w[cyp], qv);
    qv = fma(-T2[c], w[czm], qv);
    qv = fma(-T2[c + g.plane], w[czp], qv);
    q[c] = qv;
    if (MODE == 1) dot = fma(wc, qv, dot);
  }
  if (MODE == 1) {
    const double bs = block_sum(dot, sh);
    double v[1] = {bs};
    if (publish_values(partials, 1, v, 1, &st->cnt[kCntDot], &flag, b)) {
      const double dq = sum_partials(partials, (int)nblocks(b), 1, sh);
      if (threadIdx.x == 0) {
        const double alpha = st->rho / dq;
        st->dq = dq;
        st->alpha[par] = alpha;
        if (!(dq > 0.0) || !isfinite(alpha)) { st->status = kEBREAKDOWN; st->done = 1; }
        st->cnt[kCntDot] = 0;
      }
    }
  }
}
template <int MODE>
__global__ void __launch_bounds__(256) k_matvec(Geometry g, PcgState* st,
                                               const double* __restrict__ w,
                                               double* __restrict__ q,
                                               const double* __restrict__ T0,
                                               const double* __restrict__ T1,
                                               const double* __restrict__ T2,
                                               const double* __restrict__ D, double* partials,
                                               int par) {
  matvec_body<MODE>(hw_blk(), g, st, w, q, T0, T1, T2, D, partials, par);
}

// ------------------------------------------------------------------ double-float matvec
// The mixed-precision path's q = A w with the FP64-class arithmetic on the
// FP32 pipe: faces, Dirichlet planes, w and q as double-float pairs.  The
// operator is taken in its face-difference form
//   (Aw)_c = sum_f T_f (w_c - w_f) + [k = 0] B_in w_c + [k = n2-1] B_out w_c
// (Eq. scaled bilinear forms; the same operator as D w - sum T w with
// D = sum T + B), so no diagonal is read and no cancellation between D w and
// the neighbour terms occurs; the terms are summed by Sum2.  Each thread owns
// one (i, j) column of a 32 x 8 tile and marches over kchunk planes: w at k
// and k+1 stay in registers, and the flux through the face below plane k is
// the one computed through the face above plane k-1, negated.  The x/y
// neighbours come from the tile's own loads through L1.
// Neighbour offsets are the constants +-1 and +-n0 at every cell: where such
// a neighbour lies outside the box (or in the next/previous row) its face
// conductance is the zero of a Neumann face, so the value read only has to be
// finite.  w therefore needs n0 finite guard elements before w[0] and after
// w[n-1]; the z neighbour above the last plane is not read.
// MODE 1: also w.q (double-float partial per thread) -> alpha = rho / w.q.

// p + pe ~ T (a - b) for double-float T, a, b: the difference by TwoSum (plus
// the low parts), the product with hi*hi exact by FMA plus the cross terms
__device__ __forceinline__ void df_flux(float2 T, float2 a, float2 b, float& p, float& pe) {
  float dh, dl;
  two_sum(a.x, -b.x, dh, dl);
  dl += a.y - b.y;
  p = T.x * dh;
  pe = fma(T.x, dh, -p);
  pe = fma(T.x, dl, pe);
  pe = fma(T.y, dh, pe);
}
// Sum2 step (s, e) += p + pe
__device__ __forceinline__ void df_acc(float p, float pe, float& s, float& e) {
  float t;
  two_sum(s, p, s, t);
  e += t + pe;
}

template <int MODE>
__device__ __forceinline__ void matvec_df_body(const Blk& b, Geometry g, PcgState* st,
                                               const float* __restrict__ w,
                                               float2* __restrict__ q,
                                               const float2* __restrict__ T0,
                                               const float2* __restrict__ T1,
                                               const float2* __restrict__ T2,
                                               const float2* __restrict__ Bin,
                                               const float2* __restrict__ Bout,
                                               double* partials, int par, int kchunk) {
  __shared__ double sh[32];
  __shared__ int flag;
  if (MODE == 1 && st->done) return;
  const int i = b.x * 32 + (threadIdx.x & 31);
  const int j = b.y * 8 + (threadIdx.x >> 5);
  const int k0 = b.z * kchunk;
  const int k1 = min(k0 + kchunk, g.n2);
  float ds = 0.f, dc = 0.f;
  if (i < g.n0 && j < g.n1 && k0 < k1) {
    const int n0 = g.n0;
    const long long pl = g.plane;
    const long long sidx = (long long)j * n0 + i;
    const long long c0 = (long long)k0 * pl + sidx;
    // per-thread pointers, advanced by one plane per step
    const float* pw = w + c0;
    const float2* p0 = T0 + c0;
    const float2* p1 = T1 + c0;
    const float2* p2 = T2 + c0;
    float2* pq = q + c0;
    // Operands of plane k+1 are loaded during plane k (software pipelining):
    // every thread keeps a full plane's worth of loads in flight while it sums.
    struct Ops {
      float2 x0, x1, y0, y1, zp;
      float wx0, wx1, wy0, wy1, wp;
    };
    auto load = [&](bool last, float wself) {
      Ops o;
      o.x0 = p0[0];
      o.x1 = p0[1];
      o.y0 = p1[0];
      o.y1 = p1[n0];
      o.wx0 = pw[-1];
      o.wx1 = pw[1];
      o.wy0 = pw[-n0];
      o.wy1 = pw[n0];
      o.wp = last ? wself : pw[pl];
      o.zp = p2[pl];  // the extra zero plane covers k = n2 - 1
      return o;
    };
    // the FP32 direction as double-float values (low part 0)
    auto d2 = [](float v) { return make_float2(v, 0.f); };
    float wc = pw[0];
    float fz, fze;  // flux T2 (w_{k-1} - w_k) through the face below plane k
    df_flux(p2[0], d2(k0 > 0 ? pw[-pl] : wc), d2(wc), fz, fze);
    Ops cur = load(k0 == g.n2 - 1, wc);
    for (int k = k0; k < k1; ++k) {
      Ops nxt;
      pw += pl; p0 += pl; p1 += pl; p2 += pl;
      if (k + 1 < k1) nxt = load(k + 1 == g.n2 - 1, cur.wp);
      float sv, ev, p, pe;
      const float2 w2 = d2(wc);
      df_flux(cur.x0, w2, d2(cur.wx0), sv, ev);
      df_flux(cur.x1, w2, d2(cur.wx1), p, pe);
      df_acc(p, pe, sv, ev);
      df_flux(cur.y0, w2, d2(cur.wy0), p, pe);
      df_acc(p, pe, sv, ev);
      df_flux(cur.y1, w2, d2(cur.wy1), p, pe);
      df_acc(p, pe, sv, ev);
      df_acc(-fz, -fze, sv, ev);
      df_flux(cur.zp, w2, d2(cur.wp), fz, fze);
      df_acc(fz, fze, sv, ev);
      if (k == 0) df_fma_acc<1>(Bin[sidx], w2, sv, ev);
      if (k == g.n2 - 1) df_fma_acc<1>(Bout[sidx], w2, sv, ev);
      float qh, ql;
      two_sum(sv, ev, qh, ql);
      *pq = make_float2(qh, ql);
      pq += pl;
      if (MODE == 1) df_fma_acc<1>(w2, make_float2(qh, ql), ds, dc);
      wc = cur.wp;
      cur = nxt;
    }
  }
  if (MODE == 1) {
    const double bs = block_sum(widen(ds) + widen(dc), sh);
    double v[1] = {bs};
    if (publish_values(partials, 1, v, 1, &st->cnt[kCntDot], &flag, b)) {
      const double dq = sum_partials(partials, (int)nblocks(b), 1, sh);
      if (threadIdx.x == 0) {
        const double alpha = st->rho / dq;
        st->dq = dq;
        st->alpha[par] = alpha;
        if (!(dq > 0.0) || !isfinite(alpha)) { st->status = kEBREAKDOWN; st->done = 1; }
        st->cnt[kCntDot] = 0;
      }
    }
  }
}
template <int MODE>
__global__ void __launch_bounds__(256, 4) k_matvec_df(Geometry g, PcgState* st,
                                                     const float* __restrict__ w,
                                                     float2* __restrict__ q,
                                                     const float2* __restrict__ T0,
                                                     const float2* __restrict__ T1,
                                                     const float2* __restrict__ T2,
                                                     const float2* __restrict__ Bin,
                                                     const float2* __restrict__ Bout,
                                                     double* partials, int par, int kchunk) {
  matvec_df_body<MODE>(hw_blk(), g, st, w, q, T0, T1, T2, Bin, Bout, partials, par, kchunk);
}

// FP64 to double-float storage in place (8 bytes either way): the mixed
// path's residual after the initial right-hand side.  (The solution returns
// to FP64 in k_finish_x.)
__global__ void k_f64_to_df_inplace(double* a, long long n) {
  for (long long c = gidx(); c < n; c += (long long)gridDim.x * blockDim.x) {
    const float2 v = split_df(a[c]);
    reinterpret_cast<float2*>(a)[c] = v;
  }
}

// End of a solve (see PcgState::xpend): x += alpha w if the last residual
// update's step is still due, then, for double-float storage, x to FP64 in
// place.  x is viewed as V, w as W (FP32 directions with double-float x).
template <typename V, typename W>
__global__ void k_finish_x(Geometry g, const PcgState* st, V* x, const W* w) {
  const int pend = st->xpend;
  const typename Scalar<V>::T alpha = Scalar<V>::from(pend ? st->alpha[pend - 1] : 0.0);
  for (long long c = gidx(); c < g.n; c += (long long)gridDim.x * blockDim.x) {
    V v = x[c];
    if (pend) v = xaxpy(alpha, w[c], v);
    store_f64(reinterpret_cast<double*>(x) + c, v);
  }
}

// The diagonal of A (Eq. scaled bilinear forms): the six faces of each cell
// (the minus faces at c, the plus faces as the minus faces of the neighbours;
// zero on Neumann faces and in the extra plane) plus the Dirichlet terms, then
// the double-float copies of T0, T1, T2 and of B_in, B_out (FB: the two
// planes one after the other) for the mixed-precision matvec.
// Grid: blockIdx.y = plane k (n2 planes and the extra zero plane).
__global__ void k_diag_split(Geometry g, const double* __restrict__ T0,
                             const double* __restrict__ T1, const double* __restrict__ T2,
                             const double* __restrict__ Bin, const double* __restrict__ Bout,
                             double* __restrict__ D, float2* __restrict__ F0,
                             float2* __restrict__ F1, float2* __restrict__ F2,
                             float2* __restrict__ FB) {
  const int k = blockIdx.y;
  const int sidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (sidx >= g.plane) return;
  const long long c = (long long)k * g.plane + sidx;
  F0[c] = split_df(T0[c]);
  F1[c] = split_df(T1[c]);
  F2[c] = split_df(T2[c]);
  if (k == g.n2) return;  // the extra plane has faces only
  const double t0 = T0[c], t1 = T1[c], t2 = T2[c];
  const double p0 = T0[c + 1], p1 = T1[c + g.n0], p2 = T2[c + g.plane];
  double d = t0 + p0 + t1 + p1 + t2 + p2;
  if (k == 0) {
    d += Bin[sidx];
    FB[sidx] = split_df(Bin[sidx]);
  }
  if (k == g.n2 - 1) {
    d += Bout[sidx];
    FB[g.plane + sidx] = split_df(Bout[sidx]);
  }
  D[c] = d;
}

// Double-float copies of FP64 arrays (split_df per element).
__global__ void k_split_df(const double* __restrict__ a, float2* __restrict__ b, long long n) {
  for (long long c = gidx(); c < n; c += (long long)gridDim.x * blockDim.x) b[c] = split_df(a[c]);
}

// ------------------------------------------------------------------ forward DCT along axis 0
// MODE 0: initial residual (r = b already): ||r||^2 -> ||b||^2.
// MODE 1: PCG update r -= alpha q, ||r||^2 -> convergence test, and
//         x += alpha w for FP64 storage; with double-float storage the x step
//         follows in the w-update kernel, which reads w anyway (the FP64 path
//         keeps it here: its w-update kernel is FP64-bound).
// MODE 2: transform only (component entry point), no state; input rin (FP64).
// V: storage of x, w, q, r (double, or float2 double-float pairs).
template <typename R, int MODE, typename V>
__global__ void __launch_bounds__(256) k_fwd_x(Geometry g, DctPlan<R> p, PcgState* st,
                                              V* __restrict__ x, const V* __restrict__ w,
                                              const V* __restrict__ q, V* __restrict__ r,
                                              const double* __restrict__ rin,
                                              R* __restrict__ t, double* partials, int L, int par,
                                              double rtol2) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32];
  __shared__ int flag;
  if (MODE != 2 && st->done) return;
  const Lay y = make_lay(L, g.n0, false);
  c2<R>* a = reinterpret_cast<c2<R>*>(smraw);
  c2<R>* b = a + L * dct_half_alloc(g.n0);
  const long long nrows = (long long)g.n1 * g.n2;
  const long long row0 = (long long)blockIdx.x * L;
  using S = Scalar<V>;
  constexpr bool XHERE = (MODE == 1) && std::is_same<V, double>::value;
  const typename S::T alpha = S::from((MODE == 1) ? st->alpha[par] : 0.0);
  const typename S::T nalpha = S::neg(alpha);
  double acc = 0.0;
  float accf = 0.f;
  const int tot = L * g.n0;
  // U elements per thread per round: their loads are all issued before use
  constexpr int U = 4;
  for (int e0 = threadIdx.x; e0 < tot; e0 += U * blockDim.x) {
    V rv[U], qv[U], xv[U], wv[U];
    double dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      const int l = e / g.n0, i = e - l * g.n0;
      const long long row = row0 + l;
      rv[u] = vzero<V>(); qv[u] = rv[u];
      dv[u] = 0.0;
      if (e < tot && row < nrows) {
        const long long c = row * g.n0 + i;
        if (MODE == 2) dv[u] = rin[c];
        else rv[u] = r[c];
        if (MODE == 1) qv[u] = q[c];
        if (XHERE) { xv[u] = x[c]; wv[u] = w[c]; }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e >= tot) break;
      const int l = e / g.n0, i = e - l * g.n0;
      const long long row = row0 + l;
      R in;
      if (MODE == 2) {
        in = from_f64<R>(dv[u]);
      } else {
        V v = rv[u];
        if (row < nrows) {
          const long long c = row * g.n0 + i;
          if (MODE == 1) {
            if (XHERE) x[c] = vaxpy(alpha, wv[u], xv[u]);
            v = vaxpy(nalpha, qv[u], v);
            r[c] = v;
          }
          vsq_acc(v, acc, accf);
        }
        in = vround<R>(v);
      }
      dct2_put<R>(p.s, y, a, l, i, in);
    }
  }
  __syncthreads();
  dct2_run<R>(p, y, a, b, [&](int l, int k, R v) {
    const long long row = row0 + l;
    if (row < nrows) t[row * g.n0 + k] = v;
  });
  if (MODE != 2)
    fwd_x_residual_tail<MODE>(acc + widen(accf), st, partials, rtol2, sh, &flag, par, !XHERE);
}

// ------------------------------------------------------------------ DCT along axis 1 (in place)
template <typename R, int INVERSE>
__global__ void __launch_bounds__(256) k_dct_y(Geometry g, DctPlan<R> p, const PcgState* st,
                                              R* __restrict__ t, int TI, int check) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (check && st->done) return;
  const Lay y = make_lay(TI, g.n1, true);
  c2<R>* a = reinterpret_cast<c2<R>*>(smraw);
  c2<R>* b = a + TI * dct_half_alloc(g.n1);
  const long long k = blockIdx.y;
  const int i0 = blockIdx.x * TI;
  R* base = t + k * g.plane + i0;
  const int tot = TI * g.n1;
  constexpr int U = 8;
  for (int e0 = threadIdx.x; e0 < tot; e0 += U * blockDim.x) {
    R v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      const int l = e % TI, jj = e / TI;
      v[u] = (e < tot && i0 + l < g.n0) ? base[(long long)jj * g.n0 + l] : (R)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e >= tot) break;
      const int l = e % TI, jj = e / TI;
      if (INVERSE) dct3_put<R>(y, b, l, jj, v[u]);
      else dct2_put<R>(p.s, y, a, l, jj, v[u]);
    }
  }
  __syncthreads();
  auto store = [&](int l, int kk, R v) {
    if (i0 + l < g.n0) base[(long long)kk * g.n0 + l] = v;
  };
  if (INVERSE) dct3_run<R>(p, y, a, b, (R)1, store);
  else dct2_run<R>(p, y, a, b, store);
}

// ------------------------------------------------------------------ tridiagonal along axis 2
// Forward sweep y_k = r^_k + h_{k-1} y_{k-1}, backward z_k = h_k (y_k + z_{k+1})
// solves (T_{i'j'}/kappa_ref^z) z = r^.  The forward sweep stores g_k = h_k y_k,
// so that the backward sweep is one FMA per cell, z_k = g_k + h_k z_{k+1}
// (four FP64 instructions per cell for both sweeps and rho, not five).  r^.T^{-1} r^ = sum_k h_k y_k^2 / kappa_ref^z,
// so rho = r.z follows from Parseval for the DCT pair of Sec. 3.2 (weight
// 4 alpha_i' alpha_j' / (n0 n1), applied in the last block through wscale).
// MODE 0: solve only.
// MODE 1: plain PCG, rho_new -> beta = rho_new / rho.
// MODE 2: flexible PCG: keeps r^ of this iteration in rnew and reads that of
//         the previous one from rold, so that z_new . r_old (Parseval again)
//         gives the Polak-Ribiere beta = (rho_new - z_new . r_old) / rho.
// MODE 3: flexible PCG, initial apply: stores r^ in rnew, beta = 0.
template <typename R, int MODE>
__device__ __forceinline__ void tridiag_body(const Blk& b, Geometry g, PcgState* st,
                                             R* __restrict__ t, const R* __restrict__ h,
                                             double w4, const double* kd, double kz_host,
                                             double* partials, R* __restrict__ rnew,
                                             const R* __restrict__ rold) {
  __shared__ double sh[32];
  __shared__ int flag;
  if (MODE != 0 && st->done) return;
  const long long s = (long long)b.x * blockDim.x + threadIdx.x;
  double acc = 0.0, acc2 = 0.0;
  if (s < g.plane) {
    // P planes per round (4 in FP64, 8 in FP32, the faster depths measured):
    // the loads of a round are issued before the recurrence uses them
    constexpr int P = sizeof(R) == 8 ? 4 : 8;
    R yv = (R)0, hp = (R)0, part = (R)0, zr = (R)0;
    for (int kb = 0; kb < g.n2; kb += P) {
      R tv[P], hv[P];
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int k = kb + u;
        if (k < g.n2) {
          const long long c = (long long)k * g.plane + s;
          tv[u] = t[c];
          hv[u] = h[c];
        }
      }
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int k = kb + u;
        if (k < g.n2) {
          const long long c = (long long)k * g.plane + s;
          if (MODE >= 2) rnew[c] = tv[u];
          yv = fma(hp, yv, tv[u]);
          const R gv = hv[u] * yv;  // g_k = h_k y_k, kept for the backward sweep
          t[c] = gv;
          part = fma(gv, yv, part);
          hp = hv[u];
        }
      }
    }
    R zn = (R)0;
    for (int kb = g.n2 - 1; kb >= 0; kb -= P) {
      R tv[P], hv[P], ro[P];
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int k = kb - u;
        if (k >= 0) {
          const long long c = (long long)k * g.plane + s;
          tv[u] = t[c];
          hv[u] = h[c];
          if (MODE == 2) ro[u] = rold[c];
        }
      }
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int k = kb - u;
        if (k >= 0) {
          zn = fma(hv[u], zn, tv[u]);  // z_k = h_k (y_k + z_{k+1}) = g_k + h_k z_{k+1}
          t[(long long)k * g.plane + s] = zn;
          if (MODE == 2) zr = fma(zn, ro[u], zr);
        }
      }
    }
    const int i = (int)(s % g.n0), j = (int)(s / g.n0);
    const double wgt = (i == 0 ? 0.5 : 1.0) * (j == 0 ? 0.5 : 1.0);
    acc = wgt * to_f64<R>(part);
    if (MODE == 2) acc2 = wgt * to_f64<R>(zr);
  }
  if (MODE != 0) tridiag_tail<MODE>(acc, acc2, st, partials, w4, kd, kz_host, sh, &flag, b);
}
template <typename R, int MODE>
__global__ void __launch_bounds__(128) k_tridiag(Geometry g, PcgState* st, R* __restrict__ t,
                                                const R* __restrict__ h, double w4,
                                                const double* kd, double kz_host,
                                                double* partials, R* __restrict__ rnew,
                                                const R* __restrict__ rold) {
  tridiag_body<R, MODE>(hw_blk(), g, st, t, h, w4, kd, kz_host, partials, rnew, rold);
}

// ------------------------------------------------------------------ tridiagonal, FP32, pivots on the fly
// The FP32 form of the solves above for the mixed-precision paths, without a
// pivot table.  The pivots of T_{i'j'}/kappa_ref^z depend on the column only
// through sigma = s_{i'j'}/kappa_ref^z and the Dirichlet corners (Sec. 3.2:
// diagonal sigma + 2 inside, sigma + 1 + 2 kappa_in/kappa_z at k = 0 and
// sigma + 1 + 2 kappa_out/kappa_z at k = n2-1), so each thread generates them
// as it sweeps.  The pivot is carried as d_k = 1 + e_k with
//   e_0 = sigma + a_in,   e_k = sigma + e_{k-1} h_{k-1},   h_k = 1 / (1 + e_k)
// (the recurrence d_k = a - 1/d_{k-1} rewritten with 1 - h = e h), and the
// last pivot as d = sigma + a_out + e h.  Every term is positive, so no
// cancellation occurs: for the slowly converging low modes (sigma -> 0) the
// direct FP32 form a - h_{k-1} loses up to 1e-2 of the solution over 1000
// planes, this form stays within a few 1e-6, as the FP64 table rounded to FP32.
// The forward sweep keeps the state (e, y) at the start of every chunk of
// kTriChunk planes in ck; the backward sweep walks the chunks downwards,
// regenerates each chunk's h_k and y_k from its checkpoint in registers (the
// same operations on the same values, so bit-identical) and runs
// z_k = h_k (y_k + z_{k+1}) down it.
// Traffic per cell: r^ twice, z once (and r_old once for MODE 2) plus
// 2 x 8 / kTriChunk bytes of checkpoints, against r^, y twice, h twice, z
// (and r_new, r_old) for the table-driven kernel.  in and out may be the same
// buffer: each chunk's r^ (and the next lower chunk's, prefetched) is read
// before the chunk's z is written, and the chunks below are read later.
// ck holds (ceil(n2 / kTriChunk) - 1) * plane pairs.
// MODE as k_tridiag; MODE 2 reads r_old (the previous iteration's r^, kept by
// the caller) for z_new . r_old.
// MINB 8 caps the registers at 64 so that 8 blocks fit on an SM (for planes
// with more columns than 6 blocks of 128 threads on every SM; measured 0.55 ->
// 0.49 ms at 512^3); smaller planes are latency-bound and keep the
// unconstrained allocation (a few spilled registers cost 5-10 % there).
template <int MODE>
__device__ __forceinline__ void tridiag_otf_body(const Blk& b, Geometry g, PcgState* st,
                                                 const float* in, float* out,
                                                 float2* __restrict__ ck,
                                                 const double* __restrict__ lam0,
                                                 const double* __restrict__ lam1,
                                                 const double* __restrict__ kd, double w4,
                                                 double* partials,
                                                 const float* __restrict__ rold) {
  __shared__ double sh[32];
  __shared__ float coef[4];
  __shared__ int flag;
  if (MODE != 0 && st->done) return;
  if (threadIdx.x == 0) tri_coef(kd, coef);  // kappa_ref ratios, once per block
  __syncthreads();
  const long long s = (long long)b.x * blockDim.x + threadIdx.x;
  double acc = 0.0, acc2 = 0.0;
  if (s < g.plane) {
    const int i = (int)(s % g.n0), j = (int)(s / g.n0);
    const TriCol a = tri_col(i, j, g.n2, lam0, lam1, coef);
    const int n2 = g.n2;
    const int nch = (n2 + kTriChunk - 1) / kTriChunk;
    const long long pl = g.plane;
    // Each sweep loads the next chunk's operands before it runs the
    // recurrence of the current one (one chunk of loads always in flight).
    float e = 0.f, h = 0.f, y = 0.f, part = 0.f;
    float tv[kTriChunk];
#pragma unroll
    for (int u = 0; u < kTriChunk; ++u)
      if (u < n2) tv[u] = in[(long long)u * pl + s];
    for (int ch = 0; ch < nch; ++ch) {
      const int kb = ch * kTriChunk;
      float tn[kTriChunk];
      if (ch + 1 < nch) {
#pragma unroll
        for (int u = 0; u < kTriChunk; ++u)
          if (kb + kTriChunk + u < n2) tn[u] = in[(long long)(kb + kTriChunk + u) * pl + s];
      }
      if (ch > 0) ck[(long long)(ch - 1) * pl + s] = make_float2(e, y);
#pragma unroll
      for (int u = 0; u < kTriChunk; ++u) {
        const int k = kb + u;
        if (k < n2) {
          tri_step(a, k, n2, tv[u], e, h, y);
          part = fmaf(h * y, y, part);
        }
      }
#pragma unroll
      for (int u = 0; u < kTriChunk; ++u) tv[u] = tn[u];
    }
    float zn = 0.f, zr = 0.f;
    // operands of chunk ch: r^ (tv), r_old (ro) and the checkpoint (cp)
    float ro[kTriChunk];
    float2 cp = make_float2(0.f, 0.f);
    auto load_chunk = [&](int ch, float* t_, float* r_, float2& c_) {
      const int kb = ch * kTriChunk;
#pragma unroll
      for (int u = 0; u < kTriChunk; ++u)
        if (kb + u < n2) {
          t_[u] = in[(long long)(kb + u) * pl + s];
          if (MODE == 2) r_[u] = rold[(long long)(kb + u) * pl + s];
        }
      c_ = ch > 0 ? ck[(long long)(ch - 1) * pl + s] : make_float2(0.f, 0.f);
    };
    load_chunk(nch - 1, tv, ro, cp);
    for (int ch = nch - 1; ch >= 0; --ch) {
      const int kb = ch * kTriChunk;
      float tn[kTriChunk], rn[kTriChunk];
      float2 cn;
      if (ch > 0) load_chunk(ch - 1, tn, rn, cn);
      // state before the chunk: h = 1 / (1 + e) as the forward sweep formed it
      float ec = cp.x, yc = cp.y, hc = ch > 0 ? tri_rcp(1.0f + cp.x) : 0.f;
      float hv[kTriChunk], yv[kTriChunk];
#pragma unroll
      for (int u = 0; u < kTriChunk; ++u) {
        const int k = kb + u;
        if (k < n2) {
          tri_step(a, k, n2, tv[u], ec, hc, yc);
          hv[u] = hc;
          yv[u] = yc;
        }
      }
#pragma unroll
      for (int u = kTriChunk - 1; u >= 0; --u) {
        const int k = kb + u;
        if (k < n2) {
          zn = hv[u] * (yv[u] + zn);
          out[(long long)k * pl + s] = zn;
          if (MODE == 2) zr = fmaf(zn, ro[u], zr);
        }
      }
      if (ch > 0) {
#pragma unroll
        for (int u = 0; u < kTriChunk; ++u) {
          tv[u] = tn[u];
          if (MODE == 2) ro[u] = rn[u];
        }
        cp = cn;
      }
    }
    const double wgt = (i == 0 ? 0.5 : 1.0) * (j == 0 ? 0.5 : 1.0);
    acc = wgt * widen(part);
    if (MODE == 2) acc2 = wgt * widen(zr);
  }
  if (MODE != 0) tridiag_tail<MODE>(acc, acc2, st, partials, w4, kd, 1.0, sh, &flag, b);
}
template <int MODE, int MINB>
__global__ void __launch_bounds__(128, MINB) k_tridiag_otf(Geometry g, PcgState* st, const float* in,
                                                    float* out, float2* __restrict__ ck,
                                                    const double* __restrict__ lam0,
                                                    const double* __restrict__ lam1,
                                                    const double* __restrict__ kd, double w4,
                                                    double* partials,
                                                    const float* __restrict__ rold) {
  tridiag_otf_body<MODE>(hw_blk(), g, st, in, out, ck, lam0, lam1, kd, w4, partials, rold);
}

// ------------------------------------------------------------------ backward DCT along axis 0
// u = scale * (backward DCT of t along axis 0), then by MODE:
// 0: z = u (TZ).
// 2: PCG: w = u + beta w in place (z points at w, FP64 or double-float;
//    beta from the tridiagonal kernel), so the next matvec reads w directly;
//    with x given, first x += alpha w with the old w (this iteration's step),
//    which clears the pending mark of the residual-update kernel.
template <typename R, typename TZ, int MODE>
__global__ void __launch_bounds__(256) k_inv_x(Geometry g, DctPlan<R> p, PcgState* st,
                                              const R* __restrict__ t, TZ* __restrict__ z,
                                              const double* kd, double kz_host, int L,
                                              int check, typename XOf<TZ>::T* __restrict__ x, int par) {
  using TX = typename XOf<TZ>::T;  // x's storage (FP32 directions: double-float x)
  extern __shared__ __align__(16) unsigned char smraw[];
  if (check && st->done) return;
  const Lay y = make_lay(L, g.n0, false);
  c2<R>* a = reinterpret_cast<c2<R>*>(smraw);
  c2<R>* b = a + L * dct_half_alloc(g.n0);
  // MODE 2: the old w of the block's rows, staged with the transform input
  TZ* wsh = reinterpret_cast<TZ*>(b + L * dct_half_alloc(g.n0));
  const long long nrows = (long long)g.n1 * g.n2;
  const long long row0 = (long long)blockIdx.x * L;
  const int tot = L * g.n0;
  const bool upd = (MODE == 2) && x != nullptr;
  const typename Scalar<TX>::T alpha = Scalar<TX>::from(upd ? st->alpha[par] : 0.0);
  if (upd && blockIdx.x == 0 && threadIdx.x == 0) st->xpend = 0;
  constexpr int U = 8;
  for (int e0 = threadIdx.x; e0 < tot; e0 += U * blockDim.x) {
    R v[U];
    TZ wv[U];
    TX xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      const int l = e / g.n0, k = e - l * g.n0;
      const bool ok = (e < tot && row0 + l < nrows);
      v[u] = ok ? t[(row0 + l) * g.n0 + k] : (R)0;
      if (MODE == 2) wv[u] = ok ? z[(row0 + l) * g.n0 + k] : vzero<TZ>();
      if (MODE == 2 && upd && ok) xv[u] = x[(row0 + l) * g.n0 + k];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e >= tot) break;
      const int l = e / g.n0, k = e - l * g.n0;
      dct3_put<R>(y, b, l, k, v[u]);
      if (MODE == 2) wsh[e] = wv[u];
      if (MODE == 2 && upd && row0 + l < nrows)
        x[(row0 + l) * g.n0 + k] = xaxpy(alpha, wv[u], xv[u]);
    }
  }
  __syncthreads();
  const typename Scalar<TZ>::T beta = Scalar<TZ>::from((MODE == 2) ? st->beta : 0.0);
  const R scale = (R)(1.0 / (kd ? kd[2] : kz_host));
  dct3_run<R>(p, y, a, b, scale, [&](int l, int i, R v) {
    const long long row = row0 + l;
    if (row < nrows) {
      const long long c = row * g.n0 + i;
      if (MODE == 2) z[c] = vaxpy(beta, wsh[l * g.n0 + i], vfrom<TZ, R>(v));
      else z[c] = vfrom<TZ, R>(v);
    }
  });
}

// ------------------------------------------------------------------ post-processing
// Sums for Eq. (flux) / Eq. (effective formula dis) in the loading frame:
// res[0..2] internal-face flux sums T (p_minus - p_plus) per axis (times h later),
// res[3] = sum b_out (p_{n2-1} - p_out), res[4] = sum b_in (p_in - p_0).
__global__ void k_flux(Geometry g, const double* __restrict__ x, const double* __restrict__ T0,
                       const double* __restrict__ T1, const double* __restrict__ T2,
                       const double* __restrict__ Bin, const double* __restrict__ Bout,
                       double pin, double pout, double* partials, PcgState* st) {
  __shared__ double sh[32];
  __shared__ int flag;
  double a[5] = {0, 0, 0, 0, 0};
  for (long long c = gidx(); c < g.n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n0);
    const long long rem = c / g.n0;
    const int j = (int)(rem % g.n1), k = (int)(rem / g.n1);
    const double xc = x[c];
    if (i > 0) a[0] = fma(T0[c], x[c - 1] - xc, a[0]);
    if (j > 0) a[1] = fma(T1[c], x[c - g.n0] - xc, a[1]);
    if (k > 0) a[2] = fma(T2[c], x[c - g.plane] - xc, a[2]);
    const long long s = c - (long long)k * g.plane;
    if (k == g.n2 - 1) a[3] = fma(Bout[s], xc - pout, a[3]);
    if (k == 0) a[4] = fma(Bin[s], pin - xc, a[4]);
  }
  double vals[5];
  for (int e = 0; e < 5; ++e) vals[e] = block_sum(a[e], sh);
  if (publish_values(partials, 5, vals, 5, &st->cnt[kCntFlux], &flag)) {
    double tot[5];
    for (int e = 0; e < 5; ++e) tot[e] = sum_partials(partials + e, (int)nblocks(), 5, sh);
    if (threadIdx.x == 0) {
      for (int e = 0; e < 5; ++e) st->res[e] = tot[e];
      st->cnt[kCntFlux] = 0;
    }
  }
}

// ||b - A x||^2 -> res[5] (true residual at exit).
__global__ void k_true_residual(Geometry g, const double* __restrict__ x,
                                const double* __restrict__ T0, const double* __restrict__ T1,
                                const double* __restrict__ T2, const double* __restrict__ D,
                                const double* __restrict__ Bin, const double* __restrict__ Bout,
                                double pin, double pout, const double* __restrict__ pin_f,
                                const double* __restrict__ pout_f,
                                const double* __restrict__ src, double* partials, PcgState* st) {
  __shared__ double sh[32];
  __shared__ int flag;
  double acc = 0.0, en = 0.0;
  for (long long c = gidx(); c < g.n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n0);
    const long long rem = c / g.n0;
    const int j = (int)(rem % g.n1), k = (int)(rem / g.n1);
    const long long s = c - (long long)k * g.plane;
    const double xc = x[c];
    const double ein = k == 0 ? xc - (pin_f ? pin_f[s] : pin) : 0.0;
    const double eout = k == g.n2 - 1 ? xc - (pout_f ? pout_f[s] : pout) : 0.0;
    double b = src ? src[c] : 0.0;
    if (k == 0) b += Bin[s] * (pin_f ? pin_f[s] : pin);
    if (k == g.n2 - 1) b += Bout[s] * (pout_f ? pout_f[s] : pout);
    double ax = D[c] * xc;
    if (i > 0) ax -= T0[c] * x[c - 1];
    if (i < g.n0 - 1) ax -= T0[c + 1] * x[c + 1];
    if (j > 0) ax -= T1[c] * x[c - g.n0];
    if (j < g.n1 - 1) ax -= T1[c + g.n0] * x[c + g.n0];
    if (k > 0) ax -= T2[c] * x[c - g.plane];
    if (k < g.n2 - 1) ax -= T2[c + g.plane] * x[c + g.plane];
    const double d = b - ax;
    acc = fma(d, d, acc);
    // the energy x.Ax - 2 b.x + sum B p^2 as its sum of positive face terms:
    // every internal face once (the minus face of each cell) and the
    // Dirichlet faces, T (x_c - x_nb)^2 and B (x - p)^2
    if (i > 0) { const double t = xc - x[c - 1]; en = fma(T0[c] * t, t, en); }
    if (j > 0) { const double t = xc - x[c - g.n0]; en = fma(T1[c] * t, t, en); }
    if (k > 0) { const double t = xc - x[c - g.plane]; en = fma(T2[c] * t, t, en); }
    if (k == 0) en = fma(Bin[s] * ein, ein, en);
    if (k == g.n2 - 1) en = fma(Bout[s] * eout, eout, en);
  }
  double v[2];
  v[0] = block_sum(acc, sh);
  v[1] = block_sum(en, sh);
  if (publish_values(partials, 2, v, 2, &st->cnt[kCntAux], &flag)) {
    const double tot = sum_partials(partials, (int)nblocks(), 2, sh);
    const double etot = sum_partials(partials + 1, (int)nblocks(), 2, sh);
    if (threadIdx.x == 0) {
      st->res[5] = tot;
      st->res[6] = etot;
      st->cnt[kCntAux] = 0;
    }
  }
}

// ------------------------------------------------------------------ adjoint gradient
// d kappa_eff / d log kappa^a per cell (loading frame), from the forward field
// x and the adjoint field lam (A lam = cJ b_out on the last plane):
//   internal face T = 2ab/(a+b) between this cell (a) and a neighbour (b):
//     dT/dlog a = T b/(a+b), contribution -dT (x_c - x_nb)(lam_c - lam_nb);
//   Dirichlet faces B = 2 kappa~^z (d/dlog = B):
//     plane 0:      B lam (p_in - x);
//     plane n2-1:   cJ B (x - p_out) + B lam (p_out - x).
// summed != 0 writes G0 = sum over the three components.
__global__ void k_gradient(Geometry g, const double* __restrict__ x,
                           const double* __restrict__ lam, const double* __restrict__ k0,
                           const double* __restrict__ k1, const double* __restrict__ k2,
                           double ih0, double ih1, double ih2, const double* __restrict__ T0,
                           const double* __restrict__ T1, const double* __restrict__ T2,
                           double pin, double pout, double cJ, double* __restrict__ G0,
                           double* __restrict__ G1, double* __restrict__ G2, int summed) {
  for (long long c = gidx(); c < g.n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n0);
    const long long rem = c / g.n0;
    const int j = (int)(rem % g.n1), k = (int)(rem / g.n1);
    const double xc = x[c], lc = lam[c];
    double gg[3] = {0.0, 0.0, 0.0};
    const double* kk[3] = {k0, k1, k2};
    const double* TT[3] = {T0, T1, T2};
    const double ih[3] = {ih0, ih1, ih2};
    const long long st[3] = {1, g.n0, g.plane};
    const int idx[3] = {i, j, k};
    const int nn[3] = {g.n0, g.n1, g.n2};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const double a = kk[ax][c] * ih[ax];
      if (idx[ax] > 0) {
        const long long m = c - st[ax];
        const double b = kk[ax][m] * ih[ax];
        const double dT = TT[ax][c] * b / (a + b);
        gg[ax] -= dT * (xc - x[m]) * (lc - lam[m]);
      }
      if (idx[ax] < nn[ax] - 1) {
        const long long m = c + st[ax];
        const double b = kk[ax][m] * ih[ax];
        const double dT = TT[ax][m] * b / (a + b);
        gg[ax] -= dT * (xc - x[m]) * (lc - lam[m]);
      }
    }
    const double B = 2.0 * k2[c] * ih2;
    if (k == 0) gg[2] += B * lc * (pin - xc);
    if (k == g.n2 - 1) gg[2] += cJ * B * (xc - pout) + B * lc * (pout - xc);
    if (summed) {
      G0[c] = gg[0] + gg[1] + gg[2];
    } else {
      G0[c] = gg[0]; G1[c] = gg[1]; G2[c] = gg[2];
    }
  }
}

// Integer-pipe conversions applied element-wise (test support).
__global__ void k_convert(const float* __restrict__ fin, double* __restrict__ dout,
                          const double* __restrict__ din, float* __restrict__ fout,
                          long long n) {
  for (long long c = gidx(); c < n; c += (long long)gridDim.x * blockDim.x) {
    dout[c] = widen(fin[c]);
    fout[c] = narrow(din[c]);
  }
}

// Element-wise FP32 -> FP64 copy (component entry points of the mixed path).
__global__ void k_widen(const float* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long c = gidx(); c < n; c += (long long)gridDim.x * blockDim.x) b[c] = (double)a[c];
}

// ================================================================== launchers
static unsigned long long g_launches = 0;  // kernels launched by this library
unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
void count_launch() { __atomic_fetch_add(&g_launches, 1ull, __ATOMIC_RELAXED); }

static inline unsigned int grid_for(long long n, int bs, int cap = 148 * 32) {
  long long gb = (n + bs - 1) / bs;
  if (gb > cap) gb = cap;
  if (gb < 1) gb = 1;
  return (unsigned int)gb;
}

cudaError_t launch_kappa_stats(const double* a, long long n, double* partials, PcgState* st,
                               int slot, cudaStream_t s) {
  k_kappa_stats<<<grid_for(n, 256, 148 * 8), 256, 0, s>>>(a, n, partials, st, slot);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_permute(const double* in, double* out, int d0, int d1, int d2, long long s0,
                           long long s1, long long s2, cudaStream_t s) {
  const long long n = (long long)d0 * d1 * d2;
  if (s0 == 1) {
    k_permute_direct<<<grid_for(n, 256), 256, 0, s>>>(in, out, d0, d1, d2, s1, s2);
  } else {
    const int f = (s1 == 1) ? 1 : 2;
    const int df = (f == 1) ? d1 : d2;
    const int dother = (f == 1) ? d2 : d1;
    const long long so = (f == 1) ? s2 : s1;
    dim3 grid((d0 + 31) / 32, (df + 31) / 32, dother);
    k_permute_tile<<<grid, 256, 0, s>>>(in, out, d0, d1, d2, s0, so, f);
  }
  count_launch();
  return cudaGetLastError();
}

// planes x row blocks of the face assembly, capped near 8 blocks per SM so that
// the last block's extrema reduction stays short
static dim3 faces_grid(const Geometry& g) {
  long long bx = (g.plane + 255) / 256;
  if (bx > 148 * 8) bx = 148 * 8;
  long long by = (148 * 8) / bx;
  if (by < 1) by = 1;
  if (by > g.n2) by = g.n2;
  return dim3((unsigned int)bx, (unsigned int)by);
}

cudaError_t launch_faces(const Geometry& g, double ih0, double ih1, double ih2, const double* k0,
                         const double* k1, const double* k2, double* T0, double* T1, double* T2,
                         double* D, double* Bin, double* Bout, double* partials, PcgState* st,
                         cudaStream_t s) {
  k_faces<<<faces_grid(g), 256, 0, s>>>(g, ih0, ih1, ih2, k0, k1, k2, T0, T1, T2, D, Bin, Bout,
                                        partials, st);
  count_launch();
  return cudaGetLastError();
}

unsigned int faces_blocks(const Geometry& g) {
  const dim3 d = faces_grid(g);
  return d.x * d.y;
}

cudaError_t launch_diag_split(const Geometry& g, const double* T0, const double* T1,
                              const double* T2, const double* Bin, const double* Bout, double* D,
                              float2* F0, float2* F1, float2* F2, float2* FB, cudaStream_t s) {
  const dim3 grid((unsigned int)((g.plane + 255) / 256), (unsigned int)g.n2 + 1);
  k_diag_split<<<grid, 256, 0, s>>>(g, T0, T1, T2, Bin, Bout, D, F0, F1, F2, FB);
  count_launch();
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pivots(const Geometry& g, const double* lam0, const double* lam1,
                          const double* kref_dev, const double* kref_host, R* h, cudaStream_t s) {
  const double* k = kref_host;
  const double z[5] = {1, 1, 1, 1, 1};
  if (!k) k = z;
  k_pivots<R><<<grid_for(g.plane, 128, 1 << 30), 128, 0, s>>>(g, lam0, lam1, kref_dev, k[0], k[1],
                                                             k[2], k[3], k[4], h);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_pivots<double>(const Geometry&, const double*, const double*,
                                           const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_pivots<float>(const Geometry&, const double*, const double*,
                                          const double*, const double*, float*, cudaStream_t);

cudaError_t launch_select_kref(PcgState* st, int mode, const double* user, cudaStream_t s) {
  k_select_kref<<<1, 32, 0, s>>>(st, mode, user[0], user[1], user[2], user[3], user[4]);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_state_reset(PcgState* st, int maxit, cudaStream_t s) {
  k_state_reset<<<1, 32, 0, s>>>(st, maxit);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_loop_control(PcgState* st, cudaGraphConditionalHandle handle,
                                cudaStream_t s) {
  k_loop_control<<<1, 32, 0, s>>>(st, handle);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_init(const Geometry& g, const double* Bin, const double* Bout, double pin,
                        double pout, double* r, double* x, double* w0, cudaStream_t s,
                        const double* pin_f, const double* pout_f, const double* src) {
  k_init<<<grid_for(g.n, 256), 256, 0, s>>>(g, Bin, Bout, pin, pout, pin_f, pout_f, src, r, x, w0);
  count_launch();
  return cudaGetLastError();
}

unsigned int matvec_blocks(const Geometry& g) { return grid_for(g.n, 256, 148 * 16); }
// 32 x 8 (i, j) tiles, each tile column split into chunks of kc planes (a
// block's first plane costs three extra w loads and one extra face flux, which
// short chunks do not amortise).  Three regimes, from sweeps of the chunk count
// of the bulk-tensor kernel (6 resident blocks per SM) at 64^3 .. 512^3:
//  * 8-plane chunks still fit in one wave of resident blocks (64^3, 96^3):
//    kc = 8, the most blocks;
//  * the tiles fit in one wave with chunks of at most 48 planes (128^3 ..
//    192^3): one wave, chunks of at least 16 planes (128^3 34.0 -> 30.6 us,
//    160^3 48.9 -> 45.4, 192^3 66.2 -> 63.1 against 8/16-plane chunks);
//  * otherwise about 32 blocks per SM, chunks of at least 20 planes (256^3
//    129.4 -> 123 us against 16; 512^3 keeps 128-plane chunks, within 1 % of
//    every count from 3 to 8 chunks per column).
dim3 matvec_df_grid(const Geometry& g, int* kchunk) {
  static const long long sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      (void)cudaGetLastError();
      return 148LL;
    }
    return (long long)n;
  }();
  const long long bx = (g.n0 + 31) / 32, by = (g.n1 + 7) / 8, tiles = bx * by;
  const long long wave = 6 * sms;  // resident blocks of the bulk-tensor kernel
  const long long per = wave / tiles;  // chunks per tile column in one wave
  long long kc;
  if (tiles * ((g.n2 + 7) / 8) <= wave) {
    kc = 8;
  } else if (per >= 1 && (g.n2 + per - 1) / per <= 48) {
    kc = std::max<long long>(16, (g.n2 + per - 1) / per);
  } else {
    const long long nz = std::max<long long>(1, 32 * sms / tiles);
    kc = std::max<long long>(20, (g.n2 + nz - 1) / nz);
  }
  if (kc > g.n2) kc = g.n2;
  *kchunk = (int)kc;
  const long long nz = (g.n2 + kc - 1) / kc;
  return dim3((unsigned int)bx, (unsigned int)by, (unsigned int)nz);
}
unsigned int matvec_df_blocks(const Geometry& g) {
  int kc;
  const dim3 d = matvec_df_grid(g, &kc);
  return d.x * d.y * d.z;
}

cudaError_t launch_matvec_df(const Geometry& g, PcgState* st, const float* w, float2* q,
                             const float2* T0, const float2* T1, const float2* T2,
                             const float2* FB, double* partials, int par, int mode,
                             cudaStream_t s) {
  int kc;
  const dim3 grid = matvec_df_grid(g, &kc);
  const float2* Bout = FB + g.plane;
  if (mode == 1)
    k_matvec_df<1><<<grid, 256, 0, s>>>(g, st, w, q, T0, T1, T2, FB, Bout, partials, par, kc);
  else
    k_matvec_df<0><<<grid, 256, 0, s>>>(g, st, w, q, T0, T1, T2, FB, Bout, partials, par, kc);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_init_linear(const Geometry& g, double pin, double pout, const double* r,
                               double* x, double* partials, PcgState* st, cudaStream_t s) {
  k_init_linear<<<grid_for(g.n, 256), 256, 0, s>>>(g, pin, pout, r, x, partials, st);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_sub(long long n, double* r, const double* q, cudaStream_t s) {
  k_sub<<<grid_for(n, 256), 256, 0, s>>>(n, r, q);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_finish_x(const Geometry& g, const PcgState* st, double* x, const double* w,
                            const float* wf, int df, cudaStream_t s) {
  if (df)
    k_finish_x<float2, float><<<grid_for(g.n, 256), 256, 0, s>>>(
        g, st, reinterpret_cast<float2*>(x), wf);
  else
    k_finish_x<double, double><<<grid_for(g.n, 256), 256, 0, s>>>(g, st, x, w);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split_inplace(double* a, long long n, cudaStream_t s) {
  k_f64_to_df_inplace<<<grid_for(n, 256), 256, 0, s>>>(a, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split_df(const double* a, float2* b, long long n, cudaStream_t s) {
  k_split_df<<<grid_for(n, 256), 256, 0, s>>>(a, b, n);
  count_launch();
  return cudaGetLastError();
}


cudaError_t launch_matvec(const Geometry& g, PcgState* st, const double* w, double* q,
                          const double* T0, const double* T1, const double* T2, const double* D,
                          double* partials, int par, int mode, cudaStream_t s) {
  const unsigned int nb = matvec_blocks(g);
  if (mode == 0) k_matvec<0><<<nb, 256, 0, s>>>(g, st, w, q, T0, T1, T2, D, partials, par);
  else k_matvec<1><<<nb, 256, 0, s>>>(g, st, w, q, T0, T1, T2, D, partials, par);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ batch work queue
// Persistent forms of the loop kernels above for the solves of one batch class
// (BatchQueue in etc_internal.cuh): every block takes (solve, block) items
// until the queue is empty and runs the kernel body on the solve's buffers
// with the block coordinates the one-solve launch would have given it.

template <int MODE>
__global__ void __launch_bounds__(256) kq_matvec(BatchQueue* q, int slot, const BatchSolve* bs,
                                                Geometry g, unsigned int nb, int par) {
  queue_loop(q, slot, nb, [&](int sv, unsigned int l) {
    const BatchSolve& a = bs[sv];
    matvec_body<MODE>(item_blk(l, nb, 1, 1), g, a.st, a.w, a.q, a.T0, a.T1, a.T2, a.D,
                      a.partials, par);
  });
}

template <int MODE>
__global__ void __launch_bounds__(256, 4) kq_matvec_df(BatchQueue* q, int slot,
                                                      const BatchSolve* bs, Geometry g,
                                                      dim3 grid, int kchunk, int par) {
  const unsigned int per = grid.x * grid.y * grid.z;
  queue_loop(q, slot, per, [&](int sv, unsigned int l) {
    const BatchSolve& a = bs[sv];
    matvec_df_body<MODE>(item_blk(l, grid.x, grid.y, grid.z), g, a.st, a.wf,
                         reinterpret_cast<float2*>(a.q), a.F0, a.F1, a.F2, a.FB,
                         a.FB + g.plane, a.partials, par, kchunk);
  });
}

template <int MODE>
__global__ void __launch_bounds__(128) kq_tridiag(BatchQueue* q, int slot, const BatchSolve* bs,
                                                 Geometry g, unsigned int nb, double w4) {
  queue_loop(q, slot, nb, [&](int sv, unsigned int l) {
    const BatchSolve& a = bs[sv];
    tridiag_body<double, MODE>(item_blk(l, nb, 1, 1), g, a.st, a.t64, a.h64, w4, a.st->kref,
                               1.0, a.partials, nullptr, nullptr);
  });
}

template <int MODE, int MINB>
__global__ void __launch_bounds__(128, MINB) kq_tridiag_otf(BatchQueue* q, int slot,
                                                           const BatchSolve* bs, Geometry g,
                                                           unsigned int nb,
                                                           const double* __restrict__ lam0,
                                                           const double* __restrict__ lam1,
                                                           double w4, int par) {
  queue_loop(q, slot, nb, [&](int sv, unsigned int l) {
    const BatchSolve& a = bs[sv];
    tridiag_otf_body<MODE>(item_blk(l, nb, 1, 1), g, a.st, a.rhat[par], a.t32, a.ck, lam0,
                           lam1, a.st->kref, w4, a.partials, a.rhat[par ^ 1]);
  });
}

// End of one pass of a class's loop (and, with init, its start): the pass
// count and iteration cap of every solve as in k_loop_control, then the list
// of solves still iterating and the rewound item counters; the loop ends when
// no solve is left.
__global__ void k_queue_control(BatchQueue* q, const BatchSolve* bs,
                                cudaGraphConditionalHandle handle, int init) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int na = 0;
  for (int s = 0; s < q->nsolves; ++s) {
    PcgState* st = bs[s].st;
    if (!init) {
      st->passes += 1;
      if (!st->done && st->passes >= st->max_passes) {
        st->status = kENOCONV;
        st->done = 1;
      }
    }
    if (!st->done) q->active[na++] = s;
  }
  q->nactive = na;
  for (int k = 0; k < kQueueSlots; ++k) q->next[k] = 0u;
  if (!init && na == 0) cudaGraphSetConditional(handle, 0u);
}

cudaError_t launch_queue_control(BatchQueue* q, const BatchSolve* bs,
                                 cudaGraphConditionalHandle handle, int init, cudaStream_t s) {
  k_queue_control<<<1, 32, 0, s>>>(q, bs, handle, init);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_q_matvec(const Geometry& g, const QueueLaunch& ql, int par) {
  const unsigned int nb = matvec_blocks(g);
  const unsigned int grid =
      persistent_grid(kq_matvec<1>, 256, 0, (long long)nb * ql.nsolves);
  kq_matvec<1><<<grid, 256, 0, ql.s>>>(ql.q, ql.slot, ql.bs, g, nb, par);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_q_matvec_df(const Geometry& g, const QueueLaunch& ql, int par) {
  int kc;
  const dim3 d = matvec_df_grid(g, &kc);
  const long long per = (long long)d.x * d.y * d.z;
  const unsigned int grid = persistent_grid(kq_matvec_df<1>, 256, 0, per * ql.nsolves);
  kq_matvec_df<1><<<grid, 256, 0, ql.s>>>(ql.q, ql.slot, ql.bs, g, d, kc, par);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_q_tridiag(const Geometry& g, const QueueLaunch& ql) {
  const unsigned int nb = tridiag_blocks(g);
  const double w4 = 4.0 / ((double)g.n0 * g.n1);
  const unsigned int grid = persistent_grid(kq_tridiag<1>, 128, 0, (long long)nb * ql.nsolves);
  kq_tridiag<1><<<grid, 128, 0, ql.s>>>(ql.q, ql.slot, ql.bs, g, nb, w4);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_q_tridiag_otf(const Geometry& g, const QueueLaunch& ql, const double* lam0,
                                 const double* lam1, int par) {
  const unsigned int nb = tridiag_blocks(g);
  const double w4 = 4.0 / ((double)g.n0 * g.n1);
  const long long items = (long long)nb * ql.nsolves;
  // (no 64-register cap as in the one-solve launcher: in the item loop it spills)
  const unsigned int grid = persistent_grid(kq_tridiag_otf<2, 1>, 128, 0, items);
  kq_tridiag_otf<2, 1><<<grid, 128, 0, ql.s>>>(ql.q, ql.slot, ql.bs, g, nb, lam0, lam1, w4, par);
  count_launch();
  return cudaGetLastError();
}

static const size_t kMaxDyn = 200 * 1024;  // dynamic shared memory opt-in per block

// rows per block of the axis-0 transforms and their shared memory
template <typename R>
int rows_per_block(int n0) {
  int L = 2048 / (n0 > 0 ? n0 : 1);
  if (L < 1) L = 1;
  if (L > 64) L = 64;
  return L;
}
template <typename R>
size_t smem_x(int n0, int L) {
  return 2ull * L * dct_half_alloc(n0) * sizeof(c2<R>);
}
template <typename R>
int cols_per_block(int n1) {
  int TI = (sizeof(R) == 8 ? 4096 : 8192) / (n1 > 0 ? n1 : 1);
  if (TI < 1) TI = 1;
  if (TI > 32) TI = 32;
  return TI;
}
template <typename R>
size_t smem_y(int n1, int TI) {
  return 2ull * TI * dct_half_alloc(n1) * sizeof(c2<R>);
}

unsigned int fwd_x_blocks(const Geometry& g, int elem_bytes) {
  (void)elem_bytes;  // any tile down to one row per block
  return (unsigned int)((long long)g.n1 * g.n2);
}

size_t smem_x_bytes(int n0, int L, int elem_bytes) {
  return elem_bytes == 8 ? smem_x<double>(n0, L) : smem_x<float>(n0, L);
}
size_t smem_y_bytes(int n1, int TI, int elem_bytes) {
  return elem_bytes == 8 ? smem_y<double>(n1, TI) : smem_y<float>(n1, TI);
}
size_t smem_limit() { return kMaxDyn; }


// the mixed path's double-float instantiations (FP32 transforms only)
static cudaError_t set_df_attrs() {
  cudaError_t e = cudaSuccess;
  const void* fns[] = {(const void*)k_fwd_x<float, 0, float2>, (const void*)k_fwd_x<float, 1, float2>,
                       (const void*)k_fwd_x<float, 2, float2>, (const void*)k_inv_x<float, float, 0>,
                       (const void*)k_inv_x<float, float, 2>};
  for (const void* f : fns)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDyn);
  return e;
}

template <typename R>
cudaError_t set_smem_attrs() {
  cudaError_t e = cudaSuccess;
#define SETA(fn)                                                                           \
  if (e == cudaSuccess)                                                                    \
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDyn);
  SETA((k_fwd_x<R, 0, double>));
  SETA((k_fwd_x<R, 1, double>));
  SETA((k_fwd_x<R, 2, double>));
  SETA((k_dct_y<R, 0>));
  SETA((k_dct_y<R, 1>));
  SETA((k_inv_x<R, double, 0>));
  SETA((k_inv_x<R, double, 2>));
#undef SETA
  if (e == cudaSuccess && sizeof(R) == 4) e = set_df_attrs();
  if (e == cudaSuccess) e = set_fast_attrs<R>();
  if (e == cudaSuccess && sizeof(R) == 8) e = set_fx_attrs();
  return e;
}
template cudaError_t set_smem_attrs<double>();
template cudaError_t set_smem_attrs<float>();

template <typename R, typename V>
cudaError_t launch_fwd_x(const Geometry& g, const DctPlan<R>& p, PcgState* st, V* x, const V* w,
                         const V* q, V* r, const double* rin, R* t, double* partials, int par,
                         double rtol2, int mode, cudaStream_t s, int L) {
  if constexpr (std::is_same<R, double>::value && std::is_same<V, double>::value) {
    if (L == -3 || L == -4) {
      if (!fx_x_ok(g, p, mode == 2 ? (const void*)rin : (const void*)r, q, x, w))
        return cudaErrorInvalidValue;
      const cudaError_t e = launch_fx_fwd_x(g, p, st, x, w, q, r, rin, t, partials, par, rtol2,
                                            mode, s, L == -4 ? 128 : 256);
      count_launch();
      return e;
    }
  }
  if (L <= 0 && fast_x_ok<R>(g, p, mode == 2 ? (const void*)rin : (const void*)r, q, x, w)) {
    const cudaError_t e = launch_fast_fwd_x<R, V>(g, p, st, x, w, q, r, rin, t, partials, par,
                                                  rtol2, mode, s, L == -2 ? 128 : 256);
    count_launch();
    return e;
  }
  if (L < 0) return cudaErrorInvalidValue;
  if (L == 0) L = rows_per_block<R>(g.n0);
  const size_t sm = smem_x<R>(g.n0, L);
  if (sm > kMaxDyn) return cudaErrorInvalidValue;
  const long long nrows = (long long)g.n1 * g.n2;
  const unsigned int nb = (unsigned int)((nrows + L - 1) / L);
  if (mode == 0)
    k_fwd_x<R, 0, V><<<nb, 256, sm, s>>>(g, p, st, x, w, q, r, rin, t, partials, L, par, rtol2);
  else if (mode == 1)
    k_fwd_x<R, 1, V><<<nb, 256, sm, s>>>(g, p, st, x, w, q, r, rin, t, partials, L, par, rtol2);
  else
    k_fwd_x<R, 2, V><<<nb, 256, sm, s>>>(g, p, st, x, w, q, r, rin, t, partials, L, par, rtol2);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_fwd_x<double, double>(const Geometry&, const DctPlan<double>&,
                                                  PcgState*, double*, const double*,
                                                  const double*, double*, const double*, double*,
                                                  double*, int, double, int, cudaStream_t, int);
template cudaError_t launch_fwd_x<float, double>(const Geometry&, const DctPlan<float>&,
                                                 PcgState*, double*, const double*,
                                                 const double*, double*, const double*, float*,
                                                 double*, int, double, int, cudaStream_t, int);
template cudaError_t launch_fwd_x<float, float2>(const Geometry&, const DctPlan<float>&,
                                                 PcgState*, float2*, const float2*,
                                                 const float2*, float2*, const double*, float*,
                                                 double*, int, double, int, cudaStream_t, int);

template <typename R>
cudaError_t launch_dct_y(const Geometry& g, const DctPlan<R>& p, const PcgState* st, R* t,
                         int inverse, int check, cudaStream_t s, int TI) {
  if (g.n1 == 1) return cudaSuccess;  // a length-1 transform is the identity
  if constexpr (std::is_same<R, double>::value) {
    if (TI == -3) {
      if (!fx_y_ok(g, p)) return cudaErrorInvalidValue;
      const cudaError_t e = launch_fx_y(g, p, st, t, inverse, check, s);
      count_launch();
      return e;
    }
    if (TI == -4) {
      if (!fx_y3_ok(g, p)) return cudaErrorInvalidValue;
      const cudaError_t e = launch_fx_y3(g, p, st, t, inverse, check, s);
      count_launch();
      return e;
    }
  }
  if (TI <= 0 && fast_y_ok<R>(g, p)) {
    const cudaError_t e = launch_fast_y<R>(g, p, st, t, inverse, check, s);
    count_launch();
    return e;
  }
  if (TI < 0) return cudaErrorInvalidValue;
  if (TI == 0) TI = cols_per_block<R>(g.n1);
  const size_t sm = smem_y<R>(g.n1, TI);
  if (sm > kMaxDyn) return cudaErrorInvalidValue;
  dim3 grid((g.n0 + TI - 1) / TI, g.n2);
  if (inverse) k_dct_y<R, 1><<<grid, 256, sm, s>>>(g, p, st, t, TI, check);
  else k_dct_y<R, 0><<<grid, 256, sm, s>>>(g, p, st, t, TI, check);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_dct_y<double>(const Geometry&, const DctPlan<double>&,
                                          const PcgState*, double*, int, int, cudaStream_t, int);
template cudaError_t launch_dct_y<float>(const Geometry&, const DctPlan<float>&, const PcgState*,
                                         float*, int, int, cudaStream_t, int);

unsigned int tridiag_blocks(const Geometry& g) {
  return (unsigned int)((g.plane + 127) / 128);
}

template <typename R>
cudaError_t launch_tridiag(const Geometry& g, PcgState* st, R* t, const R* h, const double* kd,
                           double kz_host, double* partials, int mode, R* rnew, const R* rold,
                           cudaStream_t s) {
  const unsigned int nb = tridiag_blocks(g);
  const double w4 = 4.0 / ((double)g.n0 * g.n1);
  switch (mode) {
    case 0:
      k_tridiag<R, 0><<<nb, 128, 0, s>>>(g, st, t, h, w4, kd, kz_host, partials, rnew, rold);
      break;
    case 1:
      k_tridiag<R, 1><<<nb, 128, 0, s>>>(g, st, t, h, w4, kd, kz_host, partials, rnew, rold);
      break;
    case 2:
      k_tridiag<R, 2><<<nb, 128, 0, s>>>(g, st, t, h, w4, kd, kz_host, partials, rnew, rold);
      break;
    default:
      k_tridiag<R, 3><<<nb, 128, 0, s>>>(g, st, t, h, w4, kd, kz_host, partials, rnew, rold);
      break;
  }
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_tridiag<double>(const Geometry&, PcgState*, double*, const double*,
                                            const double*, double, double*, int, double*,
                                            const double*, cudaStream_t);
template cudaError_t launch_tridiag<float>(const Geometry&, PcgState*, float*, const float*,
                                           const double*, double, double*, int, float*,
                                           const float*, cudaStream_t);

cudaError_t launch_tridiag_otf(const Geometry& g, PcgState* st, const float* in, float* out,
                               float2* ck, const double* lam0, const double* lam1,
                               const double* kd, double* partials, int mode, const float* rold,
                               cudaStream_t s) {
  const unsigned int nb = tridiag_blocks(g);
  const double w4 = 4.0 / ((double)g.n0 * g.n1);
  const bool wide = nb > 6u * 148u;
#define ETC_TRI_OTF(M)                                                                         \
  (wide ? k_tridiag_otf<M, 8><<<nb, 128, 0, s>>>(g, st, in, out, ck, lam0, lam1, kd, w4,       \
                                                 partials, rold)                               \
        : k_tridiag_otf<M, 1><<<nb, 128, 0, s>>>(g, st, in, out, ck, lam0, lam1, kd, w4,       \
                                                 partials, rold))
  switch (mode) {
    case 0: ETC_TRI_OTF(0); break;
    case 1: ETC_TRI_OTF(1); break;
    case 2: ETC_TRI_OTF(2); break;
    default: ETC_TRI_OTF(3); break;
  }
#undef ETC_TRI_OTF
  count_launch();
  return cudaGetLastError();
}
size_t tridiag_ck_pairs(const Geometry& g) {
  return (size_t)((g.n2 + kTriChunk - 1) / kTriChunk - 1) * (size_t)g.plane;
}

template <typename R, typename TZ>
cudaError_t launch_inv_x(const Geometry& g, const DctPlan<R>& p, PcgState* st, const R* t, TZ* z,
                         const double* kd, double kz_host, int check, int mode, cudaStream_t s,
                         int L, typename XOf<TZ>::T* x, int par) {
  if constexpr (std::is_same<R, double>::value && std::is_same<TZ, double>::value) {
    if (L == -3 || L == -4) {
      // FP64 storage: x moves in the forward pass, never here
      if (x != nullptr || !fx_x_ok(g, p, t, z, z, z)) return cudaErrorInvalidValue;
      const cudaError_t e = launch_fx_inv_x(g, p, st, t, z, kd, kz_host, check, mode, s,
                                            L == -4 ? 128 : 256);
      count_launch();
      return e;
    }
  }
  if (L <= 0 && fast_x_ok<R>(g, p, t, z, x, z)) {
    const cudaError_t e = launch_fast_inv_x<R, TZ>(g, p, st, t, z, kd, kz_host, check, mode, s,
                                                   x, par, L == -2 ? 128 : 256);
    count_launch();
    return e;
  }
  if (L < 0) return cudaErrorInvalidValue;
  if (L == 0) L = rows_per_block<R>(g.n0);
  const size_t sm = smem_x<R>(g.n0, L) + (mode == 2 ? (size_t)L * g.n0 * sizeof(TZ) : 0);
  if (sm > kMaxDyn) return cudaErrorInvalidValue;
  const long long nrows = (long long)g.n1 * g.n2;
  const unsigned int nb = (unsigned int)((nrows + L - 1) / L);
  if (mode == 2)
    k_inv_x<R, TZ, 2><<<nb, 256, sm, s>>>(g, p, st, t, z, kd, kz_host, L, check, x, par);
  else
    k_inv_x<R, TZ, 0><<<nb, 256, sm, s>>>(g, p, st, t, z, kd, kz_host, L, check, x, par);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_inv_x<double, double>(const Geometry&, const DctPlan<double>&,
                                                  PcgState*, const double*, double*,
                                                  const double*, double, int, int, cudaStream_t,
                                                  int, double*, int);
template cudaError_t launch_inv_x<float, double>(const Geometry&, const DctPlan<float>&,
                                                 PcgState*, const float*, double*,
                                                 const double*, double, int, int, cudaStream_t,
                                                 int, double*, int);
template cudaError_t launch_inv_x<float, float>(const Geometry&, const DctPlan<float>&,
                                                PcgState*, const float*, float*,
                                                const double*, double, int, int, cudaStream_t,
                                                int, float2*, int);

cudaError_t launch_flux(const Geometry& g, const double* x, const double* T0, const double* T1,
                        const double* T2, const double* Bin, const double* Bout, double pin,
                        double pout, double* partials, PcgState* st, cudaStream_t s) {
  k_flux<<<grid_for(g.n, 256, 148 * 8), 256, 0, s>>>(g, x, T0, T1, T2, Bin, Bout, pin, pout,
                                                     partials, st);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_true_residual(const Geometry& g, const double* x, const double* T0,
                                 const double* T1, const double* T2, const double* D,
                                 const double* Bin, const double* Bout, double pin, double pout,
                                 double* partials, PcgState* st, cudaStream_t s,
                                 const double* pin_f, const double* pout_f, const double* src) {
  k_true_residual<<<grid_for(g.n, 256, 148 * 8), 256, 0, s>>>(g, x, T0, T1, T2, D, Bin, Bout, pin,
                                                              pout, pin_f, pout_f, src, partials,
                                                              st);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_convert(const float* fin, double* dout, const double* din, float* fout,
                           long long n, cudaStream_t s) {
  k_convert<<<grid_for(n, 256), 256, 0, s>>>(fin, dout, din, fout, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_gradient(const Geometry& g, const double* x, const double* lam,
                            const double* k0, const double* k1, const double* k2, double ih0,
                            double ih1, double ih2, const double* T0, const double* T1,
                            const double* T2, double pin, double pout, double cJ, double* G0,
                            double* G1, double* G2, int summed, cudaStream_t s) {
  k_gradient<<<grid_for(g.n, 256), 256, 0, s>>>(g, x, lam, k0, k1, k2, ih0, ih1, ih2, T0, T1, T2,
                                                pin, pout, cJ, G0, G1, G2, summed);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_widen(const float* a, double* b, long long n, cudaStream_t s) {
  k_widen<<<grid_for(n, 256), 256, 0, s>>>(a, b, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace etc
