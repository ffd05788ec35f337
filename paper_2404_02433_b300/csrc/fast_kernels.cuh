// Register-resident cosine transforms for the line lengths n whose half m = n/2
// splits as below (n = 32, 64, 96, 128, 160, 192, 256, 384, 512, 1024).
//
// Same transforms as the generic kernels (Eq. (forward DCT) and Eq. (backward
// DCT), Sec. 3.2), reached through the same half-length complex FFT with the
// even/odd reordering and the untangling twiddles, but with the FFT of length
// M = n/2 split as M = P * Q in the four-step manner:
//   thread tau of a line holds z_{tau + P s}, s < Q, and runs a length-Q DFT in
//   registers; after the twiddle exp(-+2 pi i tau k1 / M) one shared-memory
//   transpose hands each thread the values of Q/P indices k1, for which it runs
//   length-P DFTs, giving Z_{k1 + Q k2}.
// Every index is a compile-time shift or mask, which is what the generic
// Stockham code (runtime stage loop, divisions by runtime line lengths) lacks.
//
// Axis-1 passes (columns of a plane, stride n0) keep one column per lane and P
// warps per column tile, loading and storing global memory directly with the
// lanes over adjacent columns.  Axis-0 passes (rows) stage the row through
// shared memory so that the FP64 PCG vectors stay coalesced.
#pragma once

#include <type_traits>

#include "dct_device.cuh"
#include "etc_internal.cuh"
#include "launchers.h"

namespace etc {

// Four-step split m = P * Q: P threads per line (16, 8 or 4, the largest that
// works), Q values per thread with P | Q, Q a length with a register DFT
// (4, 8, 16 by radix 4; 12, 20, 24, 32 by Cooley-Tukey over 3, 4, 5, 8);
// 0 if m has no such split.
constexpr bool fast_q_ok(int q) {
  return q == 4 || q == 8 || q == 12 || q == 16 || q == 20 || q == 24 || q == 32;
}
constexpr int fast_p(int m) {
  return (m % 16 == 0 && m / 16 >= 16 && (m / 16) % 16 == 0 && fast_q_ok(m / 16)) ? 16
         : (m % 8 == 0 && m / 8 >= 8 && (m / 8) % 8 == 0 && fast_q_ok(m / 8))    ? 8
         : (m % 4 == 0 && m / 4 >= 4 && (m / 4) % 4 == 0 && fast_q_ok(m / 4))    ? 4
                                                                                  : 0;
}

template <int N> struct Fast {
  static constexpr int M = N / 2;
  static constexpr int P = fast_p(M);
  static constexpr int Q = M / P;
  static constexpr int E = Q / P;  // length-P DFTs per thread in the second step
  static_assert(P * Q == M && Q % P == 0, "four-step split");
  // Axis-0 shared layout, in complex units per row: A holds the row (staging,
  // then Z), B the transposed partial transforms.  The strides are P mod 16
  // so that the rows met by one half-warp use disjoint banks.
  static constexpr int SA = M + P;
  static constexpr int BS0 = Q * (P + 1);
  static constexpr int BS = BS0 + (((P - BS0) % 16) + 16) % 16;
  // one region per row serves both (they are never live together): stride
  // max(SA, BS), still P mod 16
  static constexpr int RS = SA > BS ? SA : BS;
};

// Axis-0 blocks of NT threads (256 or 128): L = NT / P rows each.
template <int N, int NT> struct FastX {
  static constexpr int L = NT / Fast<N>::P;
  static_assert(L * Fast<N>::P == NT, "rows per block");
};

template <typename R, int N> struct FastCols {  // columns per block of the axis-1 passes
  // FP32: 16 columns from n = 512 on (measured at 512^3: backward pass 0.274 ->
  // 0.248 ms), 32 below (16 was 5-10 % slower at 192^3 and 256^3); FP64: 16
  static constexpr int C = sizeof(R) == 4 ? (N >= 512 ? 16 : 32) : 16;
  // resident blocks per SM asked of the compiler: 1024 (FP32) or 512 (FP64)
  // threads, i.e. at most 64 or 128 registers per thread; half that for
  // Q > 16 values per thread
  static constexpr int MinBlocks() {
    return ((sizeof(R) == 4 ? 1024 : 512) >> ((N / 2) / fast_p(N / 2) > 16 ? 1 : 0)) /
           (C * fast_p(N / 2));
  }
};



// ---------------------------------------------------------------- helpers
__device__ __forceinline__ void ld4(const float* p, float& a, float& b, float& c, float& d) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double& a, double& b, double& c,
                                    double& d) {
  const double2 u = __ldg(reinterpret_cast<const double2*>(p));
  const double2 v = __ldg(reinterpret_cast<const double2*>(p + 2));
  a = u.x; b = u.y; c = v.x; d = v.y;
}

// First four-step stage of thread tau: DFT of length Q over s, then the twiddle
// exp(SIGN 2 pi i tau k1 / M) from the [tau][k1] table (forward sign stored).
template <typename R, int N, int SIGN>
__device__ __forceinline__ void four_step_a(c2<R>* v, const R* __restrict__ tw4, int tau) {
  using F = Fast<N>;
  Bfly<R, F::Q, SIGN>::run(v);
  const c2<R>* tw = reinterpret_cast<const c2<R>*>(tw4) + tau * F::Q;
#pragma unroll
  for (int k1 = 1; k1 < F::Q; ++k1) {
    c2<R> w = __ldg(tw + k1);
    if (SIGN > 0) w.y = -w.y;
    v[k1] = cmul<R>(v[k1], w);
  }
}

// Forward untangling: X_k and X_{n-k} (X_m for k = 0) from Z_k and Z_{m-k},
// with the fpost twiddles of k (and of m for k = 0).
template <typename R>
__device__ __forceinline__ void untangle(c2<R> zk, c2<R> zm, const R* __restrict__ fpost, int k,
                                         int m, R& xa, R& xb) {
  const R a1 = zk.x + zm.x, b1 = zk.y - zm.y, c1 = zk.y + zm.y, d1 = zk.x - zm.x;
  R f0, f1, f2, f3;
  ld4(fpost + 4 * k, f0, f1, f2, f3);
  xa = fma(f0, a1, fma(f1, b1, fma(f2, c1, -f3 * d1)));
  if (k != 0) {
    xb = fma(f1, a1, fma(-f0, b1, fma(f2, d1, f3 * c1)));
  } else {
    R g0, g1, g2, g3;
    ld4(fpost + 4 * m, g0, g1, g2, g3);
    xb = fma(g0, a1, g2 * c1);
  }
}

// Backward pre-twiddle of FFT input j from X_j, X_{n-j} (0 for j = 0), X_{m-j}
// and X_{m+j}: V_j = e^{i t_j} (X_j - i X_{n-j}) / (2m), V_{m-j} likewise,
// a_j = P + i O with P = V_j + conj(V_{m-j}), O = (V_j - conj(V_{m-j})) e^{4 i t_j}.
template <typename R>
__device__ __forceinline__ c2<R> inv_pre(const R* __restrict__ ipre, int j, int m, R xj, R xn,
                                         R xm, R xp) {
  R f0, f1, f2, f3, g0, g1, g2, g3;
  ld4(ipre + 4 * j, f0, f1, f2, f3);
  if constexpr (sizeof(R) == 4) {
    // the constants of m - j from those of j (m = n/2): its angle is
    // pi/4 - t_j, so cos and sin are (cos t_j +- sin t_j) / sqrt 2, and
    // 4 (pi/4 - t_j) = pi - 4 t_j; one table load instead of two (the FP32
    // backward pass is bound by the L1/shared-memory pipe)
    constexpr R h = (R)0.70710678118654752440;
    g0 = (f0 + f1) * h;
    g1 = (f0 - f1) * h;
    g2 = -f2;
    g3 = f3;
  } else {
    ld4(ipre + 4 * (m - j), g0, g1, g2, g3);
  }
  const R vr = fma(f0, xj, f1 * xn), vi = fma(f1, xj, -f0 * xn);
  const R wr = fma(g0, xm, g1 * xp), wi = fma(g1, xm, -g0 * xp);
  const R pr = vr + wr, pi = vi - wi;
  const R qr = vr - wr, qi = vi + wi;
  const R orr = fma(qr, f2, -qi * f3), oi = fma(qr, f3, qi * f2);
  return mk2<R>(pr - oi, pi + orr);
}

// Row of v (reordered input) that feeds real slot a: v_a = u_{2a} for a < m,
// u_{2(n-1-a)+1} otherwise.
template <int N>
__device__ __forceinline__ int vrow(int a) {
  return a < N / 2 ? 2 * a : 2 * (N - 1 - a) + 1;
}

// ---------------------------------------------------------------- axis 1
// In place on t: every block owns C adjacent columns of one plane k.
// The bodies take the block coordinates b (the hardware block, or a batch
// queue item standing for one block of this solve's launch).
template <typename R, int N, int INV>
__device__ __forceinline__ void fast_y_body(const Blk& b, Geometry g,
                                            DctTables<R> tb, const PcgState* st,
                                            R* __restrict__ t, int check, int pf) {
  using F = Fast<N>;
  constexpr int M = F::M, P = F::P, Q = F::Q, E = F::E, C = FastCols<R, N>::C;
  constexpr int SIGN = INV ? 1 : -1;
  extern __shared__ __align__(16) unsigned char smraw[];
  c2<R>* sm = reinterpret_cast<c2<R>*>(smraw);  // C * M complex
  if (check && st->done) return;
  if (pf > 0 && threadIdx.x == 0) {
    // the share of the buffer of the block pf blocks ahead (a plane's blocks
    // split it into equal byte ranges) goes to L2 while this block computes
    const unsigned long long total = (unsigned long long)g.plane * g.n2 * sizeof(R);
    const unsigned long long share =
        ((unsigned long long)g.plane * sizeof(R) / b.nx + 15) / 16 * 16;
    const unsigned long long a0 =
        ((unsigned long long)b.y * b.nx + b.x + (unsigned long long)pf) * share;
    if (a0 < total) {
      const unsigned long long a1 = min(a0 + share, total / 16 * 16);
      if (a1 > a0)
        l2_prefetch(reinterpret_cast<const unsigned char*>(t) + a0, (unsigned int)(a1 - a0));
    }
  }
  const int c = threadIdx.x % C, tau = threadIdx.x / C;
  const int i = b.x * C + c;
  const bool ok = i < g.n0;
  const long long n0 = g.n0;
  R* col = t + (long long)b.y * g.plane + (ok ? i : 0);
  c2<R> v[Q];
  if (!INV) {
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int q = tau + P * s;  // z_q = (v_{2q}, v_{2q+1})
      v[s] = ok ? mk2<R>(col[vrow<N>(2 * q) * n0], col[vrow<N>(2 * q + 1) * n0])
                : mk2<R>((R)0, (R)0);
    }
  } else {
    // every input j needs X_j, X_{n-j}, X_{m-j}, X_{m+j}: stage the tile's
    // columns once (real view of the buffer, row-major over the C columns)
    R* sr = reinterpret_cast<R*>(smraw);
    if constexpr (sizeof(R) == 4 && Q <= 16) {
      // the thread loads rows j = tau + P s and j + m (P Q = m): X_j and
      // X_{m+j} stay in its registers, and the staged tile supplies only
      // X_{n-j} and X_{m-j} (half the shared-memory reads; this pass is
      // bound by the L1/shared-memory pipe)
      R xa[Q], xb[Q];
#pragma unroll
      for (int s = 0; s < Q; ++s) {
        xa[s] = ok ? col[(tau + P * s) * n0] : (R)0;
        xb[s] = ok ? col[(tau + P * s + M) * n0] : (R)0;
      }
#pragma unroll
      for (int s = 0; s < Q; ++s) {
        sr[(tau + P * s) * C + c] = xa[s];
        sr[(tau + P * s + M) * C + c] = xb[s];
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < Q; ++s) {
        const int j = tau + P * s;
        v[s] = inv_pre<R>(tb.ipre, j, M, xa[s], j ? sr[(N - j) * C + c] : (R)0,
                          sr[(M - j) * C + c], xb[s]);
      }
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {  // rows tau + P s, s < 2Q, in two halves
        R xs[Q];
#pragma unroll
        for (int s = 0; s < Q; ++s) xs[s] = ok ? col[(tau + P * (s + h * Q)) * n0] : (R)0;
#pragma unroll
        for (int s = 0; s < Q; ++s) sr[(tau + P * (s + h * Q)) * C + c] = xs[s];
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < Q; ++s) {
        const int j = tau + P * s;
        v[s] = inv_pre<R>(tb.ipre, j, M, sr[j * C + c], j ? sr[(N - j) * C + c] : (R)0,
                          sr[(M - j) * C + c], sr[(M + j) * C + c]);
      }
    }
    __syncthreads();  // the staged tile is read before the transpose reuses the buffer
  }
  four_step_a<R, N, SIGN>(v, tb.tw4, tau);
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) sm[(k1 * P + tau) * C + c] = v[k1];
  __syncthreads();
  c2<R> u[Q];
#pragma unroll
  for (int e = 0; e < E; ++e) {
#pragma unroll
    for (int tt = 0; tt < P; ++tt) u[e * P + tt] = sm[((tau + P * e) * P + tt) * C + c];
    Bfly<R, P, SIGN>::run(u + e * P);
  }
  if (!INV) {
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) sm[(tau + P * e + Q * k2) * C + c] = u[e * P + k2];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) {
        const int k = tau + P * e + Q * k2;
        R xa, xb;
        untangle<R>(u[e * P + k2], sm[(k ? M - k : 0) * C + c], tb.fpost, k, M, xa, xb);
        if (ok) {
          col[k * n0] = xa;
          col[(k ? N - k : M) * n0] = xb;
        }
      }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) {
        const int j = tau + P * e + Q * k2;  // z_j = (v_{2j}, v_{2j+1})
        if (ok) {
          col[vrow<N>(2 * j) * n0] = u[e * P + k2].x;
          col[vrow<N>(2 * j + 1) * n0] = u[e * P + k2].y;
        }
      }
  }
}
template <typename R, int N, int INV>
__global__ void __launch_bounds__(FastCols<R, N>::C * Fast<N>::P, FastCols<R, N>::MinBlocks())
    k_fast_y(Geometry g, DctTables<R> tb, const PcgState* st, R* __restrict__ t, int check,
             int pf) {
  fast_y_body<R, N, INV>(hw_blk(), g, tb, st, t, check, pf);
}

// ---------------------------------------------------------------- axis 0, forward
// Same contract as k_fwd_x (MODE 0 initial residual, 1 PCG update, 2 transform
// only; V the storage of x, w, q, r; x moves here for FP64 storage only).
// Rows [row0, row0 + L) are contiguous in memory: the vector phase walks them
// as pairs of elements with 16-byte loads.
template <typename R, int N, int MODE, typename V, int NT>
__device__ __forceinline__ void fast_fwd_x_body(const Blk& b, Geometry g,
                                                DctTables<R> tb, PcgState* st,
                                                V* __restrict__ x, const V* __restrict__ w,
                                                const V* __restrict__ q, V* __restrict__ r,
                                                const double* __restrict__ rin,
                                                R* __restrict__ t, double* partials, int par,
                                                double rtol2, int pf) {
  using F = Fast<N>;
  constexpr int M = F::M, P = F::P, Q = F::Q, E = F::E, RS = F::RS;
  constexpr int L = FastX<N, NT>::L;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32];
  __shared__ int flag;
  if (MODE != 2 && st->done) return;
  c2<R>* A = reinterpret_cast<c2<R>*>(smraw);  // rows of RS complex: staging, transpose, Z
  R* Ar = reinterpret_cast<R*>(A);
  const long long nrows = (long long)g.n1 * g.n2;
  const long long row0 = (long long)b.x * L;
  if (MODE == 1 && pf > 0 && threadIdx.x == 0) {
    // the r and q rows of the block pf blocks ahead go to L2 meanwhile
    const long long pr = row0 + (long long)pf * L;
    if (pr < nrows) {
      const unsigned int bytes = (unsigned int)(min((long long)L, nrows - pr) * N * sizeof(V));
      l2_prefetch(r + pr * N, bytes);
      l2_prefetch(q + pr * N, bytes);
    }
  }
  using S = Scalar<V>;
  constexpr bool XHERE = (MODE == 1) && std::is_same<V, double>::value;
  const typename S::T alpha = S::from((MODE == 1) ? st->alpha[par] : 0.0);
  const typename S::T nalpha = S::neg(alpha);
  double acc = 0.0;
  float accf = 0.f;
  constexpr int NP = L * M;  // element pairs of the block
  // pairs per thread whose loads are in flight together (2 or 4 vectors of 16 bytes each)
  constexpr int U = std::is_same<V, float2>::value ? 4 : 2;
  static_assert(NP % (NT * U) == 0, "pair rounds");
  for (int p0 = threadIdx.x; p0 < NP; p0 += NT * U) {
    VPair<V> rv[U], qv[U], xv[U], wv[U];
    double2 dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = p0 + NT * u;
      const int l = p / M, i2 = p % M;
      const long long row = row0 + l;
      rv[u].a = rv[u].b = vzero<V>();
      qv[u] = rv[u]; xv[u] = rv[u]; wv[u] = rv[u];
      dv[u] = make_double2(0.0, 0.0);
      if (row < nrows) {
        const long long c = row * N + 2 * i2;
        if (MODE == 2) dv[u] = *reinterpret_cast<const double2*>(rin + c);
        else rv[u] = ld_pair(r + c);
        if (MODE == 1) qv[u] = ld_pair(q + c);
        if (XHERE) {
          xv[u] = ld_pair(x + c);
          wv[u] = ld_pair(w + c);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = p0 + NT * u;
      const int l = p / M, i2 = p % M;
      const long long row = row0 + l;
      R in0, in1;
      if (MODE == 2) {
        in0 = from_f64<R>(dv[u].x);
        in1 = from_f64<R>(dv[u].y);
      } else {
        V v0 = rv[u].a, v1 = rv[u].b;
        if (row < nrows) {
          const long long c = row * N + 2 * i2;
          if (MODE == 1) {
            if (XHERE)
              st_pair(x + c, vaxpy(alpha, wv[u].a, xv[u].a), vaxpy(alpha, wv[u].b, xv[u].b));
            v0 = vaxpy(nalpha, qv[u].a, v0);
            v1 = vaxpy(nalpha, qv[u].b, v1);
            st_pair(r + c, v0, v1);
          }
          vsq_acc(v0, acc, accf);
          vsq_acc(v1, acc, accf);
        }
        in0 = vround<R>(v0);
        in1 = vround<R>(v1);
      }
      // element 2 i2 -> v_{i2}; element 2 i2 + 1 -> v_{n-1-i2}
      Ar[l * 2 * RS + i2] = in0;
      Ar[l * 2 * RS + N - 1 - i2] = in1;
    }
  }
  __syncthreads();
  const int l = threadIdx.x / P, tau = threadIdx.x % P;
  c2<R> v[Q];
#pragma unroll
  for (int s = 0; s < Q; ++s) v[s] = A[l * RS + tau + P * s];
  four_step_a<R, N, -1>(v, tb.tw4, tau);
  __syncthreads();  // the row is read before the transpose overwrites it
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) A[l * RS + k1 * (P + 1) + tau] = v[k1];
  __syncthreads();
  c2<R> u[Q];
#pragma unroll
  for (int e = 0; e < E; ++e) {
#pragma unroll
    for (int tt = 0; tt < P; ++tt) u[e * P + tt] = A[l * RS + (tau + P * e) * (P + 1) + tt];
    Bfly<R, P, -1>::run(u + e * P);
  }
  __syncthreads();  // the transpose is read before Z overwrites it
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) A[l * RS + tau + P * e + Q * k2] = u[e * P + k2];
  __syncthreads();
  const long long row = row0 + l;
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) {
      const int k = tau + P * e + Q * k2;
      R xa, xb;
      untangle<R>(u[e * P + k2], A[l * RS + (k ? M - k : 0)], tb.fpost, k, M, xa, xb);
      if (row < nrows) {
        t[row * N + k] = xa;
        t[row * N + (k ? N - k : M)] = xb;
      }
    }
  if (MODE != 2)
    fwd_x_residual_tail<MODE>(acc + widen(accf), st, partials, rtol2, sh, &flag, par, !XHERE,
                              b);
}
template <typename R, int N, int MODE, typename V, int NT>
__global__ void __launch_bounds__(NT)
    k_fast_fwd_x(Geometry g, DctTables<R> tb, PcgState* st, V* __restrict__ x,
                 const V* __restrict__ w, const V* __restrict__ q, V* __restrict__ r,
                 const double* __restrict__ rin, R* __restrict__ t, double* partials, int par,
                 double rtol2, int pf) {
  fast_fwd_x_body<R, N, MODE, V, NT>(hw_blk(), g, tb, st, x, w, q, r, rin, t, partials, par,
                                     rtol2, pf);
}

// ---------------------------------------------------------------- axis 0, backward
// Same contract as k_inv_x: u = scale * (backward DCT of t along axis 0), then
// MODE 0: z = u; MODE 2: w = u + beta w in place (z points at w), after
// x += alpha w with the old w when x is given.
template <typename R, typename TZ, int N, int MODE, int NT>
__device__ __forceinline__ void fast_inv_x_body(const Blk& b, Geometry g,
                                                DctTables<R> tb, PcgState* st,
                                                const R* __restrict__ t, TZ* __restrict__ z,
                                                const double* kd, double kz_host, int check,
                                                typename XOf<TZ>::T* __restrict__ x, int par) {
  using TX = typename XOf<TZ>::T;  // x's storage (FP32 directions: double-float x)
  using F = Fast<N>;
  constexpr int M = F::M, P = F::P, Q = F::Q, E = F::E, RS = F::RS;
  constexpr int L = FastX<N, NT>::L;
  constexpr int SR = N + P;  // real stride of the staged input rows
  extern __shared__ __align__(16) unsigned char smraw[];
  if (check && st->done) return;
  c2<R>* A = reinterpret_cast<c2<R>*>(smraw);  // rows of RS complex: staging, transpose, z
  R* Ar = reinterpret_cast<R*>(A);
  const long long nrows = (long long)g.n1 * g.n2;
  const long long row0 = (long long)b.x * L;
  // stage the block's rows in natural order, 16 bytes per access, all of a
  // thread's loads issued before the first shared-memory store
  using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
  constexpr int VW = 16 / (int)sizeof(R);
  constexpr int NR = L * N / VW / NT;
  static_assert(NR * NT * VW == L * N, "staging rounds");
  {
    V val[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int e = threadIdx.x + NT * r;
      const int l = (e * VW) / N, i = (e * VW) % N;
      const long long row = row0 + l;
      val[r] = row < nrows ? *reinterpret_cast<const V*>(t + row * N + i) : V{};
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int e = threadIdx.x + NT * r;
      const int l = (e * VW) / N, i = (e * VW) % N;
      *reinterpret_cast<V*>(Ar + l * SR + i) = val[r];
    }
  }
  __syncthreads();
  const int l = threadIdx.x / P, tau = threadIdx.x % P;
  const R* X = Ar + l * SR;
  c2<R> v[Q];
#pragma unroll
  for (int s = 0; s < Q; ++s) {
    const int j = tau + P * s;
    v[s] = inv_pre<R>(tb.ipre, j, M, X[j], j ? X[N - j] : (R)0, X[M - j], X[M + j]);
  }
  four_step_a<R, N, 1>(v, tb.tw4, tau);
  __syncthreads();  // the staged row is read before the transpose overwrites it
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) A[l * RS + k1 * (P + 1) + tau] = v[k1];
  __syncthreads();
  c2<R> u[Q];
#pragma unroll
  for (int e = 0; e < E; ++e) {
#pragma unroll
    for (int tt = 0; tt < P; ++tt) u[e * P + tt] = A[l * RS + (tau + P * e) * (P + 1) + tt];
    Bfly<R, P, 1>::run(u + e * P);
  }
  __syncthreads();  // the transpose is read before z overwrites it
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) A[l * RS + tau + P * e + Q * k2] = u[e * P + k2];
  __syncthreads();
  // real view of A: slot a of row l holds v_a
  const R scale = (R)(1.0 / (kd ? kd[2] : kz_host));
  const typename Scalar<TZ>::T beta = Scalar<TZ>::from((MODE == 2) ? st->beta : 0.0);
  const bool upd = (MODE == 2) && x != nullptr;
  const typename Scalar<TX>::T alpha = Scalar<TX>::from(upd ? st->alpha[par] : 0.0);
  if (upd && b.x == 0 && threadIdx.x == 0) st->xpend = 0;
  constexpr int NQ = L * M / NT;  // element pairs per thread
  constexpr int G = NQ < 4 ? NQ : 4;  // pairs whose loads are in flight together
  static_assert(NQ % G == 0, "pair groups");
#pragma unroll 1
  for (int r0 = 0; r0 < NQ; r0 += G) {
    VPair<TZ> wo[G];
    VPair<TX> xo[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int p = threadIdx.x + NT * (r0 + u);
      const long long row = row0 + p / M;
      wo[u].a = wo[u].b = vzero<TZ>();
      xo[u].a = xo[u].b = vzero<TX>();
      if (MODE == 2 && row < nrows) {
        wo[u] = ld_pair(z + row * N + 2 * (p % M));
        if (upd) xo[u] = ld_pair(x + row * N + 2 * (p % M));
      }
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int p = threadIdx.x + NT * (r0 + u);
      const int lr = p / M, i2 = p % M;
      const long long row = row0 + lr;
      if (row >= nrows) continue;
      const long long c = row * N + 2 * i2;
      const R u0 = Ar[lr * 2 * RS + i2] * scale;          // element 2 i2     <- v_{i2}
      const R u1 = Ar[lr * 2 * RS + N - 1 - i2] * scale;  // element 2 i2 + 1 <- v_{n-1-i2}
      if (MODE == 2) {
        if (upd) st_pair(x + c, xaxpy(alpha, wo[u].a, xo[u].a), xaxpy(alpha, wo[u].b, xo[u].b));
        st_pair(z + c, vaxpy(beta, wo[u].a, vfrom<TZ, R>(u0)),
                vaxpy(beta, wo[u].b, vfrom<TZ, R>(u1)));
      }
      else
        st_pair(z + c, vfrom<TZ, R>(u0), vfrom<TZ, R>(u1));
    }
  }
}
template <typename R, typename TZ, int N, int MODE, int NT>
__global__ void __launch_bounds__(NT)
    k_fast_inv_x(Geometry g, DctTables<R> tb, PcgState* st, const R* __restrict__ t,
                 TZ* __restrict__ z, const double* kd, double kz_host, int check,
                 typename XOf<TZ>::T* __restrict__ x, int par) {
  fast_inv_x_body<R, TZ, N, MODE, NT>(hw_blk(), g, tb, st, t, z, kd, kz_host, check, x, par);
}

// ---------------------------------------------------------------- batch work queue
// Persistent forms of the three transforms over the solves of a batch class
// (BatchQueue in etc_internal.cuh), with the operands of the PCG iteration:
// FP64 (R = double) on the FP64 vectors, mixed (R = float) on the
// double-float vectors and the FP32 search direction.
template <typename R, int N, int NT>
__global__ void __launch_bounds__(NT)
    kq_fast_fwd_x(BatchQueue* q, int slot, const BatchSolve* bs, Geometry g, DctTables<R> tb,
                  unsigned int nb, int par) {
  queue_loop(q, slot, nb, [&](int sv, unsigned int l) {
    const BatchSolve& a = bs[sv];
    if constexpr (sizeof(R) == 8)
      fast_fwd_x_body<R, N, 1, double, NT>(item_blk(l, nb, 1, 1), g, tb, a.st, a.x, a.w, a.q,
                                           a.r, nullptr, a.t64, a.partials, par, 0.0, 0);
    else
      fast_fwd_x_body<R, N, 1, float2, NT>(
          item_blk(l, nb, 1, 1), g, tb, a.st, nullptr, nullptr,
          reinterpret_cast<const float2*>(a.q), reinterpret_cast<float2*>(a.r), nullptr,
          a.rhat[par], a.partials, par, 0.0, 0);
  });
}

// buf: 0 = t64, 1 = rhat[par], 2 = t32
template <typename R, int N, int INV>
__global__ void __launch_bounds__(FastCols<R, N>::C * Fast<N>::P, FastCols<R, N>::MinBlocks())
    kq_fast_y(BatchQueue* q, int slot, const BatchSolve* bs, Geometry g, DctTables<R> tb,
              unsigned int nbx, int buf, int par) {
  const unsigned int per = nbx * (unsigned int)g.n2;
  queue_loop(q, slot, per, [&](int sv, unsigned int l) {
    const BatchSolve& a = bs[sv];
    R* t;
    if constexpr (sizeof(R) == 8) t = a.t64;
    else t = buf == 1 ? a.rhat[par] : a.t32;
    fast_y_body<R, N, INV>(item_blk(l, nbx, (unsigned int)g.n2, 1), g, tb, a.st, t, 1, 0);
  });
}

template <typename R, int N, int NT>
__global__ void __launch_bounds__(NT)
    kq_fast_inv_x(BatchQueue* q, int slot, const BatchSolve* bs, Geometry g, DctTables<R> tb,
                  unsigned int nb, int par) {
  queue_loop(q, slot, nb, [&](int sv, unsigned int l) {
    const BatchSolve& a = bs[sv];
    if constexpr (sizeof(R) == 8)
      fast_inv_x_body<R, double, N, 2, NT>(item_blk(l, nb, 1, 1), g, tb, a.st, a.t64, a.w,
                                           a.st->kref, 1.0, 1, nullptr, par);
    else
      fast_inv_x_body<R, float, N, 2, NT>(item_blk(l, nb, 1, 1), g, tb, a.st, a.t32, a.wf,
                                          a.st->kref, 1.0, 1, reinterpret_cast<float2*>(a.x),
                                          par);
  });
}

// ---------------------------------------------------------------- per-size launchers
// Defined here, instantiated per length in fast_sizes_*.cu (several translation
// units, so that the library builds in parallel), called by fast_dispatch.cu.

template <typename R, int N, int NT>
size_t fast_x_smem() {
  return (size_t)FastX<N, NT>::L * Fast<N>::RS * sizeof(c2<R>);
}
template <typename R, int N>
size_t fast_y_smem() {
  return (size_t)FastCols<R, N>::C * Fast<N>::M * sizeof(c2<R>);
}


constexpr size_t kFastSmemMax = 200 * 1024;  // dynamic shared memory opt-in per block
template <typename R, int N, int NT>
constexpr bool fast_x_fits() {
  return (size_t)FastX<N, NT>::L * Fast<N>::RS * sizeof(c2<R>) <= kFastSmemMax;
}

template <typename R, int N, typename V, int NT>
cudaError_t fwd_x_nt(const Geometry& g, const DctTables<R>& tb, PcgState* st, V* x, const V* w,
                     const V* q, V* r, const double* rin, R* t, double* partials, int par,
                     double rtol2, int mode, cudaStream_t s) {
  constexpr int L = FastX<N, NT>::L;
  const long long nrows = (long long)g.n1 * g.n2;
  const unsigned int nb = (unsigned int)((nrows + L - 1) / L);
  const size_t sm = fast_x_smem<R, N, NT>();
  // PCG update: the block's r and q rows about 3 MB ahead go to L2 (mixed,
  // 512^3: 0.641 -> 0.607 ms, flat from 0.8 to 3.2 MB; 5 MB and more ahead
  // slower), when the grid is more than two waves
  static const int resident = resident_blocks(k_fast_fwd_x<R, N, 1, V, NT>, NT, sm);
  const int pf = resident > 0 && (long long)nb > 2LL * resident
                     ? max(1, (int)((3u << 20) / (2u * L * N * sizeof(V))))
                     : 0;
  if (mode == 0)
    k_fast_fwd_x<R, N, 0, V, NT><<<nb, NT, sm, s>>>(g, tb, st, x, w, q, r, rin, t, partials,
                                                    par, rtol2, pf);
  else if (mode == 1)
    k_fast_fwd_x<R, N, 1, V, NT><<<nb, NT, sm, s>>>(g, tb, st, x, w, q, r, rin, t, partials,
                                                    par, rtol2, pf);
  else
    k_fast_fwd_x<R, N, 2, V, NT><<<nb, NT, sm, s>>>(g, tb, st, x, w, q, r, rin, t, partials,
                                                    par, rtol2, pf);
  return cudaGetLastError();
}
template <typename R, int N, typename V>
cudaError_t fwd_x_n(const Geometry& g, const DctTables<R>& tb, PcgState* st, V* x, const V* w,
                    const V* q, V* r, const double* rin, R* t, double* partials, int par,
                    double rtol2, int mode, cudaStream_t s, int nt) {
  if (nt == 128 || !fast_x_fits<R, N, 256>())
    return fwd_x_nt<R, N, V, 128>(g, tb, st, x, w, q, r, rin, t, partials, par, rtol2, mode, s);
  return fwd_x_nt<R, N, V, 256>(g, tb, st, x, w, q, r, rin, t, partials, par, rtol2, mode, s);
}

template <typename R, typename TZ, int N, int NT>
cudaError_t inv_x_nt(const Geometry& g, const DctTables<R>& tb, PcgState* st, const R* t, TZ* z,
                     const double* kd, double kz_host, int check, int mode, cudaStream_t s,
                     typename XOf<TZ>::T* x, int par) {
  constexpr int L = FastX<N, NT>::L;
  const long long nrows = (long long)g.n1 * g.n2;
  const unsigned int nb = (unsigned int)((nrows + L - 1) / L);
  const size_t sm = fast_x_smem<R, N, NT>();
  if (mode == 2)
    k_fast_inv_x<R, TZ, N, 2, NT><<<nb, NT, sm, s>>>(g, tb, st, t, z, kd, kz_host, check, x, par);
  else
    k_fast_inv_x<R, TZ, N, 0, NT><<<nb, NT, sm, s>>>(g, tb, st, t, z, kd, kz_host, check, x, par);
  return cudaGetLastError();
}
template <typename R, typename TZ, int N>
cudaError_t inv_x_n(const Geometry& g, const DctTables<R>& tb, PcgState* st, const R* t, TZ* z,
                    const double* kd, double kz_host, int check, int mode, cudaStream_t s,
                    typename XOf<TZ>::T* x, int par, int nt) {
  if (nt == 128 || !fast_x_fits<R, N, 256>())
    return inv_x_nt<R, TZ, N, 128>(g, tb, st, t, z, kd, kz_host, check, mode, s, x, par);
  return inv_x_nt<R, TZ, N, 256>(g, tb, st, t, z, kd, kz_host, check, mode, s, x, par);
}

template <typename R, int N>
cudaError_t y_n(const Geometry& g, const DctTables<R>& tb, const PcgState* st, R* t,
                int inverse, int check, cudaStream_t s) {
  constexpr int C = FastCols<R, N>::C;
  dim3 grid((g.n0 + C - 1) / C, g.n2);
  const size_t sm = fast_y_smem<R, N>();
  // L2 prefetch distance: a quarter of the blocks resident on the GPU (FP32,
  // 512^3: forward 0.217 -> 0.197 ms, flat from a quarter to all of them;
  // backward unchanged), when the grid is more than two waves
  static const int resident = resident_blocks(k_fast_y<R, N, 0>, C * Fast<N>::P, sm);
  const int pf = resident > 0 && (long long)grid.x * grid.y > 2LL * resident ? resident / 4 : 0;
  if (inverse)
    k_fast_y<R, N, 1><<<grid, C * Fast<N>::P, sm, s>>>(g, tb, st, t, check, pf);
  else
    k_fast_y<R, N, 0><<<grid, C * Fast<N>::P, sm, s>>>(g, tb, st, t, check, pf);
  return cudaGetLastError();
}

template <typename R, int N, int NT>
cudaError_t q_x_nt(const Geometry& g, const DctTables<R>& tb, const QueueLaunch& ql, int par,
                   int inverse) {
  constexpr int L = FastX<N, NT>::L;
  const long long nrows = (long long)g.n1 * g.n2;
  const unsigned int nb = (unsigned int)((nrows + L - 1) / L);
  const size_t sm = fast_x_smem<R, N, NT>();
  const long long items = (long long)nb * ql.nsolves;
  if (inverse) {
    const unsigned int grid = persistent_grid(kq_fast_inv_x<R, N, NT>, NT, sm, items);
    kq_fast_inv_x<R, N, NT><<<grid, NT, sm, ql.s>>>(ql.q, ql.slot, ql.bs, g, tb, nb, par);
  } else {
    const unsigned int grid = persistent_grid(kq_fast_fwd_x<R, N, NT>, NT, sm, items);
    kq_fast_fwd_x<R, N, NT><<<grid, NT, sm, ql.s>>>(ql.q, ql.slot, ql.bs, g, tb, nb, par);
  }
  return cudaGetLastError();
}
template <typename R, int N>
cudaError_t q_x_n(const Geometry& g, const DctTables<R>& tb, const QueueLaunch& ql, int par,
                  int inverse, int nt) {
  if (nt == 128 || !fast_x_fits<R, N, 256>()) return q_x_nt<R, N, 128>(g, tb, ql, par, inverse);
  return q_x_nt<R, N, 256>(g, tb, ql, par, inverse);
}
template <typename R, int N>
cudaError_t q_y_n(const Geometry& g, const DctTables<R>& tb, const QueueLaunch& ql, int inverse,
                  int buf, int par) {
  constexpr int C = FastCols<R, N>::C;
  constexpr int NTY = C * Fast<N>::P;
  const unsigned int nbx = (unsigned int)((g.n0 + C - 1) / C);
  const size_t sm = fast_y_smem<R, N>();
  const long long items = (long long)nbx * g.n2 * ql.nsolves;
  if (inverse) {
    const unsigned int grid = persistent_grid(kq_fast_y<R, N, 1>, NTY, sm, items);
    kq_fast_y<R, N, 1><<<grid, NTY, sm, ql.s>>>(ql.q, ql.slot, ql.bs, g, tb, nbx, buf, par);
  } else {
    const unsigned int grid = persistent_grid(kq_fast_y<R, N, 0>, NTY, sm, items);
    kq_fast_y<R, N, 0><<<grid, NTY, sm, ql.s>>>(ql.q, ql.slot, ql.bs, g, tb, nbx, buf, par);
  }
  return cudaGetLastError();
}

template <typename R, int N, int NT>
cudaError_t attrs_nt() {
  cudaError_t e = cudaSuccess;
  if (!fast_x_fits<R, N, NT>()) return e;  // never launched
  const int sx = (int)fast_x_smem<R, N, NT>();
#define SETF(fn, b) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  SETF((k_fast_fwd_x<R, N, 0, double, NT>), sx);
  SETF((k_fast_fwd_x<R, N, 1, double, NT>), sx);
  SETF((k_fast_fwd_x<R, N, 2, double, NT>), sx);
  SETF((k_fast_inv_x<R, double, N, 0, NT>), sx);
  SETF((k_fast_inv_x<R, double, N, 2, NT>), sx);
  SETF((kq_fast_fwd_x<R, N, NT>), sx);
  SETF((kq_fast_inv_x<R, N, NT>), sx);
  if (sizeof(R) == 4) {
    SETF((k_fast_fwd_x<float, N, 0, float2, NT>), sx);
    SETF((k_fast_fwd_x<float, N, 1, float2, NT>), sx);
    SETF((k_fast_inv_x<float, float, N, 2, NT>), sx);
  }
#undef SETF
  return e;
}

template <typename R, int N>
cudaError_t attrs_n() {
  cudaError_t e = attrs_nt<R, N, 256>();
  if (e == cudaSuccess) e = attrs_nt<R, N, 128>();
  const int sy = (int)fast_y_smem<R, N>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fast_y<R, N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fast_y<R, N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kq_fast_y<R, N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kq_fast_y<R, N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
  return e;
}


// The lengths with register-resident transforms, and the per-length launchers
// each of them instantiates (PREFIX: "template" in fast_sizes_*.cu, "extern
// template" where they are only called).
#define ETC_FAST_SIZES(X) X(32) X(64) X(96) X(128) X(160) X(192) X(256) X(384) X(512) X(1024)

#define ETC_FAST_LAUNCHERS(PREFIX, N)                                                        \
  PREFIX cudaError_t fwd_x_n<double, N, double>(                                             \
      const Geometry&, const DctTables<double>&, PcgState*, double*, const double*,          \
      const double*, double*, const double*, double*, double*, int, double, int, cudaStream_t, \
      int);                                                                                  \
  PREFIX cudaError_t fwd_x_n<float, N, double>(                                              \
      const Geometry&, const DctTables<float>&, PcgState*, double*, const double*,           \
      const double*, double*, const double*, float*, double*, int, double, int, cudaStream_t, \
      int);                                                                                  \
  PREFIX cudaError_t fwd_x_n<float, N, float2>(                                              \
      const Geometry&, const DctTables<float>&, PcgState*, float2*, const float2*,           \
      const float2*, float2*, const double*, float*, double*, int, double, int, cudaStream_t, \
      int);                                                                                  \
  PREFIX cudaError_t inv_x_n<double, double, N>(                                             \
      const Geometry&, const DctTables<double>&, PcgState*, const double*, double*,          \
      const double*, double, int, int, cudaStream_t, double*, int, int);                     \
  PREFIX cudaError_t inv_x_n<float, double, N>(                                              \
      const Geometry&, const DctTables<float>&, PcgState*, const float*, double*,            \
      const double*, double, int, int, cudaStream_t, double*, int, int);                     \
  PREFIX cudaError_t inv_x_n<float, float, N>(                                               \
      const Geometry&, const DctTables<float>&, PcgState*, const float*, float*,             \
      const double*, double, int, int, cudaStream_t, float2*, int, int);                     \
  PREFIX cudaError_t y_n<double, N>(const Geometry&, const DctTables<double>&, const PcgState*, \
                                    double*, int, int, cudaStream_t);                        \
  PREFIX cudaError_t y_n<float, N>(const Geometry&, const DctTables<float>&, const PcgState*, \
                                   float*, int, int, cudaStream_t);                          \
  PREFIX cudaError_t q_x_n<double, N>(const Geometry&, const DctTables<double>&,              \
                                      const QueueLaunch&, int, int, int);                    \
  PREFIX cudaError_t q_x_n<float, N>(const Geometry&, const DctTables<float>&,                \
                                     const QueueLaunch&, int, int, int);                     \
  PREFIX cudaError_t q_y_n<double, N>(const Geometry&, const DctTables<double>&,              \
                                      const QueueLaunch&, int, int, int);                    \
  PREFIX cudaError_t q_y_n<float, N>(const Geometry&, const DctTables<float>&,                \
                                     const QueueLaunch&, int, int, int);                     \
  PREFIX cudaError_t attrs_n<double, N>();                                                   \
  PREFIX cudaError_t attrs_n<float, N>();
#define ETC_FAST_EXTERN(N) ETC_FAST_LAUNCHERS(extern template, N)
#define ETC_FAST_INSTANTIATE(N) ETC_FAST_LAUNCHERS(template, N)

}  // namespace etc
