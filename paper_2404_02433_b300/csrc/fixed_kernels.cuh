// Register-resident cosine transforms of the FP64 path in block floating point
// (fixed_point.cuh): the same four-step layout and data movement as the
// floating-point kernels of fast_kernels.cuh (Eq. (forward DCT) and Eq.
// (backward DCT) through the half-length complex FFT, Sec. 3.2), for their
// lengths n = 32 .. 1024, on FP64 vectors.  Each line (a row of
// axis 0, a column of axis 1) is converted to 64-bit integers with its own
// exponent after its largest exponent is known (a shuffle over the line's P
// threads on axis 0, a shared-memory maximum over its P warps on axis 1),
// transformed with integer arithmetic, and converted back to binary64.
#pragma once

#include "fast_kernels.cuh"
#include "fixed_point.cuh"

namespace etc {

constexpr bool fx_len_c(int n) {
  return n == 32 || n == 64 || n == 96 || n == 128 || n == 160 || n == 192 || n == 256 ||
         n == 384 || n == 512 || n == 1024;
}

// Four-step split m = P * Q of these kernels (P threads per line).  A 64-bit
// complex value takes twice the registers of an FP32 one, so where the
// floating-point split gives a thread 20 or 24 values (n = 160, 192, 384:
// up to 254 registers and 8 warps per SM) these kernels take twice the
// threads per line and half the values.  Q need not then be a multiple of P:
// the Q length-P DFTs of the second stage go round-robin over the P threads
// in E = ceil(Q / P) rounds, the last one partly idle.
constexpr int fx_p(int m) { return (m == 80 || m == 96) ? 8 : m == 192 ? 16 : fast_p(m); }
template <int N> struct FxFast {
  static constexpr int M = N / 2;
  static constexpr int P = fx_p(M);
  static constexpr int Q = M / P;
  static constexpr int E = (Q + P - 1) / P;  // second-stage rounds per thread
  static constexpr bool EXACT = Q % P == 0;
  static_assert(P * Q == M, "four-step split");
  // axis-0 shared layout, in complex units per row (as Fast<N>)
  static constexpr int SA = M + P;
  static constexpr int BS0 = Q * (P + 1);
  static constexpr int BS = BS0 + (((P - BS0) % 16) + 16) % 16;
  static constexpr int RS = SA > BS ? SA : BS;
  // axis-1 blocks of 16 columns: at most 128 registers a thread (255 for
  // more than 16 values a thread)
  static constexpr int YMIN = ((512 >> (Q > 16 ? 1 : 0)) / (16 * P)) > 0
                                  ? ((512 >> (Q > 16 ? 1 : 0)) / (16 * P)) : 1;
};
template <int N, int NT> struct FxX {  // axis-0 blocks of NT threads: L rows
  static constexpr int L = NT / FxFast<N>::P;
  static_assert(L * FxFast<N>::P == NT, "rows per block");
};
template <int N, int NT>
constexpr size_t fx_x_smem() {
  return (size_t)FxX<N, NT>::L * FxFast<N>::RS * sizeof(fxp::cx);
}
template <int N, int NT>
constexpr bool fx_x_fits() {
  return fx_x_smem<N, NT>() <= kFastSmemMax;
}

// First four-step stage of thread tau: DFT of length Q, then the twiddle
// exp(SIGN 2 pi i tau k1 / M) (forward sign stored).
template <int N, int SIGN>
__device__ __forceinline__ void fx_four_step_a(fxp::cx* v, const int4* __restrict__ tw4,
                                               int tau) {
  using F = FxFast<N>;
  fxp::Fb<F::Q, SIGN>::run(v);
  const int4* tw = tw4 + tau * F::Q;
#pragma unroll
  for (int k1 = 1; k1 < F::Q; ++k1) {
    const fxp::Kc2 w = fxp::ld_k2(tw + k1);
    v[k1] = SIGN < 0 ? fxp::crot(v[k1], w.a, w.b) : fxp::crotc(v[k1], w.a, w.b);
  }
}

// Largest exponent field over the P consecutive lanes of a line.
template <int P>
__device__ __forceinline__ int fx_lane_max(int e) {
#pragma unroll
  for (int o = 1; o < P; o *= 2) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  return e;
}

__device__ __forceinline__ fxp::cx ld_cx(const fxp::cx* p) {
  const longlong2 v = *reinterpret_cast<const longlong2*>(p);
  return fxp::mk(v.x, v.y);
}
__device__ __forceinline__ void st_cx(fxp::cx* p, fxp::cx v) {
  *reinterpret_cast<longlong2*>(p) = make_longlong2(v.x, v.y);
}

// ---------------------------------------------------------------- axis 1
// In place on t: every block owns C = 16 adjacent columns of one plane.  The
// conversions use the hardware's (the FP64 pipe is idle here); the axis-0
// forward kernel, whose FP64 pipe carries the x/r updates and the norm, uses
// the integer forms.
template <int N>
constexpr size_t fx_y_smem() {
  return (size_t)16 * (N / 2 + 1) * sizeof(fxp::cx) + 16 * sizeof(int);
}
template <int N, int INV>
__device__ __forceinline__ void fx_y_body(const Blk& b, Geometry g, DctTables<double> tb,
                                          const PcgState* st, double* __restrict__ t,
                                          int check) {
  using F = FxFast<N>;
  using fxp::cx;
  using fxp::i64;
  constexpr int M = F::M, P = F::P, Q = F::Q, E = F::E, C = 16;
  constexpr int SIGN = INV ? 1 : -1;
  constexpr int B = INV ? fxp::FxBits<M>::I : fxp::FxBits<M>::F;
  extern __shared__ __align__(16) unsigned char smraw[];
  cx* sm = reinterpret_cast<cx*>(smraw);                 // C (M + 1) complex
  int* emx = reinterpret_cast<int*>(smraw + (size_t)C * (M + 1) * sizeof(cx));
  if (check && st->done) return;
  const int4* tw4 = tb.fxq;
  const int4* post = tb.fxq + fxp::fx_off_post(M);
  const int4* pre = tb.fxq + fxp::fx_off_pre(M);
  const int c = threadIdx.x % C, tau = threadIdx.x / C;
  const int i = b.x * C + c;
  const bool ok = i < g.n0;
  const long long n0 = g.n0;
  double* col = t + (long long)b.y * g.plane + (ok ? i : 0);
  if (tau == 0) emx[c] = 1;
  __syncthreads();
  cx v[Q];
  int emax;
  if (!INV) {
    double d0[Q], d1[Q];
    int em = 1;
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int q = tau + P * s;  // z_q = (v_{2q}, v_{2q+1})
      d0[s] = ok ? col[vrow<N>(2 * q) * n0] : 0.0;
      d1[s] = ok ? col[vrow<N>(2 * q + 1) * n0] : 0.0;
      em = max(em, max(fxp::bexp(d0[s]), fxp::bexp(d1[s])));
    }
    atomicMax(&emx[c], em);
    __syncthreads();
    emax = emx[c];
#pragma unroll
    for (int s = 0; s < Q; ++s)
      v[s] = fxp::mk(fxp::to_fx_hw<B>(d0[s], emax), fxp::to_fx_hw<B>(d1[s], emax));
  } else {
    // the pre-twiddle of input j needs X_j, X_{n-j}, X_{m-j} and X_{m+j}:
    // stage the tile's columns as integers, form every V_k once, then a_j
    i64* sr = reinterpret_cast<i64*>(smraw);  // real rows of C integers
    double xs[2 * Q];
    int em = 1;
#pragma unroll
    for (int s = 0; s < 2 * Q; ++s) {
      xs[s] = ok ? col[(tau + P * s) * n0] : 0.0;
      em = max(em, fxp::bexp(xs[s]));
    }
    atomicMax(&emx[c], em);
    __syncthreads();
    emax = emx[c];
#pragma unroll
    for (int s = 0; s < 2 * Q; ++s) sr[(tau + P * s) * C + c] = fxp::to_fx_hw<B>(xs[s], emax);
    __syncthreads();
    cx vv[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int j = tau + P * s;
      vv[s] = fxp::inv_v(pre, j, sr[j * C + c], j ? sr[(N - j) * C + c] : 0);
    }
    cx vm = fxp::mk(0, 0);
    if (tau == 0) vm = fxp::inv_v(pre, M, sr[M * C + c], sr[M * C + c]);
    __syncthreads();  // the staged columns are read before V overwrites them
#pragma unroll
    for (int s = 0; s < Q; ++s) st_cx(sm + (tau + P * s) * C + c, vv[s]);
    if (tau == 0) st_cx(sm + M * C + c, vm);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int j = tau + P * s;
      v[s] = fxp::inv_a(pre, j, vv[s], ld_cx(sm + (M - j) * C + c));
    }
    __syncthreads();  // V is read before the transpose reuses the buffer
  }
  fx_four_step_a<N, SIGN>(v, tw4, tau);
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) st_cx(sm + (k1 * P + tau) * C + c, v[k1]);
  __syncthreads();
  cx u[E * P];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (!F::EXACT && tau + P * e >= Q) continue;  // this round's DFT index is past Q
#pragma unroll
    for (int tt = 0; tt < P; ++tt) u[e * P + tt] = ld_cx(sm + ((tau + P * e) * P + tt) * C + c);
    fxp::Fb<P, SIGN>::run(u + e * P);
  }
  const bool bad = emax == 2047;  // an infinity or NaN in the line
  if (!INV) {
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2)
        if (F::EXACT || tau + P * e < Q) st_cx(sm + (tau + P * e + Q * k2) * C + c, u[e * P + k2]);
    __syncthreads();
    const int e2 = emax - 1022 - B;
    // only a line near the top of the range (or holding an infinity or NaN)
    // takes the tests for the range's top
    auto out = [&](auto satc) {
      constexpr bool S = decltype(satc)::value;
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) {
          if (!F::EXACT && tau + P * e >= Q) continue;
          const int k = tau + P * e + Q * k2;
          i64 xa, xb;
          fxp::untangle(u[e * P + k2], ld_cx(sm + (k ? M - k : 0) * C + c), post, k, M, xa, xb);
          if (ok) {
            col[k * n0] = (S && bad) ? fxp::nan_f64() : fxp::from_fx_hw<S>(xa, e2);
            col[(k ? N - k : M) * n0] = (S && bad) ? fxp::nan_f64() : fxp::from_fx_hw<S>(xb, e2);
          }
        }
    };
    if (bad || 1086 + e2 >= 2047) out(std::true_type{});
    else out(std::false_type{});
  } else {
    // the pre-twiddle omitted 1 / (2m) = f 2^E0: a power of two goes to the
    // exponent, otherwise one more product by f (after halving: the FFT output
    // may reach 2^62, a product's operand may not)
    using FB = fxp::FxBits<M>;
    constexpr fxp::Kc kf = fxp::kc(FB::f());
    const int e2 = emax - 1022 - B + FB::E + (FB::POW2 ? -1 : 1);
    auto outs = [&](auto satc) {
      constexpr bool S = decltype(satc)::value;
      auto out = [&](i64 y) {
        if (S && bad) return fxp::nan_f64();
        if constexpr (FB::POW2) return fxp::from_fx_hw<S>(y, e2);
        else return fxp::from_fx_hw<S>(fxp::mulk(y >> 1, kf), e2);
      };
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) {
          if (!F::EXACT && tau + P * e >= Q) continue;
          const int j = tau + P * e + Q * k2;  // z_j = (v_{2j}, v_{2j+1})
          if (ok) {
            col[vrow<N>(2 * j) * n0] = out(u[e * P + k2].x);
            col[vrow<N>(2 * j + 1) * n0] = out(u[e * P + k2].y);
          }
        }
    };
    if (bad || 1086 + e2 >= 2047) outs(std::true_type{});
    else outs(std::false_type{});
  }
}
template <int N, int INV>
__global__ void __launch_bounds__(16 * FxFast<N>::P, FxFast<N>::YMIN)
    k_fx_y(Geometry g, DctTables<double> tb, const PcgState* st, double* __restrict__ t,
           int check) {
  fx_y_body<N, INV>(hw_blk(), g, tb, st, t, check);
}

// ---------------------------------------------------------------- axis 1, three stages
// The axis-1 transforms for m = 8 * 8 * P2 (n = 256, 512, 1024) over P = 8 P2
// threads per line with 8 values each, half the registers of the two-stage
// split (16 values), so that more warps hide the latency of the integer
// products: stage 1, thread tau: DFT-8 of z_{tau + P s} and the twiddle
// exp(SIGN 2 pi i tau k1 / m); stage 2, thread (k1, tb): DFT-8 over ta of the
// stage-1 values of tau = tb + P2 ta and the twiddle exp(SIGN 2 pi i tb ka / P);
// stage 3: DFT-P2 over tb for Q / P2 pairs (k1, ka) a thread, giving
// Z_{k1 + 8 ka + 64 kb}.  Two shared-memory exchanges instead of one, and the
// second-stage twiddles, in exchange for the occupancy.
template <int N> struct FxY3 {
  static constexpr int M = N / 2, Q = 8, P2 = M / 64, P = Q * P2, R = Q / P2;
  static constexpr int C = 256 / P;  // columns per block: blocks of 256 threads
  static constexpr int NT = C * P;
  static_assert(M == Q * Q * P2 && P2 >= 2 && P2 <= 8, "three-stage split");
};
template <int N>
constexpr size_t fx_y3_smem() {
  return (size_t)FxY3<N>::C * (N / 2 + 1) * sizeof(fxp::cx) + FxY3<N>::C * sizeof(int);
}
template <int N, int INV>
__device__ __forceinline__ void fx_y3_body(const Blk& b, Geometry g, DctTables<double> tb,
                                           const PcgState* st, double* __restrict__ t,
                                           int check) {
  using Y = FxY3<N>;
  using fxp::cx;
  using fxp::i64;
  constexpr int M = Y::M, Q = Y::Q, P2 = Y::P2, P = Y::P, R = Y::R, C = Y::C;
  constexpr int SIGN = INV ? 1 : -1;
  constexpr int B = INV ? fxp::FxBits<M>::I : fxp::FxBits<M>::F;
  extern __shared__ __align__(16) unsigned char smraw[];
  cx* sm = reinterpret_cast<cx*>(smraw);  // C (M + 1) complex
  int* emx = reinterpret_cast<int*>(smraw + (size_t)C * (M + 1) * sizeof(cx));
  if (check && st->done) return;
  const int4* post = tb.fxq + fxp::fx_off_post(M);
  const int4* pre = tb.fxq + fxp::fx_off_pre(M);
  const int4* tw1 = tb.fxq + fxp::fx_off_y3(M);
  const int4* tw2 = tw1 + M;
  const int c = threadIdx.x % C, tau = threadIdx.x / C;
  const int i = b.x * C + c;
  const bool ok = i < g.n0;
  const long long n0 = g.n0;
  double* col = t + (long long)b.y * g.plane + (ok ? i : 0);
  if (tau == 0) emx[c] = 1;
  __syncthreads();
  cx v[Q];
  int emax;
  if (!INV) {
    double d0[Q], d1[Q];
    int em = 1;
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int q = tau + P * s;  // z_q = (v_{2q}, v_{2q+1})
      d0[s] = ok ? col[vrow<N>(2 * q) * n0] : 0.0;
      d1[s] = ok ? col[vrow<N>(2 * q + 1) * n0] : 0.0;
      em = max(em, max(fxp::bexp(d0[s]), fxp::bexp(d1[s])));
    }
    atomicMax(&emx[c], em);
    __syncthreads();
    emax = emx[c];
#pragma unroll
    for (int s = 0; s < Q; ++s)
      v[s] = fxp::mk(fxp::to_fx_hw<B>(d0[s], emax), fxp::to_fx_hw<B>(d1[s], emax));
  } else {
    i64* sr = reinterpret_cast<i64*>(smraw);  // real rows of C integers
    double xs[2 * Q];
    int em = 1;
#pragma unroll
    for (int s = 0; s < 2 * Q; ++s) {
      xs[s] = ok ? col[(tau + P * s) * n0] : 0.0;
      em = max(em, fxp::bexp(xs[s]));
    }
    atomicMax(&emx[c], em);
    __syncthreads();
    emax = emx[c];
#pragma unroll
    for (int s = 0; s < 2 * Q; ++s) sr[(tau + P * s) * C + c] = fxp::to_fx_hw<B>(xs[s], emax);
    __syncthreads();
    cx vv[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int j = tau + P * s;
      vv[s] = fxp::inv_v(pre, j, sr[j * C + c], j ? sr[(N - j) * C + c] : 0);
    }
    cx vm = fxp::mk(0, 0);
    if (tau == 0) vm = fxp::inv_v(pre, M, sr[M * C + c], sr[M * C + c]);
    __syncthreads();  // the staged columns are read before V overwrites them
#pragma unroll
    for (int s = 0; s < Q; ++s) st_cx(sm + (tau + P * s) * C + c, vv[s]);
    if (tau == 0) st_cx(sm + M * C + c, vm);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int j = tau + P * s;
      v[s] = fxp::inv_a(pre, j, vv[s], ld_cx(sm + (M - j) * C + c));
    }
    __syncthreads();  // V is read before stage 1 reuses the buffer
  }
  // stage 1: DFT-8 over s, twiddle exp(SIGN 2 pi i tau k1 / M); values to S1[k1][tau]
  fxp::Fb<Q, SIGN>::run(v);
#pragma unroll
  for (int k1 = 1; k1 < Q; ++k1) {
    const fxp::Kc2 w = fxp::ld_k2(tw1 + tau * Q + k1);
    v[k1] = SIGN < 0 ? fxp::crot(v[k1], w.a, w.b) : fxp::crotc(v[k1], w.a, w.b);
  }
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) st_cx(sm + (k1 * P + tau) * C + c, v[k1]);
  __syncthreads();
  // stage 2, thread (k1, tb): DFT-8 over ta of S1[k1][tb + P2 ta], twiddle
  // exp(SIGN 2 pi i tb ka / P); values to S2[k1][ka][tb]
  {
    const int k1 = tau / P2, tbi = tau % P2;
#pragma unroll
    for (int ta = 0; ta < Q; ++ta) v[ta] = ld_cx(sm + (k1 * P + tbi + P2 * ta) * C + c);
    fxp::Fb<Q, SIGN>::run(v);
#pragma unroll
    for (int ka = 1; ka < Q; ++ka) {
      const fxp::Kc2 w = fxp::ld_k2(tw2 + tbi * Q + ka);
      v[ka] = SIGN < 0 ? fxp::crot(v[ka], w.a, w.b) : fxp::crotc(v[ka], w.a, w.b);
    }
    __syncthreads();  // S1 is read before S2 overwrites it
#pragma unroll
    for (int ka = 0; ka < Q; ++ka) st_cx(sm + ((k1 * Q + ka) * P2 + tbi) * C + c, v[ka]);
  }
  __syncthreads();
  // stage 3: pairs pr = k1 Q + ka (R a thread), DFT-P2 over tb; u[r P2 + kb]
  // holds Z_k, k = k1 + Q ka + Q^2 kb
  cx u[Q];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int pr = tau + P * r;
#pragma unroll
    for (int tt = 0; tt < P2; ++tt) u[r * P2 + tt] = ld_cx(sm + (pr * P2 + tt) * C + c);
    fxp::Fb<P2, SIGN>::run(u + r * P2);
  }
  auto kof = [&](int r, int kb) {
    const int pr = tau + P * r;
    return pr / Q + Q * (pr % Q) + Q * Q * kb;
  };
  const bool bad = emax == 2047;  // an infinity or NaN in the line
  if (!INV) {
    __syncthreads();  // S2 is read before Z overwrites it
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int kb = 0; kb < P2; ++kb) st_cx(sm + kof(r, kb) * C + c, u[r * P2 + kb]);
    __syncthreads();
    const int e2 = emax - 1022 - B;
    auto out = [&](auto satc) {  // the tests for the range's top near it only
      constexpr bool S = decltype(satc)::value;
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int kb = 0; kb < P2; ++kb) {
          const int k = kof(r, kb);
          i64 xa, xb;
          fxp::untangle(u[r * P2 + kb], ld_cx(sm + (k ? M - k : 0) * C + c), post, k, M, xa, xb);
          if (ok) {
            col[k * n0] = (S && bad) ? fxp::nan_f64() : fxp::from_fx_hw<S>(xa, e2);
            col[(k ? N - k : M) * n0] = (S && bad) ? fxp::nan_f64() : fxp::from_fx_hw<S>(xb, e2);
          }
        }
    };
    if (bad || 1086 + e2 >= 2047) out(std::true_type{});
    else out(std::false_type{});
  } else {
    // the pre-twiddle omitted 1 / (2m), a power of two here
    static_assert(fxp::FxBits<M>::POW2, "power-of-two lengths");
    const int e2 = emax - 1022 - B + fxp::FxBits<M>::E - 1;
    auto out = [&](auto satc) {  // the tests for the range's top near it only
      constexpr bool S = decltype(satc)::value;
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int kb = 0; kb < P2; ++kb) {
          const int j = kof(r, kb);  // z_j = (v_{2j}, v_{2j+1})
          if (ok) {
            col[vrow<N>(2 * j) * n0] =
                (S && bad) ? fxp::nan_f64() : fxp::from_fx_hw<S>(u[r * P2 + kb].x, e2);
            col[vrow<N>(2 * j + 1) * n0] =
                (S && bad) ? fxp::nan_f64() : fxp::from_fx_hw<S>(u[r * P2 + kb].y, e2);
          }
        }
    };
    if (bad || 1086 + e2 >= 2047) out(std::true_type{});
    else out(std::false_type{});
  }
}
template <int N, int INV>
__global__ void __launch_bounds__(FxY3<N>::NT, 3)
    k_fx_y3(Geometry g, DctTables<double> tb, const PcgState* st, double* __restrict__ t,
            int check) {
  fx_y3_body<N, INV>(hw_blk(), g, tb, st, t, check);
}

// ---------------------------------------------------------------- axis 0, forward
// Same contract as k_fast_fwd_x on FP64 vectors (MODE 0 initial residual, 1 PCG
// update with x moved here, 2 transform only).
template <int N, int MODE, int NT>
__device__ __forceinline__ void fx_fwd_x_body(const Blk& b, Geometry g, DctTables<double> tb,
                                              PcgState* st, double* __restrict__ x,
                                              const double* __restrict__ w,
                                              const double* __restrict__ q,
                                              double* __restrict__ r,
                                              const double* __restrict__ rin,
                                              double* __restrict__ t, double* partials, int par,
                                              double rtol2, int pf) {
  using F = FxFast<N>;
  using fxp::cx;
  using fxp::i64;
  constexpr int M = F::M, P = F::P, Q = F::Q, E = F::E, RS = F::RS;
  constexpr int L = FxX<N, NT>::L;
  constexpr int B = fxp::FxBits<M>::F;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double sh[32];
  __shared__ int flag;
  if (MODE != 2 && st->done) return;
  cx* A = reinterpret_cast<cx*>(smraw);  // rows of RS complex: staging, transpose, Z
  double* Ar = reinterpret_cast<double*>(smraw);
  const long long nrows = (long long)g.n1 * g.n2;
  const long long row0 = (long long)b.x * L;
  const double alpha = (MODE == 1) ? st->alpha[par] : 0.0;
  if (MODE == 1 && pf > 0 && threadIdx.x == 0) {
    // the rows of the block pf blocks ahead go to L2 while this block computes
    const long long pr = row0 + (long long)pf * L;
    if (pr < nrows) {
      const unsigned int bytes = (unsigned int)(min((long long)L, nrows - pr) * N * 8);
      const long long c = pr * N;
      l2_prefetch(r + c, bytes);
      l2_prefetch(q + c, bytes);
      l2_prefetch(x + c, bytes);
      l2_prefetch(w + c, bytes);
    }
  }
  double acc = 0.0;
  constexpr int NP = L * M;  // element pairs of the block
  // pairs per thread whose loads are in flight together (4: 1.95 -> 1.80 ms at
  // 512^3 against 2), or the largest of 2, 1 that divides the block's pairs
  constexpr int U = (L * M) % (NT * 4) == 0 ? 4 : (L * M) % (NT * 2) == 0 ? 2 : 1;
  static_assert(NP % (NT * U) == 0, "pair rounds");
  for (int p0 = threadIdx.x; p0 < NP; p0 += NT * U) {
    VPair<double> rv[U], qv[U], xv[U], wv[U];
    double2 dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = p0 + NT * u;
      const int l = p / M, i2 = p % M;
      const long long row = row0 + l;
      rv[u].a = rv[u].b = 0.0;
      qv[u] = rv[u]; xv[u] = rv[u]; wv[u] = rv[u];
      dv[u] = make_double2(0.0, 0.0);
      if (row < nrows) {
        const long long c = row * N + 2 * i2;
        if (MODE == 2) dv[u] = *reinterpret_cast<const double2*>(rin + c);
        else rv[u] = ld_pair(r + c);
        if (MODE == 1) {
          qv[u] = ld_pair(q + c);
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
      double in0, in1;
      if (MODE == 2) {
        in0 = dv[u].x;
        in1 = dv[u].y;
      } else {
        double v0 = rv[u].a, v1 = rv[u].b;
        if (row < nrows) {
          const long long c = row * N + 2 * i2;
          if (MODE == 1) {
            st_pair(x + c, fma(alpha, wv[u].a, xv[u].a), fma(alpha, wv[u].b, xv[u].b));
            v0 = fma(-alpha, qv[u].a, v0);
            v1 = fma(-alpha, qv[u].b, v1);
            st_pair(r + c, v0, v1);
          }
          acc = fma(v0, v0, acc);
          acc = fma(v1, v1, acc);
        }
        in0 = v0;
        in1 = v1;
      }
      // element 2 i2 -> v_{i2}; element 2 i2 + 1 -> v_{n-1-i2}
      Ar[l * 2 * RS + i2] = in0;
      Ar[l * 2 * RS + N - 1 - i2] = in1;
    }
  }
  __syncthreads();
  const int l = threadIdx.x / P, tau = threadIdx.x % P;
  cx v[Q];
  int emax;
  {
    double2 dv[Q];
    int em = 1;
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      dv[s] = *reinterpret_cast<const double2*>(A + l * RS + tau + P * s);
      em = max(em, max(fxp::bexp(dv[s].x), fxp::bexp(dv[s].y)));
    }
    emax = fx_lane_max<P>(em);
    if (emax >= 10 + B) {  // zeros and subnormals of the row round to 0 anyway
#pragma unroll
      for (int s = 0; s < Q; ++s)
        v[s] = fxp::mk(fxp::to_fx<B, false>(dv[s].x, emax), fxp::to_fx<B, false>(dv[s].y, emax));
    } else {
#pragma unroll
      for (int s = 0; s < Q; ++s)
        v[s] = fxp::mk(fxp::to_fx<B>(dv[s].x, emax), fxp::to_fx<B>(dv[s].y, emax));
    }
  }
  fx_four_step_a<N, -1>(v, tb.fxq, tau);
  __syncthreads();  // the row is read before the transpose overwrites it
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) st_cx(A + l * RS + k1 * (P + 1) + tau, v[k1]);
  __syncthreads();
  cx u[E * P];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (!F::EXACT && tau + P * e >= Q) continue;  // this round's DFT index is past Q
#pragma unroll
    for (int tt = 0; tt < P; ++tt) u[e * P + tt] = ld_cx(A + l * RS + (tau + P * e) * (P + 1) + tt);
    fxp::Fb<P, -1>::run(u + e * P);
  }
  __syncthreads();  // the transpose is read before Z overwrites it
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2)
      if (F::EXACT || tau + P * e < Q) st_cx(A + l * RS + tau + P * e + Q * k2, u[e * P + k2]);
  __syncthreads();
  const long long row = row0 + l;
  const int4* post = tb.fxq + fxp::fx_off_post(M);
  const bool bad = emax == 2047;  // an infinity or NaN in the row
  const int e2 = emax - 1022 - B;
  // |Y| < 2^63 puts an output's biased exponent at most at 1086 + e2: only a
  // row whose largest element lies within 2^(64 - B) of the top of the range
  // (and a row holding an infinity or NaN) takes the tests for the range's top
  const bool sat = bad || 1086 + e2 >= 2047;
  auto out = [&](auto satc) {
    constexpr bool S = decltype(satc)::value;
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) {
        if (!F::EXACT && tau + P * e >= Q) continue;
        const int k = tau + P * e + Q * k2;
        i64 xa, xb;
        fxp::untangle(u[e * P + k2], ld_cx(A + l * RS + (k ? M - k : 0)), post, k, M, xa, xb);
        if (row < nrows) {
          t[row * N + k] = (S && bad) ? fxp::nan_f64() : fxp::from_fx<S>(xa, e2);
          t[row * N + (k ? N - k : M)] = (S && bad) ? fxp::nan_f64() : fxp::from_fx<S>(xb, e2);
        }
      }
  };
  if (sat) out(std::true_type{});
  else out(std::false_type{});
  if (MODE != 2) fwd_x_residual_tail<MODE>(acc, st, partials, rtol2, sh, &flag, par, false, b);
}
template <int N, int MODE, int NT>
__global__ void __launch_bounds__(NT)
    k_fx_fwd_x(Geometry g, DctTables<double> tb, PcgState* st, double* __restrict__ x,
               const double* __restrict__ w, const double* __restrict__ q,
               double* __restrict__ r, const double* __restrict__ rin, double* __restrict__ t,
               double* partials, int par, double rtol2, int pf) {
  fx_fwd_x_body<N, MODE, NT>(hw_blk(), g, tb, st, x, w, q, r, rin, t, partials, par, rtol2, pf);
}

// ---------------------------------------------------------------- axis 0, backward
// Same contract as k_fast_inv_x on FP64 vectors: u = scale * (backward DCT of
// t along axis 0), then MODE 0: z = u; MODE 2: w = u + beta w in place (z
// points at w).  The output converts with the hardware conversion and takes
// scale = 1 / kappa_ref^z, times the 1 / (2m) the pre-twiddle omitted, as one
// FP64 product (the FP64 pipe here carries only the w update; 1.47 -> 1.38 ms
// at 512^3 against an integer conversion and a fixed-point product).
template <int N, int MODE, int NT>
__device__ __forceinline__ void fx_inv_x_body(const Blk& b, Geometry g, DctTables<double> tb,
                                              PcgState* st, const double* __restrict__ t,
                                              double* __restrict__ z, const double* kd,
                                              double kz_host, int check, int pf) {
  using F = FxFast<N>;
  using fxp::cx;
  using fxp::i64;
  constexpr int M = F::M, P = F::P, Q = F::Q, E = F::E, RS = F::RS;
  constexpr int L = FxX<N, NT>::L;
  constexpr int SR = N + P;  // real stride of the staged input rows
  constexpr int B = fxp::FxBits<M>::I;
  extern __shared__ __align__(16) unsigned char smraw[];
  if (check && st->done) return;
  cx* A = reinterpret_cast<cx*>(smraw);  // rows of RS complex: V, transpose, z
  double* Ar = reinterpret_cast<double*>(smraw);
  i64* Ai = reinterpret_cast<i64*>(smraw);
  const long long nrows = (long long)g.n1 * g.n2;
  const long long row0 = (long long)b.x * L;
  if (pf > 0 && threadIdx.x == 0) {
    // the rows of the block pf blocks ahead go to L2 while this block computes
    const long long pr = row0 + (long long)pf * L;
    if (pr < nrows) {
      const unsigned int bytes = (unsigned int)(min((long long)L, nrows - pr) * N * 8);
      l2_prefetch(t + pr * N, bytes);
      if (MODE == 2) l2_prefetch(z + pr * N, bytes);
    }
  }
  // stage the block's rows in natural order, 16 bytes per access, all of a
  // thread's loads issued before the first shared-memory store
  constexpr int NR = L * N / 2 / NT;
  static_assert(NR * NT * 2 == L * N, "staging rounds");
  {
    double2 val[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int e = threadIdx.x + NT * r;
      const int l = (e * 2) / N, i = (e * 2) % N;
      const long long row = row0 + l;
      val[r] = row < nrows ? *reinterpret_cast<const double2*>(t + row * N + i)
                           : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int e = threadIdx.x + NT * r;
      const int l = (e * 2) / N, i = (e * 2) % N;
      *reinterpret_cast<double2*>(Ar + l * SR + i) = val[r];
    }
  }
  __syncthreads();
  const int l = threadIdx.x / P, tau = threadIdx.x % P;
  const double* X = Ar + l * SR;
  int em = 1;
#pragma unroll
  for (int r = 0; r < 2 * Q; ++r) em = max(em, fxp::bexp(X[tau + P * r]));
  const int emax = fx_lane_max<P>(em);
  const int4* pre = tb.fxq + fxp::fx_off_pre(M);
  // V_k = e^{i t_k} (X_k - i X_{n-k}) for the thread's own k = tau + P s, and V_m
  cx vv[Q];
  cx vm = fxp::mk(0, 0);
  auto in = [&](auto lowc) {  // LOW false: zeros and subnormals round to 0 anyway
    constexpr bool LOW = decltype(lowc)::value;
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int j = tau + P * s;
      vv[s] = fxp::inv_v(pre, j, fxp::to_fx<B, LOW>(X[j], emax),
                         j ? fxp::to_fx<B, LOW>(X[N - j], emax) : 0);
    }
    if (tau == 0) {
      const i64 xm = fxp::to_fx<B, LOW>(X[M], emax);
      vm = fxp::inv_v(pre, M, xm, xm);
    }
  };
  if (emax >= 10 + B) in(std::false_type{});
  else in(std::true_type{});
  __syncthreads();  // the staged rows are read before V overwrites them
#pragma unroll
  for (int s = 0; s < Q; ++s) st_cx(A + l * RS + tau + P * s, vv[s]);
  if (tau == 0) st_cx(A + l * RS + M, vm);
  __syncthreads();
  cx v[Q];
#pragma unroll
  for (int s = 0; s < Q; ++s) {
    const int j = tau + P * s;
    v[s] = fxp::inv_a(pre, j, vv[s], ld_cx(A + l * RS + M - j));
  }
  fx_four_step_a<N, 1>(v, tb.fxq, tau);
  __syncthreads();  // V is read before the transpose overwrites it
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) st_cx(A + l * RS + k1 * (P + 1) + tau, v[k1]);
  __syncthreads();
  cx u[E * P];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (!F::EXACT && tau + P * e >= Q) continue;  // this round's DFT index is past Q
#pragma unroll
    for (int tt = 0; tt < P; ++tt) u[e * P + tt] = ld_cx(A + l * RS + (tau + P * e) * (P + 1) + tt);
    fxp::Fb<P, 1>::run(u + e * P);
  }
  __syncthreads();  // the transpose is read before z overwrites it
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2)
      if (F::EXACT || tau + P * e < Q) st_cx(A + l * RS + tau + P * e + Q * k2, u[e * P + k2]);
  // the row's exponent for the output pass, which walks other rows; rows near
  // the top of the range (or holding an infinity or NaN) put the block on the
  // output path with the tests for the range's top
  __shared__ int erow[NT / P];
  __shared__ int anysat;
  if (threadIdx.x == 0) anysat = 0;
  __syncthreads();
  if (tau == 0) {
    erow[l] = emax;
    if (emax == 2047 || 1086 + emax - 1022 - B >= 2047) anysat = 1;
  }
  __syncthreads();
  // scale = 1 / (kappa_ref^z 2m): the pre-twiddle omitted 1 / (2m)
  const double scale = 1.0 / ((kd ? kd[2] : kz_host) * (2.0 * M));
  constexpr int EOFF = -1022 - B;
  const double beta = (MODE == 2) ? st->beta : 0.0;
  constexpr int NQ = L * M / NT;      // element pairs per thread
  // pairs whose loads are in flight together: the largest of 4, 2, 1 dividing NQ
  // (8 measured slower: 1.47 -> 1.60 ms at 512^3)
  constexpr int G = NQ % 4 == 0 ? 4 : NQ % 2 == 0 ? 2 : 1;
  static_assert(NQ % G == 0, "pair groups");
  auto out = [&](auto satc) {
    constexpr bool S = decltype(satc)::value;
#pragma unroll 1
    for (int r0 = 0; r0 < NQ; r0 += G) {
      VPair<double> wo[G];
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int p = threadIdx.x + NT * (r0 + u);
        const long long row = row0 + p / M;
        wo[u].a = wo[u].b = 0.0;
        if (MODE == 2 && row < nrows) wo[u] = ld_pair(z + row * N + 2 * (p % M));
      }
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int p = threadIdx.x + NT * (r0 + u);
        const int lr = p / M, i2 = p % M;
        const long long row = row0 + lr;
        if (row >= nrows) continue;
        const long long c = row * N + 2 * i2;
        const int er = erow[lr];
        const int e2 = er + EOFF;
        // element 2 i2 <- v_{i2}; element 2 i2 + 1 <- v_{n-1-i2}
        double u0 = fxp::from_fx_hw<S>(Ai[lr * 2 * RS + i2], e2) * scale;
        double u1 = fxp::from_fx_hw<S>(Ai[lr * 2 * RS + N - 1 - i2], e2) * scale;
        if (S && er == 2047) u0 = u1 = fxp::nan_f64();
        if (MODE == 2) st_pair(z + c, fma(beta, wo[u].a, u0), fma(beta, wo[u].b, u1));
        else st_pair(z + c, u0, u1);
      }
    }
  };
  if (anysat) out(std::true_type{});
  else out(std::false_type{});
}
template <int N, int MODE, int NT>
__global__ void __launch_bounds__(NT)
    k_fx_inv_x(Geometry g, DctTables<double> tb, PcgState* st, const double* __restrict__ t,
               double* __restrict__ z, const double* kd, double kz_host, int check, int pf) {
  fx_inv_x_body<N, MODE, NT>(hw_blk(), g, tb, st, t, z, kd, kz_host, check, pf);
}

// ---------------------------------------------------------------- batch work queue
// Persistent forms of the three transforms over the FP64 solves of a batch
// class (BatchQueue in etc_internal.cuh), as kq_fast_* in fast_kernels.cuh.
template <int N, int NT>
__global__ void __launch_bounds__(NT)
    kq_fx_fwd_x(BatchQueue* q, int slot, const BatchSolve* bs, Geometry g,
                DctTables<double> tb, unsigned int nb, int par) {
  queue_loop(q, slot, nb, [&](int sv, unsigned int l) {
    const BatchSolve& a = bs[sv];
    fx_fwd_x_body<N, 1, NT>(item_blk(l, nb, 1, 1), g, tb, a.st, a.x, a.w, a.q, a.r, nullptr,
                            a.t64, a.partials, par, 0.0, 0);
  });
}
template <int N, int INV>
__global__ void __launch_bounds__(16 * FxFast<N>::P, FxFast<N>::YMIN)
    kq_fx_y(BatchQueue* q, int slot, const BatchSolve* bs, Geometry g, DctTables<double> tb,
            unsigned int nbx) {
  const unsigned int per = nbx * (unsigned int)g.n2;
  queue_loop(q, slot, per, [&](int sv, unsigned int l) {
    const BatchSolve& a = bs[sv];
    fx_y_body<N, INV>(item_blk(l, nbx, (unsigned int)g.n2, 1), g, tb, a.st, a.t64, 1);
  });
}
template <int N, int NT>
__global__ void __launch_bounds__(NT)
    kq_fx_inv_x(BatchQueue* q, int slot, const BatchSolve* bs, Geometry g,
                DctTables<double> tb, unsigned int nb) {
  queue_loop(q, slot, nb, [&](int sv, unsigned int l) {
    const BatchSolve& a = bs[sv];
    fx_inv_x_body<N, 2, NT>(item_blk(l, nb, 1, 1), g, tb, a.st, a.t64, a.w, a.st->kref, 1.0, 1, 0);
  });
}

// ---------------------------------------------------------------- per-size launchers
// Defined here, instantiated per length in fixed_sizes_*.cu, called by
// fixed_dispatch.cu.  The axis-0 kernels' shared memory is laid out as the
// floating-point kernels' (16-byte complex values), with this split's P and Q.
template <int N, int NT>
cudaError_t fx_fwd_x_nt(const Geometry& g, const DctTables<double>& tb, PcgState* st, double* x,
                        const double* w, const double* q, double* r, const double* rin,
                        double* t, double* partials, int par, double rtol2, int mode,
                        cudaStream_t s) {
  constexpr int L = FxX<N, NT>::L;
  const long long nrows = (long long)g.n1 * g.n2;
  const unsigned int nb = (unsigned int)((nrows + L - 1) / L);
  const size_t sm = fx_x_smem<N, NT>();
  // PCG update: the block's x, w, r, q rows about 3 MB ahead go to L2
  // (512^3: 1.77 -> 1.73 ms at 3 MB; 9 MB and more ahead slower than none),
  // when the grid is more than two waves
  static const int resident = resident_blocks(k_fx_fwd_x<N, 1, NT>, NT, sm);
  const int pf = resident > 0 && (long long)nb > 2LL * resident
                     ? max(1, (int)((3u << 20) / (4u * L * N * 8u)))
                     : 0;
  if (mode == 0)
    k_fx_fwd_x<N, 0, NT><<<nb, NT, sm, s>>>(g, tb, st, x, w, q, r, rin, t, partials, par, rtol2, pf);
  else if (mode == 1)
    k_fx_fwd_x<N, 1, NT><<<nb, NT, sm, s>>>(g, tb, st, x, w, q, r, rin, t, partials, par, rtol2, pf);
  else
    k_fx_fwd_x<N, 2, NT><<<nb, NT, sm, s>>>(g, tb, st, x, w, q, r, rin, t, partials, par, rtol2, pf);
  return cudaGetLastError();
}
template <int N>
cudaError_t fx_fwd_x_n(const Geometry& g, const DctTables<double>& tb, PcgState* st, double* x,
                       const double* w, const double* q, double* r, const double* rin, double* t,
                       double* partials, int par, double rtol2, int mode, cudaStream_t s,
                       int nt) {
  if (nt == 128 || !fx_x_fits<N, 256>())
    return fx_fwd_x_nt<N, 128>(g, tb, st, x, w, q, r, rin, t, partials, par, rtol2, mode, s);
  return fx_fwd_x_nt<N, 256>(g, tb, st, x, w, q, r, rin, t, partials, par, rtol2, mode, s);
}

template <int N, int NT>
cudaError_t fx_inv_x_nt(const Geometry& g, const DctTables<double>& tb, PcgState* st,
                        const double* t, double* z, const double* kd, double kz_host, int check,
                        int mode, cudaStream_t s) {
  constexpr int L = FxX<N, NT>::L;
  const long long nrows = (long long)g.n1 * g.n2;
  const unsigned int nb = (unsigned int)((nrows + L - 1) / L);
  const size_t sm = fx_x_smem<N, NT>();
  // L2 prefetch distance: 3/8 of the blocks resident on the GPU (at 512^3
  // 1.43 -> 1.35 ms, flat from 1/4 to 1/2), when the grid is more than two
  // waves; the first wave's rows are read cold either way
  static const int resident = resident_blocks(k_fx_inv_x<N, 2, NT>, NT, sm);
  const int pf = resident > 0 && (long long)nb > 2LL * resident ? resident * 3 / 8 : 0;
  if (mode == 2)
    k_fx_inv_x<N, 2, NT><<<nb, NT, sm, s>>>(g, tb, st, t, z, kd, kz_host, check, pf);
  else
    k_fx_inv_x<N, 0, NT><<<nb, NT, sm, s>>>(g, tb, st, t, z, kd, kz_host, check, pf);
  return cudaGetLastError();
}
template <int N>
cudaError_t fx_inv_x_n(const Geometry& g, const DctTables<double>& tb, PcgState* st,
                       const double* t, double* z, const double* kd, double kz_host, int check,
                       int mode, cudaStream_t s, int nt) {
  if (nt == 128 || !fx_x_fits<N, 256>())
    return fx_inv_x_nt<N, 128>(g, tb, st, t, z, kd, kz_host, check, mode, s);
  return fx_inv_x_nt<N, 256>(g, tb, st, t, z, kd, kz_host, check, mode, s);
}

template <int N>
cudaError_t fx_y_n(const Geometry& g, const DctTables<double>& tb, const PcgState* st, double* t,
                   int inverse, int check, cudaStream_t s) {
  dim3 grid((g.n0 + 15) / 16, g.n2);
  const size_t sm = fx_y_smem<N>();
  if (inverse)
    k_fx_y<N, 1><<<grid, 16 * FxFast<N>::P, sm, s>>>(g, tb, st, t, check);
  else
    k_fx_y<N, 0><<<grid, 16 * FxFast<N>::P, sm, s>>>(g, tb, st, t, check);
  return cudaGetLastError();
}

template <int N, int NT>
cudaError_t q_fx_x_nt(const Geometry& g, const DctTables<double>& tb, const QueueLaunch& ql,
                      int par, int inverse) {
  constexpr int L = FxX<N, NT>::L;
  const long long nrows = (long long)g.n1 * g.n2;
  const unsigned int nb = (unsigned int)((nrows + L - 1) / L);
  const size_t sm = fx_x_smem<N, NT>();
  const long long items = (long long)nb * ql.nsolves;
  if (inverse) {
    const unsigned int grid = persistent_grid(kq_fx_inv_x<N, NT>, NT, sm, items);
    kq_fx_inv_x<N, NT><<<grid, NT, sm, ql.s>>>(ql.q, ql.slot, ql.bs, g, tb, nb);
  } else {
    const unsigned int grid = persistent_grid(kq_fx_fwd_x<N, NT>, NT, sm, items);
    kq_fx_fwd_x<N, NT><<<grid, NT, sm, ql.s>>>(ql.q, ql.slot, ql.bs, g, tb, nb, par);
  }
  return cudaGetLastError();
}
template <int N>
cudaError_t q_fx_x_n(const Geometry& g, const DctTables<double>& tb, const QueueLaunch& ql,
                     int par, int inverse, int nt) {
  if (nt == 128 || !fx_x_fits<N, 256>()) return q_fx_x_nt<N, 128>(g, tb, ql, par, inverse);
  return q_fx_x_nt<N, 256>(g, tb, ql, par, inverse);
}
template <int N>
cudaError_t q_fx_y_n(const Geometry& g, const DctTables<double>& tb, const QueueLaunch& ql,
                     int inverse) {
  constexpr int NTY = 16 * FxFast<N>::P;
  const unsigned int nbx = (unsigned int)((g.n0 + 15) / 16);
  const size_t sm = fx_y_smem<N>();
  const long long items = (long long)nbx * g.n2 * ql.nsolves;
  if (inverse) {
    const unsigned int grid = persistent_grid(kq_fx_y<N, 1>, NTY, sm, items);
    kq_fx_y<N, 1><<<grid, NTY, sm, ql.s>>>(ql.q, ql.slot, ql.bs, g, tb, nbx);
  } else {
    const unsigned int grid = persistent_grid(kq_fx_y<N, 0>, NTY, sm, items);
    kq_fx_y<N, 0><<<grid, NTY, sm, ql.s>>>(ql.q, ql.slot, ql.bs, g, tb, nbx);
  }
  return cudaGetLastError();
}

template <int N, int NT>
cudaError_t fx_attrs_nt() {
  cudaError_t e = cudaSuccess;
  if (!fx_x_fits<N, NT>()) return e;  // never launched
  const int sx = (int)fx_x_smem<N, NT>();
#define SETF(fn, b) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  SETF((k_fx_fwd_x<N, 0, NT>), sx);
  SETF((k_fx_fwd_x<N, 1, NT>), sx);
  SETF((k_fx_fwd_x<N, 2, NT>), sx);
  SETF((k_fx_inv_x<N, 0, NT>), sx);
  SETF((k_fx_inv_x<N, 2, NT>), sx);
  SETF((kq_fx_fwd_x<N, NT>), sx);
  SETF((kq_fx_inv_x<N, NT>), sx);
#undef SETF
  return e;
}
template <int N>
cudaError_t fx_attrs_n() {
  cudaError_t e = fx_attrs_nt<N, 256>();
  if (e == cudaSuccess) e = fx_attrs_nt<N, 128>();
  const int sy = (int)fx_y_smem<N>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fx_y<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fx_y<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kq_fx_y<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kq_fx_y<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
  return e;
}

template <int N>
cudaError_t fx_y3_n(const Geometry& g, const DctTables<double>& tb, const PcgState* st, double* t,
                    int inverse, int check, cudaStream_t s) {
  using Y = FxY3<N>;
  dim3 grid((g.n0 + Y::C - 1) / Y::C, g.n2);
  const size_t sm = fx_y3_smem<N>();
  if (inverse)
    k_fx_y3<N, 1><<<grid, Y::NT, sm, s>>>(g, tb, st, t, check);
  else
    k_fx_y3<N, 0><<<grid, Y::NT, sm, s>>>(g, tb, st, t, check);
  return cudaGetLastError();
}
template <int N>
cudaError_t fx_y3_attrs_n() {
  const int sy = (int)fx_y3_smem<N>();
  cudaError_t e =
      cudaFuncSetAttribute(k_fx_y3<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fx_y3<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
  return e;
}

// The lengths with block-floating-point transforms, and the per-length
// launchers each instantiates (PREFIX as for ETC_FAST_LAUNCHERS).
#define ETC_FX_SIZES(X) X(32) X(64) X(96) X(128) X(160) X(192) X(256) X(384) X(512) X(1024)
#define ETC_FX_LAUNCHERS(PREFIX, N)                                                            \
  PREFIX cudaError_t fx_fwd_x_n<N>(const Geometry&, const DctTables<double>&, PcgState*,       \
                                   double*, const double*, const double*, double*,             \
                                   const double*, double*, double*, int, double, int,          \
                                   cudaStream_t, int);                                          \
  PREFIX cudaError_t fx_inv_x_n<N>(const Geometry&, const DctTables<double>&, PcgState*,       \
                                   const double*, double*, const double*, double, int, int,    \
                                   cudaStream_t, int);                                          \
  PREFIX cudaError_t fx_y_n<N>(const Geometry&, const DctTables<double>&, const PcgState*,     \
                               double*, int, int, cudaStream_t);                                \
  PREFIX cudaError_t q_fx_x_n<N>(const Geometry&, const DctTables<double>&, const QueueLaunch&, \
                                 int, int, int);                                                \
  PREFIX cudaError_t q_fx_y_n<N>(const Geometry&, const DctTables<double>&, const QueueLaunch&, \
                                 int);                                                          \
  PREFIX cudaError_t fx_attrs_n<N>();
#define ETC_FX_EXTERN(N) ETC_FX_LAUNCHERS(extern template, N)
#define ETC_FX_INSTANTIATE(N) ETC_FX_LAUNCHERS(template, N)
// The lengths with three-stage axis-1 kernels and their launchers.
#define ETC_FX_Y3_SIZES(X) X(256) X(512) X(1024)
#define ETC_FX_Y3_LAUNCHERS(PREFIX, N)                                                          \
  PREFIX cudaError_t fx_y3_n<N>(const Geometry&, const DctTables<double>&, const PcgState*,    \
                                double*, int, int, cudaStream_t);                               \
  PREFIX cudaError_t fx_y3_attrs_n<N>();
#define ETC_FX_Y3_EXTERN(N) ETC_FX_Y3_LAUNCHERS(extern template, N)
#define ETC_FX_Y3_INSTANTIATE(N) ETC_FX_Y3_LAUNCHERS(template, N)

}  // namespace etc
