// Block-floating-point arithmetic for the cosine transforms of the FP64 path.
//
// B300 executes FP64 at 2 results per clock per SM; 32-bit integer additions,
// logic, shifts and multiply-adds issue at 64 per clock per SM.  The
// transforms of Algorithm 3 (Sec. 3.2) are sums of products by fixed
// constants, so they run here in 64-bit two's complement fixed point with one
// exponent per line (one transform):
//   * a line's values v become X = v 2^S with S chosen from the largest
//     exponent of the line, so that X keeps B = 51..53 bits of the largest
//     element (53 up to n = 256, 52 at n = 512, 51 at n = 1024: about the
//     rounding FP64's own first butterfly applies) and no intermediate value
//     of the transform can reach 2^62;
//   * additions and subtractions are exact;
//   * a product by a constant c in [-1, 1], held as C = c 2^62 rounded, keeps
//     the top bits of the exact 128-bit product X C, rounded: error about half
//     a unit, i.e. 2^-62 of the largest intermediate value, where FP64 rounds
//     every operation at 2^-53 of its result.
// For random lines the transform error is that of an FP64 transform
// (measured at n = 512 against exact sums, 2-D: 1.05e-15 of the largest output
// forward and 1.45e-15 backward, where FP64 transforms give 0.97e-15 and
// 1.27e-15), while the FP64 pipe only carries the PCG vector updates around
// it.  Being relative to a line's largest value, it can trail FP64's for lines
// of very uneven values: a spectrum of one dominant coefficient over rounding
// noise comes back with up to n units of 2^-(B-1) of its output (3.4e-14 at
// n = 512, against 1e-16).  Values below 2^-1022 come out as zero, values
// above the binary64 range as infinities; a line holding an infinity or NaN
// comes out as NaN.
#pragma once

#include "dct_device.cuh"

namespace etc {
namespace fxp {

typedef long long i64;
typedef unsigned long long u64;

struct cx {
  i64 x, y;
};
__device__ __forceinline__ cx mk(i64 a, i64 b) {
  cx z;
  z.x = a;
  z.y = b;
  return z;
}
__device__ __forceinline__ cx add(cx a, cx b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cx sub(cx a, cx b) { return mk(a.x - b.x, a.y - b.y); }
// multiply by SIGN * i
template <int SIGN>
__device__ __forceinline__ cx rot(cx a) {
  return SIGN < 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);
}

// A constant c in [-1, 1] as C = c 2^62 (|C| <= 2^62 - 1), split as
// C = h 2^31 + l with 0 <= l < 2^31.
struct Kc {
  int h, l;
};
constexpr i64 kQ62Max = 4611686018427387903LL;  // 2^62 - 1
__host__ __device__ constexpr Kc kc_split(i64 c) {
  return Kc{(int)(c >> 31), (int)(c & 0x7fffffffLL)};
}
// c 2^62 is an integer in binary64 for |c| >= 2^-10 (53-bit significand);
// below that the conversion truncates by less than one unit.
__host__ __device__ constexpr i64 q62(double c) {
  const double v = c * 4611686018427387904.0;
  return v >= 4611686018427387903.0 ? kQ62Max
         : v <= -4611686018427387903.0 ? -kQ62Max
                                       : (i64)v;
}
__host__ __device__ constexpr Kc kc(double c) { return kc_split(q62(c)); }

// A multiplicand X (|X| < 2^62) split as X = h 2^31 + l, 0 <= l < 2^31, and
// l2 = 2 l (for the high word of l times a constant's low part).
struct Sp {
  int h, l;
  unsigned int l2;
};
__device__ __forceinline__ Sp split(i64 X) {
  const unsigned int lo = (unsigned int)(u64)X, hi = (unsigned int)((u64)X >> 32);
  Sp s;
  s.h = (int)__funnelshift_r(lo, hi, 31);
  s.l = (int)(lo & 0x7fffffffu);
  s.l2 = lo << 1;
  return s;
}
// X C / 2^62 rounded to nearest:
//   X C / 2^62 = h_x h_c + (h_x l_c + l_x h_c + l_x l_c / 2^31) / 2^31,
// with l_x l_c / 2^31 rounded down and the outer division rounded half up:
// within 1/2 + 2^-31 of the exact value.  Rounding (not truncating) matters:
// truncation errors all have one sign, and the DFTs add them up coherently in
// their zero-frequency outputs (m/2 units over a length-m transform).
__device__ __forceinline__ i64 mulk(const Sp& x, Kc k) {
  const i64 mid = (i64)x.h * k.l + (i64)x.l * k.h +
                  (i64)(__umulhi(x.l2, (unsigned int)k.l) + 0x40000000u);
  return (i64)x.h * k.h + (mid >> 31);
}
__device__ __forceinline__ i64 mulk(i64 X, Kc k) { return mulk(split(X), k); }

// a e^{i phi} and a e^{-i phi}, (c, s) = (cos phi, sin phi)
__device__ __forceinline__ cx crot(cx a, Kc c, Kc s) {
  const Sp x = split(a.x), y = split(a.y);
  return mk(mulk(x, c) - mulk(y, s), mulk(x, s) + mulk(y, c));
}
__device__ __forceinline__ cx crotc(cx a, Kc c, Kc s) {
  const Sp x = split(a.x), y = split(a.y);
  return mk(mulk(x, c) + mulk(y, s), mulk(y, c) - mulk(x, s));
}
// a e^{SIGN i phi}
template <int SIGN>
__device__ __forceinline__ cx crot_s(cx a, Kc c, Kc s) {
  return SIGN < 0 ? crotc(a, c, s) : crot(a, c, s);
}
// a e^{SIGN i pi/4} and a e^{SIGN 3 i pi/4}: two products each
template <int SIGN>
__device__ __forceinline__ cx rot45(cx a) {
  constexpr Kc kH = kc(0.70710678118654752440);  // 1/sqrt(2)
  const i64 p = a.x + a.y, d = a.y - a.x;
  return SIGN < 0 ? mk(mulk(p, kH), mulk(d, kH)) : mk(-mulk(d, kH), mulk(p, kH));
}
template <int SIGN>
__device__ __forceinline__ cx rot135(cx a) {
  constexpr Kc kH = kc(0.70710678118654752440);
  const i64 p = a.x + a.y, d = a.y - a.x;
  return SIGN < 0 ? mk(mulk(d, kH), -mulk(p, kH)) : mk(-mulk(p, kH), -mulk(d, kH));
}

// In-register DFT of length RADIX with kernel exp(SIGN 2 pi i r q / RADIX),
// output in natural order (the same factorisations as the floating-point
// butterflies of the register-resident kernels).
template <int RADIX, int SIGN> struct Fb;

template <int SIGN> struct Fb<4, SIGN> {
  static __device__ __forceinline__ void run(cx* v) {
    const cx t0 = add(v[0], v[2]), t1 = sub(v[0], v[2]);
    const cx t2 = add(v[1], v[3]), t3 = rot<SIGN>(sub(v[1], v[3]));
    v[0] = add(t0, t2);
    v[2] = sub(t0, t2);
    v[1] = add(t1, t3);
    v[3] = sub(t1, t3);
  }
};

template <int SIGN> struct Fb<8, SIGN> {
  static __device__ __forceinline__ void run(cx* v) {
    cx e[4] = {v[0], v[2], v[4], v[6]};
    cx o[4] = {v[1], v[3], v[5], v[7]};
    Fb<4, SIGN>::run(e);
    Fb<4, SIGN>::run(o);
    o[1] = rot45<SIGN>(o[1]);
    o[2] = rot<SIGN>(o[2]);
    o[3] = rot135<SIGN>(o[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] = add(e[q], o[q]);
      v[q + 4] = sub(e[q], o[q]);
    }
  }
};

// 16 = 4 x 4: DFT-4 over s2 of x[s1 + 4 s2], twiddle exp(SIGN 2 pi i s1 k1 / 16),
// DFT-4 over s1.
template <int SIGN> struct Fb<16, SIGN> {
  static __device__ __forceinline__ void run(cx* v) {
    constexpr Kc c8 = kc(0.92387953251128675613), s8 = kc(0.38268343236508977173);
    constexpr Kc mc8 = kc(-0.92387953251128675613), ms8 = kc(-0.38268343236508977173);
    cx a[4][4];
#pragma unroll
    for (int s1 = 0; s1 < 4; ++s1) {
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2) a[s1][s2] = v[s1 + 4 * s2];
      Fb<4, SIGN>::run(a[s1]);
    }
    a[1][1] = crot_s<SIGN>(a[1][1], c8, s8);    // e = 1
    a[1][2] = rot45<SIGN>(a[1][2]);             // e = 2
    a[1][3] = crot_s<SIGN>(a[1][3], s8, c8);    // e = 3
    a[2][1] = rot45<SIGN>(a[2][1]);             // e = 2
    a[2][2] = rot<SIGN>(a[2][2]);               // e = 4
    a[2][3] = rot135<SIGN>(a[2][3]);            // e = 6
    a[3][1] = crot_s<SIGN>(a[3][1], s8, c8);    // e = 3
    a[3][2] = rot135<SIGN>(a[3][2]);            // e = 6
    a[3][3] = crot_s<SIGN>(a[3][3], mc8, ms8);  // e = 9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      cx b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      Fb<4, SIGN>::run(b);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
    }
  }
};

// t / 2 rounded to nearest, ties to even (no bias: a one-sided rounding of
// the exact halves would add up coherently in the DFTs' zero-frequency outputs)
__device__ __forceinline__ i64 half_even(i64 t) { return (t >> 1) + (t & (t >> 1) & 1); }

template <int SIGN> struct Fb<2, SIGN> {
  static __device__ __forceinline__ void run(cx* v) {
    const cx a = v[0];
    v[0] = add(a, v[1]);
    v[1] = sub(a, v[1]);
  }
};

template <int SIGN> struct Fb<3, SIGN> {
  static __device__ __forceinline__ void run(cx* v) {
    constexpr Kc s3 = kc(0.86602540378443864676);  // sqrt(3)/2
    const cx t1 = add(v[1], v[2]);
    const cx t2 = mk(v[0].x - half_even(t1.x), v[0].y - half_even(t1.y));
    const cx d = sub(v[1], v[2]);
    const cx t3 = rot<SIGN>(mk(mulk(d.x, s3), mulk(d.y, s3)));  // SIGN i sqrt(3)/2 (v1 - v2)
    v[0] = add(v[0], t1);
    v[1] = add(t2, t3);
    v[2] = sub(t2, t3);
  }
};

template <int SIGN> struct Fb<5, SIGN> {
  static __device__ __forceinline__ void run(cx* v) {
    constexpr Kc c1 = kc(0.30901699437494742410), c2 = kc(-0.80901699437494742410);
    constexpr Kc n1 = kc(0.95105651629515357212), n2 = kc(0.58778525229247312917);
    constexpr Kc mn1 = kc(-0.95105651629515357212);
    const cx b1 = add(v[1], v[4]), b2 = add(v[2], v[3]);
    const cx d1 = sub(v[1], v[4]), d2 = sub(v[2], v[3]);
    const cx a = v[0];
    const Sp b1x = split(b1.x), b1y = split(b1.y), b2x = split(b2.x), b2y = split(b2.y);
    const Sp d1x = split(d1.x), d1y = split(d1.y), d2x = split(d2.x), d2y = split(d2.y);
    const cx p1 = mk(a.x + mulk(b1x, c1) + mulk(b2x, c2), a.y + mulk(b1y, c1) + mulk(b2y, c2));
    const cx p2 = mk(a.x + mulk(b1x, c2) + mulk(b2x, c1), a.y + mulk(b1y, c2) + mulk(b2y, c1));
    const cx q1 = rot<SIGN>(mk(mulk(d1x, n1) + mulk(d2x, n2), mulk(d1y, n1) + mulk(d2y, n2)));
    const cx q2 = rot<SIGN>(mk(mulk(d1x, n2) + mulk(d2x, mn1), mulk(d1y, n2) + mulk(d2y, mn1)));
    v[0] = add(a, add(b1, b2));
    v[1] = add(p1, q1);
    v[4] = sub(p1, q1);
    v[2] = add(p2, q2);
    v[3] = sub(p2, q2);
  }
};

// Length A*B by Cooley-Tukey (as the floating-point composite butterflies):
// DFT-B over s2 of x[s1 + A s2] for each s1, twiddle exp(SIGN 2 pi i s1 k1 /
// (A B)) from compile-time constants, DFT-A over s1 for each k1; output
// X[k1 + B k2] in natural order.
template <int A, int B, int SIGN> struct FbCT {
  static __device__ __forceinline__ void run(cx* v) {
    cx y[A][B];
#pragma unroll
    for (int s1 = 0; s1 < A; ++s1) {
#pragma unroll
      for (int s2 = 0; s2 < B; ++s2) y[s1][s2] = v[s1 + A * s2];
      Fb<B, SIGN>::run(y[s1]);
    }
    SFor<1, A>::run([&](auto i1) {
      constexpr int s1 = decltype(i1)::value;
      SFor<1, B>::run([&](auto j1) {
        constexpr int k1 = decltype(j1)::value;
        constexpr CosSin w = cis2pi(s1 * k1, A * B);
        constexpr Kc wc = kc(w.c), ws = kc(w.s);
        y[s1][k1] = crot_s<SIGN>(y[s1][k1], wc, ws);
      });
    });
#pragma unroll
    for (int k1 = 0; k1 < B; ++k1) {
      cx z[A];
#pragma unroll
      for (int s1 = 0; s1 < A; ++s1) z[s1] = y[s1][k1];
      Fb<A, SIGN>::run(z);
#pragma unroll
      for (int k2 = 0; k2 < A; ++k2) v[k1 + B * k2] = z[k2];
    }
  }
};
template <int SIGN> struct Fb<10, SIGN> : FbCT<2, 5, SIGN> {};
template <int SIGN> struct Fb<12, SIGN> : FbCT<4, 3, SIGN> {};
template <int SIGN> struct Fb<20, SIGN> : FbCT<4, 5, SIGN> {};
template <int SIGN> struct Fb<24, SIGN> : FbCT<8, 3, SIGN> {};
template <int SIGN> struct Fb<32, SIGN> : FbCT<8, 4, SIGN> {};

// ---------------------------------------------------------------- conversions
// Biased exponent field of a binary64 value, 1 for zero and subnormals.
__device__ __forceinline__ int bexp(double v) {
  const int e = (int)(((unsigned int)__double2hiint(v) >> 20) & 0x7ffu);
  return e > 1 ? e : 1;
}
// Scale exponent of a line whose largest exponent field is emax, with B bits
// kept for its largest element: X = v 2^S, S = 1022 - emax + B.  The binary64
// value +-mant 2^(e - 1075) becomes mant 2^(e - emax - (53 - B)), rounded to
// nearest (ties up), with integer operations only.  LOW false drops the cases
// of zeros and subnormals, for lines with emax >= 10 + B: the shift of such a
// value is then at least 63 and it comes out 0 either way.
template <int B, bool LOW = true>
__device__ __forceinline__ i64 to_fx(double v, int emax) {
  static_assert(B <= 53, "at most the binary64 significand");
  const unsigned int hi = (unsigned int)__double2hiint(v), lo = (unsigned int)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7ffu);
  const u64 mant = ((u64)((hi & 0xfffffu) | ((!LOW || e) ? 0x100000u : 0u)) << 32) | lo;
  int sh = emax - (LOW ? (e > 1 ? e : 1) : e) + (53 - B);
  sh = sh < 63 ? sh : 63;
  const i64 X = (i64)((((mant << 1) >> sh) + 1ull) >> 1);
  return (int)hi < 0 ? -X : X;
}
// Y 2^e2 rounded to the nearest binary64 (ties to even), |Y| < 2^63; 0 below
// the normal range, an infinity above it.  The exponent field comes out at
// most 1086 + e2 (leading one at bit 62, plus a rounding carry): SAT false
// drops the test for the top of the range, for callers with 1086 + e2 < 2047.
template <bool SAT = true>
__device__ __forceinline__ double from_fx(i64 Y, int e2) {
  const u64 sgn = (u64)(Y >> 63);
  u64 a = ((u64)Y ^ sgn) - sgn;
  const int lz = __clzll((i64)a);  // 64 for a = 0
  a <<= (lz - 1) & 63;             // leading one at bit 62
  const u64 mant = (a + 0x1ffull + ((a >> 10) & 1ull)) >> 10;  // 2^52 .. 2^53
  const int be = 1086 - lz + e2;  // biased exponent of the leading one
  // mant carries the leading one: added onto the field be - 1 it gives be (be + 1
  // when the rounding reached 2^53)
  const u64 bits = (SAT && be >= 2047) ? 0x7ff0000000000000ull + (sgn << 63)
                                       : ((u64)(be - 1) << 52) + mant + (sgn << 63);
  return (lz == 64 || be <= 0) ? 0.0 : __longlong_as_double((i64)bits);
}
__device__ __forceinline__ double nan_f64() { return __longlong_as_double(0x7ff8000000000000LL); }

// The same two conversions by the hardware's binary64 <-> 64-bit integer
// conversions (round to nearest even), with the power-of-two scaling done on
// the exponent field: one FP64-pipe instruction and a few integer ones each,
// where the integer forms above take 15 to 25.  The transforms leave the FP64
// pipe otherwise idle (axis 1) or lightly used (axis 0).
template <int B>
__device__ __forceinline__ i64 to_fx_hw(double v, int emax) {
  const int hi = __double2hiint(v), lo = __double2loint(v);
  const int e = (hi >> 20) & 0x7ff;
  const int sc = 1022 - emax + B;  // S
  // zero, subnormal, or below half a unit of the line: 0
  if (e == 0 || e + sc <= 0) return 0;
  return __double2ll_rn(__hiloint2double(hi + (sc << 20), lo));
}
// (SAT false: without the test for the top of the range, for 1086 + e2 < 2047)
template <bool SAT = true>
__device__ __forceinline__ double from_fx_hw(i64 Y, int e2) {
  const double d = __ll2double_rn(Y);
  const int hi = __double2hiint(d), lo = __double2loint(d);
  const int e = (hi >> 20) & 0x7ff;
  if (e == 0 || e + e2 <= 0) return 0.0;
  if (SAT && e + e2 >= 2047) return __hiloint2double((hi & (int)0x80000000) | 0x7ff00000, 0);
  return __hiloint2double(hi + (e2 << 20), lo);
}

// Bits kept for the largest element of a line (at most binary64's 53), so that
// no intermediate value reaches 2^62:
//   forward, FFT of length m: |Z_k| <= 2 m max|u| / sqrt(2) per component pair,
//     the untangling sums a1 = Re Z_k + Re Z_{m-k} <= 2 m sqrt(2) max|u|;
//   backward: |V_k| <= sqrt(2) max|X| and |p|^2 + |o|^2 = 2 (|V_j|^2 +
//     |V_{m-j}|^2), so the packed FFT input |a_j| <= |p| + |o| <= 4 max|X| and
//     its FFT output <= 4 m max|X| (halved before a product by an output
//     scale).
constexpr int clog2c(int v) { return v <= 1 ? 0 : 1 + clog2c((v + 1) / 2); }  // ceil(log2 v)
template <int M> struct FxBits {
  static constexpr int F = (61 - clog2c(2 * M)) < 53 ? (61 - clog2c(2 * M)) : 53;  // 61.5 - log2(2m)
  static constexpr int I = (60 - clog2c(M)) < 53 ? (60 - clog2c(M)) : 53;          // 62 - log2(4m)
  // 1 / (2m) = f 2^E with f in [1/2, 1): the backward scale the pre-twiddle omits
  static constexpr bool POW2 = (M & (M - 1)) == 0;
  static constexpr int E = 1 - clog2c(2 * M);
  static constexpr double f() { return (double)(1LL << clog2c(2 * M)) / (2.0 * M) / 2.0; }
};

// ---------------------------------------------------------------- tables
// Constants of the register-resident transforms as (h, l) pairs, four per
// int4 (fxq in DctTables):
//   [0, m)              four-step twiddles exp(-2 pi i tau k1 / m), [tau][k1]: (cos, sin)
//   m + 2k, m + 2k + 1  untangling, t = pi k / (2n): (cos t / 2, sin t / 2), (cos 5t / 2, sin 5t / 2)
//   3m + 2 + 2k, +1     backward pre-twiddle: (cos t, sin t), (cos 4t, sin 4t)
// for k = 0..m.  The backward pre-twiddle omits the floating-point tables'
// factor 1/(2m), which the output conversion applies (a power of two in the
// exponent, otherwise one more product by its significand).
struct Kc2 {
  Kc a, b;
};
__device__ __forceinline__ Kc2 ld_k2(const int4* p) {
  const int4 v = __ldg(p);
  Kc2 k;
  k.a = Kc{v.x, v.y};
  k.b = Kc{v.z, v.w};
  return k;
}
__host__ __device__ constexpr int fx_off_post(int m) { return m; }
__host__ __device__ constexpr int fx_off_pre(int m) { return m + 2 * (m + 1); }
// Three-stage axis-1 kernels (m = 8 * 8 * P2, m = 128 .. 512): their first-stage
// twiddles exp(-2 pi i tau k1 / m), [tau][k1] for tau < m / 8, k1 < 8, then the
// second-stage twiddles exp(-2 pi i tb ka / (m / 8)), [tb][ka] for tb < m / 64.
__host__ __device__ constexpr bool fx_has_y3(int m) { return m == 128 || m == 256 || m == 512; }
__host__ __device__ constexpr int fx_off_y3(int m) { return m + 4 * (m + 1); }
__host__ __device__ constexpr int fx_table_int4(int m) {
  return m + 4 * (m + 1) + (fx_has_y3(m) ? m + m / 8 : 0);
}

// ---------------------------------------------------------------- transform steps
// Forward untangling of the pair (k, m - k): X_k and X_{n-k} (X_m for k = 0)
// from Z_k and Z_{m-k}, the same combination as the floating-point kernels.
__device__ __forceinline__ void untangle(cx zk, cx zm, const int4* __restrict__ post, int k,
                                         int m, i64& xa, i64& xb) {
  const Sp a = split(zk.x + zm.x), b = split(zk.y - zm.y);
  const Sp c = split(zk.y + zm.y), d = split(zk.x - zm.x);
  const Kc2 f01 = ld_k2(post + 2 * k), f23 = ld_k2(post + 2 * k + 1);
  xa = mulk(a, f01.a) + mulk(b, f01.b) + mulk(c, f23.a) - mulk(d, f23.b);
  if (k != 0) {
    xb = mulk(a, f01.b) - mulk(b, f01.a) + mulk(d, f23.a) + mulk(c, f23.b);
  } else {
    const Kc2 g01 = ld_k2(post + 2 * m), g23 = ld_k2(post + 2 * m + 1);
    xb = mulk(a, g01.a) + mulk(c, g23.a);
  }
}
// Backward pre-twiddle, first half: V_k = e^{i t_k} (X_k - i X_{n-k}) for
// k = 0..m (X_n = 0; k = m pairs X_m with itself).
__device__ __forceinline__ cx inv_v(const int4* __restrict__ pre, int k, i64 xk, i64 xn) {
  const Kc2 f = ld_k2(pre + 2 * k);
  const Sp a = split(xk), b = split(xn);
  return mk(mulk(a, f.a) + mulk(b, f.b), mulk(a, f.b) - mulk(b, f.a));
}
// Second half: FFT input a_j = P + i O with P = V_j + conj(V_{m-j}) and
// O = (V_j - conj(V_{m-j})) e^{4 i t_j}.
__device__ __forceinline__ cx inv_a(const int4* __restrict__ pre, int j, cx vj, cx vm) {
  const Kc2 f = ld_k2(pre + 2 * j + 1);
  const i64 pr = vj.x + vm.x, pi = vj.y - vm.y;
  const Sp qr = split(vj.x - vm.x), qi = split(vj.y + vm.y);
  const i64 orr = mulk(qr, f.a) - mulk(qi, f.b), oi = mulk(qr, f.b) + mulk(qi, f.a);
  return mk(pr - oi, pi + orr);
}

}  // namespace fxp
}  // namespace etc
