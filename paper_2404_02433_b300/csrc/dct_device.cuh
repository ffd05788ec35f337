// Batched 1-D cosine transforms of lines held in shared memory.
//
// Forward: Eq. (forward DCT), X_k = sum_{i<n} u_i cos(pi (2i+1) k / 2n).
// Backward: Eq. (backward DCT), u_i = (2/n) sum_{k<n} alpha_k X_k cos(...),
// alpha_0 = 1/2 -- the exact inverse of the forward transform.
//
// Even n uses the even/odd reordering of the input (v_j = u_{2j},
// v_{n-1-j} = u_{2j+1}), packs v into m = n/2 complex values, runs a complex
// Stockham FFT of length m and untangles the real transform with twiddles (the
// classical route from a real DCT-II to a half-length complex FFT).  Odd n, or
// m with a prime factor above 5, uses the direct O(n^2) sum with an exactly
// reduced cosine table.  R is the arithmetic type (double or float).
#pragma once

#include <type_traits>

#include "etc_internal.cuh"

namespace etc {

template <typename R> struct C2T;
template <> struct C2T<double> { using T = double2; };
template <> struct C2T<float> { using T = float2; };
template <typename R> using c2 = typename C2T<R>::T;

template <typename R>
__device__ __forceinline__ c2<R> mk2(R a, R b) { c2<R> z; z.x = a; z.y = b; return z; }
template <typename R>
__device__ __forceinline__ c2<R> add2(c2<R> a, c2<R> b) { return mk2<R>(a.x + b.x, a.y + b.y); }
template <typename R>
__device__ __forceinline__ c2<R> sub2(c2<R> a, c2<R> b) { return mk2<R>(a.x - b.x, a.y - b.y); }
// a * w
template <typename R>
__device__ __forceinline__ c2<R> cmul(c2<R> a, c2<R> w) {
  return mk2<R>(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
// multiply by SIGN * i (SIGN = -1: the forward kernel e^{-i pi/2})
template <typename R, int SIGN>
__device__ __forceinline__ c2<R> rot(c2<R> a) {
  return SIGN < 0 ? mk2<R>(a.y, -a.x) : mk2<R>(-a.y, a.x);
}

// Mathematical constants (decimal expansions).
template <typename R> struct K {
  static constexpr R s2 = (R)0.70710678118654752440;   // 1/sqrt(2)
  static constexpr R s3 = (R)0.86602540378443864676;   // sqrt(3)/2
  static constexpr R c1 = (R)0.30901699437494742410;   // cos(2 pi/5)
  static constexpr R c2 = (R)-0.80901699437494742410;  // cos(4 pi/5)
  static constexpr R n1 = (R)0.95105651629515357212;   // sin(2 pi/5)
  static constexpr R n2 = (R)0.58778525229247312917;   // sin(4 pi/5)
};

// In-register DFT of length RADIX with kernel exp(SIGN 2 pi i r q / RADIX).
template <typename R, int RADIX, int SIGN> struct Bfly;

template <typename R, int SIGN> struct Bfly<R, 2, SIGN> {
  static __device__ __forceinline__ void run(c2<R>* v) {
    c2<R> a = v[0];
    v[0] = add2<R>(a, v[1]);
    v[1] = sub2<R>(a, v[1]);
  }
};

template <typename R, int SIGN> struct Bfly<R, 4, SIGN> {
  static __device__ __forceinline__ void run(c2<R>* v) {
    c2<R> t0 = add2<R>(v[0], v[2]), t1 = sub2<R>(v[0], v[2]);
    c2<R> t2 = add2<R>(v[1], v[3]), t3 = rot<R, SIGN>(sub2<R>(v[1], v[3]));
    v[0] = add2<R>(t0, t2);
    v[2] = sub2<R>(t0, t2);
    v[1] = add2<R>(t1, t3);
    v[3] = sub2<R>(t1, t3);
  }
};

template <typename R, int SIGN> struct Bfly<R, 8, SIGN> {
  static __device__ __forceinline__ void run(c2<R>* v) {
    c2<R> e[4] = {v[0], v[2], v[4], v[6]};
    c2<R> o[4] = {v[1], v[3], v[5], v[7]};
    Bfly<R, 4, SIGN>::run(e);
    Bfly<R, 4, SIGN>::run(o);
    // o[q] *= exp(SIGN 2 pi i q / 8)
    const R s = K<R>::s2;
    if (SIGN < 0) {
      o[1] = mk2<R>((o[1].x + o[1].y) * s, (o[1].y - o[1].x) * s);
      o[3] = mk2<R>((o[3].y - o[3].x) * s, -(o[3].x + o[3].y) * s);
    } else {
      o[1] = mk2<R>((o[1].x - o[1].y) * s, (o[1].x + o[1].y) * s);
      o[3] = mk2<R>(-(o[3].x + o[3].y) * s, (o[3].x - o[3].y) * s);
    }
    o[2] = rot<R, SIGN>(o[2]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] = add2<R>(e[q], o[q]);
      v[q + 4] = sub2<R>(e[q], o[q]);
    }
  }
};

// x * exp(SIGN i phi) for a constant angle given by its cosine and sine
template <typename R, int SIGN>
__device__ __forceinline__ c2<R> crot(c2<R> x, R c, R s) {
  const R ss = SIGN < 0 ? -s : s;
  return mk2<R>(fma(x.x, c, -x.y * ss), fma(x.x, ss, x.y * c));
}

// Length 16 as 4 x 4: DFT-4 over s2 of x[s1 + 4 s2], twiddle exp(SIGN 2 pi i s1 k1 / 16),
// DFT-4 over s1; output in natural order.
template <typename R, int SIGN> struct Bfly<R, 16, SIGN> {
  static __device__ __forceinline__ void run(c2<R>* v) {
    constexpr R c8 = (R)0.92387953251128675613;  // cos(pi/8)
    constexpr R s8 = (R)0.38268343236508977173;  // sin(pi/8)
    constexpr R h = K<R>::s2;
    c2<R> a[4][4];
#pragma unroll
    for (int s1 = 0; s1 < 4; ++s1) {
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2) a[s1][s2] = v[s1 + 4 * s2];
      Bfly<R, 4, SIGN>::run(a[s1]);
    }
    a[1][1] = crot<R, SIGN>(a[1][1], c8, s8);   // e = 1
    a[1][2] = crot<R, SIGN>(a[1][2], h, h);     // e = 2
    a[1][3] = crot<R, SIGN>(a[1][3], s8, c8);   // e = 3
    a[2][1] = crot<R, SIGN>(a[2][1], h, h);     // e = 2
    a[2][2] = rot<R, SIGN>(a[2][2]);            // e = 4
    a[2][3] = crot<R, SIGN>(a[2][3], -h, h);    // e = 6
    a[3][1] = crot<R, SIGN>(a[3][1], s8, c8);   // e = 3
    a[3][2] = crot<R, SIGN>(a[3][2], -h, h);    // e = 6
    a[3][3] = crot<R, SIGN>(a[3][3], -c8, -s8); // e = 9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      c2<R> b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      Bfly<R, 4, SIGN>::run(b);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
    }
  }
};

// exp(2 pi i m / q) at compile time, for the twiddles of the composite
// lengths below.  The angle 2 pi (m mod q) / q is written exactly as
// k pi/2 +- psi with psi in [0, pi/4] (integer octant arithmetic), and cos psi,
// sin psi are summed from their Taylor series (14 terms; the first omitted
// term is below 1e-30).
struct CosSin {
  double c, s;
};
constexpr double kPiD = 3.14159265358979323846264338327950288;
constexpr double taylor_sin(double x) {
  double t = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += t;
  }
  return sum;
}
constexpr double taylor_cos(double x) {
  double t = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += t;
  }
  return sum;
}
constexpr CosSin cis2pi(int m, int q) {
  const int r = ((m % q) + q) % q;
  const int o = (8 * r) / q, rem = 8 * r - o * q;  // angle = o pi/4 + pi rem / (4q)
  const bool even = (o % 2) == 0;
  const int k = even ? o / 2 : (o + 1) / 2;       // angle = k pi/2 + th
  const double psi = even ? kPiD * rem / (4.0 * q) : kPiD * (q - rem) / (4.0 * q);
  const double c0 = taylor_cos(psi), s0 = even ? taylor_sin(psi) : -taylor_sin(psi);
  switch (k & 3) {
    case 0: return {c0, s0};
    case 1: return {-s0, c0};
    case 2: return {-c0, -s0};
    default: return {s0, -c0};
  }
}

// compile-time loop: f(std::integral_constant<int, I>) for I in [I0, I1)
template <int I, int I1> struct SFor {
  template <class F>
  static __device__ __forceinline__ void run(F&& f) {
    f(std::integral_constant<int, I>{});
    SFor<I + 1, I1>::run(f);
  }
};
template <int I1> struct SFor<I1, I1> {
  template <class F>
  static __device__ __forceinline__ void run(F&&) {}
};

// Length A*B by Cooley-Tukey: DFT-B over s2 of x[s1 + A s2] for each s1,
// twiddle exp(SIGN 2 pi i s1 k1 / (A B)), DFT-A over s1 for each k1; output
// X[k1 + B k2] in natural order.
template <typename R, int A, int B, int SIGN> struct BflyCT {
  static __device__ __forceinline__ void run(c2<R>* v) {
    c2<R> y[A][B];
#pragma unroll
    for (int s1 = 0; s1 < A; ++s1) {
#pragma unroll
      for (int s2 = 0; s2 < B; ++s2) y[s1][s2] = v[s1 + A * s2];
      Bfly<R, B, SIGN>::run(y[s1]);
    }
    SFor<1, A>::run([&](auto i1) {
      constexpr int s1 = decltype(i1)::value;
      SFor<1, B>::run([&](auto j1) {
        constexpr int k1 = decltype(j1)::value;
        constexpr CosSin w = cis2pi(s1 * k1, A * B);
        y[s1][k1] = crot<R, SIGN>(y[s1][k1], (R)w.c, (R)w.s);
      });
    });
#pragma unroll
    for (int k1 = 0; k1 < B; ++k1) {
      c2<R> z[A];
#pragma unroll
      for (int s1 = 0; s1 < A; ++s1) z[s1] = y[s1][k1];
      Bfly<R, A, SIGN>::run(z);
#pragma unroll
      for (int k2 = 0; k2 < A; ++k2) v[k1 + B * k2] = z[k2];
    }
  }
};

template <typename R, int SIGN> struct Bfly<R, 12, SIGN> : BflyCT<R, 4, 3, SIGN> {};
template <typename R, int SIGN> struct Bfly<R, 20, SIGN> : BflyCT<R, 4, 5, SIGN> {};
template <typename R, int SIGN> struct Bfly<R, 24, SIGN> : BflyCT<R, 8, 3, SIGN> {};
template <typename R, int SIGN> struct Bfly<R, 32, SIGN> : BflyCT<R, 8, 4, SIGN> {};

template <typename R, int SIGN> struct Bfly<R, 3, SIGN> {
  static __device__ __forceinline__ void run(c2<R>* v) {
    c2<R> t1 = add2<R>(v[1], v[2]);
    c2<R> t2 = mk2<R>(fma((R)-0.5, t1.x, v[0].x), fma((R)-0.5, t1.y, v[0].y));
    c2<R> d = sub2<R>(v[1], v[2]);
    // SIGN i sqrt(3)/2 (v1 - v2)
    c2<R> t3 = rot<R, SIGN>(mk2<R>(d.x * K<R>::s3, d.y * K<R>::s3));
    v[0] = add2<R>(v[0], t1);
    v[1] = add2<R>(t2, t3);
    v[2] = sub2<R>(t2, t3);
  }
};

template <typename R, int SIGN> struct Bfly<R, 5, SIGN> {
  static __device__ __forceinline__ void run(c2<R>* v) {
    c2<R> b1 = add2<R>(v[1], v[4]), b2 = add2<R>(v[2], v[3]);
    c2<R> d1 = sub2<R>(v[1], v[4]), d2 = sub2<R>(v[2], v[3]);
    c2<R> a = v[0];
    c2<R> p1 = mk2<R>(fma(K<R>::c2, b2.x, fma(K<R>::c1, b1.x, a.x)),
                      fma(K<R>::c2, b2.y, fma(K<R>::c1, b1.y, a.y)));
    c2<R> p2 = mk2<R>(fma(K<R>::c1, b2.x, fma(K<R>::c2, b1.x, a.x)),
                      fma(K<R>::c1, b2.y, fma(K<R>::c2, b1.y, a.y)));
    c2<R> q1 = rot<R, SIGN>(mk2<R>(fma(K<R>::n1, d1.x, K<R>::n2 * d2.x),
                                   fma(K<R>::n1, d1.y, K<R>::n2 * d2.y)));
    c2<R> q2 = rot<R, SIGN>(mk2<R>(fma(K<R>::n2, d1.x, -K<R>::n1 * d2.x),
                                   fma(K<R>::n2, d1.y, -K<R>::n1 * d2.y)));
    v[0] = add2<R>(a, add2<R>(b1, b2));
    v[1] = add2<R>(p1, q1);
    v[4] = sub2<R>(p1, q1);
    v[2] = add2<R>(p2, q2);
    v[3] = sub2<R>(p2, q2);
  }
};

// Shared-memory layout of a batch of L lines.  Complex element (l, j) sits at
// l*lc + j*mc; the real view of the same bytes holds element (l, i) at
// l*lr + i*mr.  line_fast puts the line index innermost (column transforms).
struct Lay {
  int L, lc, mc, lr, mr;
  bool line_fast;
};

__host__ __device__ inline int dct_half_alloc(int n) { return (n + 1) / 2; }

__device__ __forceinline__ Lay make_lay(int L, int n, bool line_fast) {
  Lay y;
  y.L = L;
  y.line_fast = line_fast;
  const int mh = dct_half_alloc(n);
  if (line_fast) { y.lc = 1; y.mc = L; y.lr = 1; y.mr = L; }
  else { y.lc = mh; y.mc = 1; y.lr = 2 * mh; y.mr = 1; }
  return y;
}

// One Stockham pass of radix RADIX over all lines.
template <typename R, int RADIX, int SIGN>
__device__ __forceinline__ void stockham_pass(const c2<R>* __restrict__ src,
                                              c2<R>* __restrict__ dst, const Lay& y, int m,
                                              int ns, const c2<R>* __restrict__ tw) {
  const int nb = m / RADIX;
  const int total = y.L * nb;
  const int step = m / (ns * RADIX);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int l, j;
    if (y.line_fast) { l = t % y.L; j = t / y.L; }
    else { j = t % nb; l = t / nb; }
    const c2<R>* s = src + l * y.lc;
    c2<R>* d = dst + l * y.lc;
    const int k = j % ns;
    c2<R> v[RADIX];
#pragma unroll
    for (int r = 0; r < RADIX; ++r) v[r] = s[(j + r * nb) * y.mc];
    if (ns > 1) {
#pragma unroll
      for (int r = 1; r < RADIX; ++r) {
        c2<R> w = tw[r * k * step];
        if (SIGN > 0) w.y = -w.y;
        v[r] = cmul<R>(v[r], w);
      }
    }
    Bfly<R, RADIX, SIGN>::run(v);
    const int base = (j / ns) * ns * RADIX + k;
#pragma unroll
    for (int r = 0; r < RADIX; ++r) d[(base + r * ns) * y.mc] = v[r];
  }
}

// Complex FFT of length m on every line; input in a, returns the buffer that
// holds the result (a or b).  Ends with __syncthreads().
template <typename R, int SIGN>
__device__ c2<R>* fft_lines(const DctShape& s, const Lay& y, c2<R>* a, c2<R>* b,
                            const c2<R>* tw) {
  c2<R>* src = a;
  c2<R>* dst = b;
  int ns = 1;
  for (int st = 0; st < s.nst; ++st) {
    const int rad = s.radix[st];
    switch (rad) {
      case 2: stockham_pass<R, 2, SIGN>(src, dst, y, s.m, ns, tw); break;
      case 3: stockham_pass<R, 3, SIGN>(src, dst, y, s.m, ns, tw); break;
      case 4: stockham_pass<R, 4, SIGN>(src, dst, y, s.m, ns, tw); break;
      case 5: stockham_pass<R, 5, SIGN>(src, dst, y, s.m, ns, tw); break;
      default: stockham_pass<R, 8, SIGN>(src, dst, y, s.m, ns, tw); break;
    }
    __syncthreads();
    c2<R>* t = src; src = dst; dst = t;
    ns *= rad;
  }
  return src;
}

// ---------------------------------------------------------------- forward
// Place input value u_i of line l before dct2_run (FFT path: packed complex
// slot of the reordered sequence; direct path: real slot i).
template <typename R>
__device__ __forceinline__ void dct2_put(const DctShape& s, const Lay& y, c2<R>* a, int l,
                                         int i, R u) {
  R* base = reinterpret_cast<R*>(a);
  if (s.fft) {
    const int v = (i & 1) ? (s.n - 1 - (i >> 1)) : (i >> 1);
    base[2 * (l * y.lc + (v >> 1) * y.mc) + (v & 1)] = u;
  } else {
    base[l * y.lr + i * y.mr] = u;
  }
}

// Forward transform of the lines placed by dct2_put; store(l, k, X_k) receives
// every output exactly once.  a and b are the two shared buffers.
template <typename R, class Store>
__device__ void dct2_run(const DctPlan<R>& p, const Lay& y, c2<R>* a, c2<R>* b, Store store) {
  const DctShape& s = p.s;
  const int n = s.n;
  if (!s.fft) {
    const R* u = reinterpret_cast<const R*>(a);
    const int total = y.L * n;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int l, k;
      if (y.line_fast) { l = t % y.L; k = t / y.L; }
      else { k = t % n; l = t / n; }
      const R* ul = u + l * y.lr;
      const int n4 = 4 * n;
      const int stepq = (2 * k) % n4;
      int q = k % n4;
      R acc = 0;
      for (int i = 0; i < n; ++i) {
        acc = fma(ul[i * y.mr], p.t.cosq[q], acc);
        q += stepq;
        if (q >= n4) q -= n4;
      }
      store(l, k, acc);
    }
    return;
  }
  const int m = s.m;
  const c2<R>* z = fft_lines<R, -1>(s, y, a, b, reinterpret_cast<const c2<R>*>(p.t.tw));
  const int half = m / 2;
  const int total = y.L * (half + 1);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int l, k;
    if (y.line_fast) { l = t % y.L; k = t / y.L; }
    else { k = t % (half + 1); l = t / (half + 1); }
    const int km = (k == 0) ? 0 : m - k;
    const c2<R> zk = z[l * y.lc + k * y.mc];
    const c2<R> zm = z[l * y.lc + km * y.mc];
    const R a1 = zk.x + zm.x, b1 = zk.y - zm.y, c1 = zk.y + zm.y, d1 = zk.x - zm.x;
    if (k == 0) {
      const R* f = p.t.fpost;
      const R* g = p.t.fpost + 4 * m;
      store(l, 0, fma(f[0], a1, f[2] * c1));
      store(l, m, fma(g[0], a1, g[2] * c1));
    } else {
      const R* f = p.t.fpost + 4 * k;
      store(l, k, fma(f[0], a1, fma(f[1], b1, fma(f[2], c1, -f[3] * d1))));
      store(l, n - k, fma(f[1], a1, fma(-f[0], b1, fma(f[2], d1, f[3] * c1))));
      if (km != k) {
        const R* g = p.t.fpost + 4 * km;
        store(l, km, fma(g[0], a1, fma(-g[1], b1, fma(g[2], c1, g[3] * d1))));
        store(l, n - km, fma(g[1], a1, fma(g[0], b1, fma(-g[2], d1, g[3] * c1))));
      }
    }
  }
}

// ---------------------------------------------------------------- backward
// Stage input X_k of line l before dct3_run (real slot k of buffer b).
template <typename R>
__device__ __forceinline__ void dct3_put(const Lay& y, c2<R>* b, int l, int k, R xk) {
  reinterpret_cast<R*>(b)[l * y.lr + k * y.mr] = xk;
}

// Backward transform of the values staged by dct3_put; store(l, i, u_i) gets
// every output once, already multiplied by `scale`.
template <typename R, class Store>
__device__ void dct3_run(const DctPlan<R>& p, const Lay& y, c2<R>* a, c2<R>* b, R scale,
                         Store store) {
  const DctShape& s = p.s;
  const int n = s.n;
  const R* X = reinterpret_cast<const R*>(b);
  if (!s.fft) {
    const int total = y.L * n;
    const R w0 = scale / (R)n, w1 = (R)2 * scale / (R)n;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int l, i;
      if (y.line_fast) { l = t % y.L; i = t / y.L; }
      else { i = t % n; l = t / n; }
      const R* xl = X + l * y.lr;
      const int n4 = 4 * n;
      const int stepq = (2 * i + 1) % n4;
      int q = 0;
      R acc = 0;
      for (int k = 1; k < n; ++k) {
        q += stepq;
        if (q >= n4) q -= n4;
        acc = fma(xl[k * y.mr], p.t.cosq[q], acc);
      }
      store(l, i, fma(w1, acc, w0 * xl[0]));
    }
    return;
  }
  const int m = s.m;
  const int half = m / 2;
  const int total = y.L * (half + 1);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int l, k;
    if (y.line_fast) { l = t % y.L; k = t / y.L; }
    else { k = t % (half + 1); l = t / (half + 1); }
    const int km = m - k;  // k = 0 pairs with m
    const R* xl = X + l * y.lr;
    const R xk = xl[k * y.mr];
    const R xnk = (k == 0) ? (R)0 : xl[(n - k) * y.mr];
    const R xm = xl[km * y.mr];
    const R xnm = xl[(n - km) * y.mr];
    const R* f = p.t.ipre + 4 * k;
    const R* g = p.t.ipre + 4 * km;
    // V_k = e^{i t_k} (X_k - i X_{n-k}) and V_km, both scaled by 1/(2m)
    const R vr = fma(f[0], xk, f[1] * xnk), vi = fma(f[1], xk, -f[0] * xnk);
    const R wr = fma(g[0], xm, g[1] * xnm), wi = fma(g[1], xm, -g[0] * xnm);
    const R pr = vr + wr, pi = vi - wi;  // V_k + conj(V_km)
    const R qr = vr - wr, qi = vi + wi;  // V_k - conj(V_km)
    const R orr = fma(qr, f[2], -qi * f[3]), oi = fma(qr, f[3], qi * f[2]);
    c2<R>* al = a + l * y.lc;
    al[k * y.mc] = mk2<R>(pr - oi, pi + orr);
    if (k != 0 && km != k) {
      const R omr = fma(-qr, g[2], -qi * g[3]), omi = fma(-qr, g[3], qi * g[2]);
      al[km * y.mc] = mk2<R>(pr - omi, omr - pi);
    }
  }
  __syncthreads();
  const c2<R>* z = fft_lines<R, 1>(s, y, a, b, reinterpret_cast<const c2<R>*>(p.t.tw));
  const int tot2 = y.L * m;
  for (int t = threadIdx.x; t < tot2; t += blockDim.x) {
    int l, j;
    if (y.line_fast) { l = t % y.L; j = t / y.L; }
    else { j = t % m; l = t / m; }
    const c2<R> zv = z[l * y.lc + j * y.mc];
    const int v0 = 2 * j, v1 = 2 * j + 1;
    const int i0 = (v0 < m) ? 2 * v0 : 2 * (n - 1 - v0) + 1;
    const int i1 = (v1 < m) ? 2 * v1 : 2 * (n - 1 - v1) + 1;
    store(l, i0, zv.x * scale);
    store(l, i1, zv.y * scale);
  }
}

}  // namespace etc
