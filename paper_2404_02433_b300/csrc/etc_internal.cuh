// Internal declarations shared by the CUDA translation units of libetc.
//
// Layout convention (all kernels): a voxel field is a dense array in the
// LOADING frame, index c = (k * N1 + j) * N0 + i, with i (axis 0) fastest and
// k (axis 2) the loading axis that carries the Dirichlet faces (the paper puts
// Gamma_in / Gamma_out at the two z faces, Sec. 2.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace etc {

constexpr int kMaxStages = 12;

// Cosine-transform plan for one axis length n (Sec. 3.2, Definition "1D DCT").
// fft == 1: even n, complex FFT of length m = n/2 by Stockham stages with the
// listed radices; fft == 0: direct O(n^2) summation with the cos table.
template <typename R>
struct DctTables {
  const R* tw;     // m complex: exp(-2 pi i j / m)
  const R* fpost;  // (m+1) x 4: cos(t)/2, sin(t)/2, cos(5t)/2, sin(5t)/2, t = pi k / (2n)
  const R* ipre;   // (m+1) x 4: cos(t)/(2m), sin(t)/(2m), cos(4t), sin(4t)
  const R* cosq;   // 4n: cos(pi q / (2n))
  const R* tw4 = nullptr;  // P x Q complex exp(-2 pi i tau k1 / m), [tau][k1], for the
                           // register-resident transforms (n = 32..512); NULL: not built
  const int4* fxq = nullptr;  // the same constants in 62-bit fixed point for the
                              // block-floating-point transforms (fixed_point.cuh);
                              // FP64 tables of n = 32..512, powers of two
};

struct DctShape {
  int n, m, fft, nst;
  int radix[kMaxStages];
};

template <typename R>
struct DctPlan {
  DctShape s;
  DctTables<R> t;
};

// Device-resident PCG scalars (Algorithm 1).  Written by the last block of the
// kernel that finishes each reduction; read by the kernels that follow.
struct PcgState {
  double rho;        // r . z of the current residual
  double beta;       // rho_new / rho (0 before the first search direction)
  double alpha[2];   // step length, by parity of the iteration
  double rr;         // ||r||^2
  double bb;         // ||b||^2
  double thresh2;    // rtol^2 ||b||^2
  double dq;         // w . A w of the current iteration
  double zq;         // flexible PCG: z_new . q_old
  double res[8];     // post-processing sums
  double ext[10];    // group extrema of the face assembly
  double kref_lp[5]; // centred LP optimum sqrt(min_g max_g) (Algorithm 2), from ext
  double kref[5];    // reference parameters in use (x, y, z, in, out)
  int iter;          // completed iterations (products with A)
  int maxit;
  int done;          // 1 once converged / stopped; kernels then return at entry
  int status;        // ETC_OK / ETC_ENOCONV / ETC_EBREAKDOWN
  int phase;         // 0 = initial preconditioner apply, 1 = iterating
  int passes;        // loop-body passes of a device-driven (graph) loop
  int max_passes;    // hard cap on passes (ends the loop even without `done`)
  int xpend;         // 1 + parity of an iteration whose x += alpha w is still due
                     // (r was updated, the w update that carries x has not run)
  unsigned int cnt[8];  // arrival counters of the last-block reductions
  double* hist;      // ring of ||r_i||^2 by iteration i (i = 0: ||r_0||^2), hist_cap entries
  int hist_cap;
  double bb_given;   // ||b||^2 when the initial guess is not 0 (else 0: ||b|| = ||r_0||)
};

enum CounterSlot { kCntDot = 0, kCntRes = 1, kCntRho = 2, kCntAux = 3, kCntFlux = 4,
                   kCntExt = 5, kCntZq = 6 };

// Status values mirrored from include/etc.h.
enum { kOK = 0, kEINVAL = 1, kENOMEM = 2, kECUDA = 3, kENOCONV = 4, kEBREAKDOWN = 5,
       kESTATE = 6 };

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block in a fixed order; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) t += sh[w];
  return t;
}

// Coordinates of one unit of work of a kernel: the hardware block of an
// ordinary launch, or an item that a persistent block took from a batch work
// queue (batch.cu), which stands for block (x, y, z) of the launch of one
// solve that the item replaces.  The reductions below count arrivals and
// index partials by these coordinates, so a kernel body written against them
// runs unchanged in both forms.
struct Blk {
  unsigned int x, y, z, nx, ny, nz;
};
// Bulk prefetch of [p, p + bytes) into L2: nothing is waited on and no
// register is held (p 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned int bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// Blocks of kernel k (nt threads, sm bytes of dynamic shared memory) resident
// on the current device at once; 0 if a query fails.
template <typename K>
int resident_blocks(K k, int nt, size_t sm) {
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, sm) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return per_sm * sms;
}
__device__ __forceinline__ Blk hw_blk() {
  return {blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z};
}

// Publish one partial per block; returns true in the block that arrives last.
// That block may then read every partial (with __ldcg) in index order, which
// makes the reduction deterministic.  The counter is reset for the next use.
__device__ __forceinline__ bool publish_partial(double* partials, int nparts, double value,
                                                int slot_stride, unsigned int* counter,
                                                int* is_last_sh) {
  const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
  (void)nparts;
  if (threadIdx.x == 0) {
    partials[(size_t)bid * slot_stride] = value;
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    *is_last_sh = (prev == nb - 1);
  }
  __syncthreads();
  const bool last = *is_last_sh != 0;
  if (last) __threadfence();
  return last;
}

// Fixed-order sum of nb partials by one block (deterministic).
__device__ __forceinline__ double sum_partials(const double* partials, int nb, int stride,
                                               double* sh) {
  double v = 0.0;
  // each thread sums a contiguous chunk, then the chunks are added in order;
  // the chunk's loads are issued eight at a time ahead of the additions
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  const int b1 = min(b0 + per, nb);
  int b = b0;
  for (; b + 8 <= b1; b += 8) {
    double t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = __ldcg(partials + (size_t)(b + u) * stride);
#pragma unroll
    for (int u = 0; u < 8; ++u) v += t[u];
  }
  for (; b < b1; ++b) v += __ldcg(partials + (size_t)b * stride);
  // ordered combination of the per-thread chunks
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  // warp-level ordered tree is deterministic for a fixed blockDim
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) t += sh[w];
  return t;
}

// Each block writes nv values, the last block to arrive gets true.
__device__ __forceinline__ bool publish_values(double* partials, int stride, const double* vals,
                                               int nv, unsigned int* counter, int* flag,
                                               const Blk& b = hw_blk()) {
  const unsigned int bid = b.x + b.nx * (b.y + b.ny * b.z);
  const unsigned int nb = b.nx * b.ny * b.nz;
  if (threadIdx.x == 0) {
    for (int v = 0; v < nv; ++v) partials[(size_t)bid * stride + v] = vals[v];
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    *flag = (prev == nb - 1);
  }
  __syncthreads();
  const bool last = *flag != 0;
  if (last) __threadfence();
  return last;
}

__device__ __forceinline__ unsigned int nblocks(const Blk& b = hw_blk()) {
  return b.nx * b.ny * b.nz;
}

// End of the residual-update kernels (Algorithm 1, exit test): block partials
// of ||r||^2, summed in block order by the last block, which records ||r||^2
// (MODE 0: also ||b||^2 and the threshold rtol^2 ||b||^2) and decides
// convergence, the iteration cap and breakdown.  MODE 1 with `defer` marks
// this iteration's x += alpha w as due (the w-update kernel applies it).
template <int MODE>
__device__ __forceinline__ void fwd_x_residual_tail(double acc, PcgState* st, double* partials,
                                                    double rtol2, double* sh, int* flag,
                                                    int par, bool defer,
                                                    const Blk& b = hw_blk()) {
  const double bs = block_sum(acc, sh);
  double v[1] = {bs};
  if (publish_values(partials, 1, v, 1, &st->cnt[kCntRes], flag, b)) {
    const double rr = sum_partials(partials, (int)nblocks(b), 1, sh);
    if (threadIdx.x == 0) {
      st->rr = rr;
      if (MODE == 0) {
        // the exit test is relative to ||b|| (Eq. exit): r_0 = b for x0 = 0
        const double bb = st->bb_given > 0.0 ? st->bb_given : rr;
        st->bb = bb;
        st->thresh2 = rtol2 * bb;
        if (!(bb > 0.0) || !isfinite(rr)) { st->status = kEBREAKDOWN; st->done = 1; }
        else if (st->bb_given > 0.0 && rr <= st->thresh2) { st->status = kOK; st->done = 1; }
      } else {
        st->iter += 1;
        st->xpend = defer ? par + 1 : 0;
        if (!isfinite(rr)) { st->status = kEBREAKDOWN; st->done = 1; }
        else if (rr <= st->thresh2) { st->status = kOK; st->done = 1; }
        else if (st->iter >= st->maxit) { st->status = kENOCONV; st->done = 1; }
      }
      // convergence history: ||r||^2 of iteration st->iter (0 after the start)
      if (st->hist) st->hist[st->iter % st->hist_cap] = rr;
      st->cnt[kCntRes] = 0;
    }
  }
}

// ---------------------------------------------------------------- host launchers
struct Geometry {
  int n0, n1, n2;     // loading-frame sizes
  long long n;        // n0 * n1 * n2
  long long plane;    // n0 * n1
};

// ---------------------------------------------------------------- batch work queue
// The iterations of a batch run as persistent launches, one per kernel of the
// PCG iteration and per class of solves (the same loading-frame sizes and
// precision).  Each block of such a launch takes items from the class's queue
// with one atomic add per item; item i stands for block i % per of the
// one-solve launch of solve active[i / per], and the kernel body runs with
// those block coordinates (Blk).  Only solves still iterating are listed, so
// finished solves cost nothing; the loop control of each pass rebuilds the
// list and rewinds the counters.
constexpr int kQueueSlots = 12;  // launches per pass of the loop body: 2 iterations x 6 kernels
struct BatchQueue {
  unsigned int next[kQueueSlots];  // items taken, per launch of the pass
  int nactive;                     // solves still iterating (entries of active)
  int nsolves;
  int* active;                     // nsolves entries, ascending solve index
};

// Device addresses of one solve of a batch (one RVE, one loading direction).
// The mixed path views x, r and q as double-float pairs (same 8 bytes).
struct BatchSolve {
  PcgState* st;
  double* partials;
  double *x, *r, *q, *w;          // solution, residual, A w, search direction (FP64 path)
  float* wf;                      // FP32 search direction (mixed path)
  const double *T0, *T1, *T2, *D; // FP64 faces (with the zero plane) and diagonal
  const float2 *F0, *F1, *F2, *FB;  // double-float faces and Dirichlet planes (mixed path)
  double* t64;                    // FP64 transform buffer
  const double* h64;              // FP64 reciprocal pivots
  float* t32;                     // FP32 transform buffer (z^, z)
  float* rhat[2];                 // FP32 r^ of the last two iterations
  float2* ck;                     // checkpoints of the FP32 tridiagonal sweeps
};

// The item loop of a persistent launch on slot `slot` (every thread of the
// block runs it): body(solve, local) for each item the block takes, items
// numbered solve-major over the active solves, `per` (blocks of one solve)
// each.  Thread 0 requests the next item with one atomic add as the current
// one starts and reads the answer only when it ends, so the round trip to
// the counter overlaps the item's work.
template <class Body>
__device__ __forceinline__ void queue_loop(BatchQueue* q, int slot, unsigned int per,
                                           Body body) {
  __shared__ unsigned int next_sh;
  const unsigned int total = (unsigned int)q->nactive * per;
  if (threadIdx.x == 0) next_sh = atomicAdd(&q->next[slot], 1u);
  __syncthreads();
  unsigned int cur = next_sh;
#pragma unroll 1
  while (cur < total) {
    __syncthreads();  // every thread holds cur before next_sh is rewritten
    unsigned int pre = 0u;
    if (threadIdx.x == 0) pre = atomicAdd(&q->next[slot], 1u);
    body(q->active[cur / per], cur % per);
    if (threadIdx.x == 0) next_sh = pre;
    __syncthreads();
    cur = next_sh;
  }
}

// Block coordinates of item `local` of a launch of nx x ny x nz blocks.
__device__ __forceinline__ Blk item_blk(unsigned int local, unsigned int nx, unsigned int ny,
                                        unsigned int nz) {
  return {local % nx, (local / nx) % ny, local / (nx * ny), nx, ny, nz};
}

}  // namespace etc

namespace etc {

// ---------------------------------------------------------------- conversions
// FP32 <-> FP64 with integer operations only, from the IEEE-754 binary32 and
// binary64 formats.  On B300 the hardware conversion instructions issue on
// the FP64 pipe, which the FP64 arithmetic of the solver already saturates;
// these versions run on the integer pipes instead.

// Exact widening (every binary32 value, subnormals, infinities and NaN).
__device__ __forceinline__ double widen(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int s = u & 0x80000000u;
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned int m = u & 0x7FFFFFu;
  unsigned int hi, lo;
  if (e != 0u && e != 0xFFu) {            // normal: rebias 127 -> 1023
    hi = s | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  } else if (e == 0xFFu) {                // infinity / NaN
    hi = s | 0x7FF00000u | (m >> 3);
    lo = m << 29;
  } else if (m == 0u) {                   // signed zero
    hi = s;
    lo = 0u;
  } else {                                // subnormal: value m * 2^-149
    const int p = 31 - __clz((int)m);     // position of the leading one
    const unsigned long long frac = (unsigned long long)(m ^ (1u << p)) << (52 - p);
    hi = s | ((unsigned int)(p + 874) << 20) | (unsigned int)(frac >> 32);
    lo = (unsigned int)frac;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// Narrowing with round-to-nearest-even (binary32 subnormals produced, values
// above the binary32 range become infinity, NaN stays NaN).
__device__ __forceinline__ float narrow(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned int s = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  if (e == 0x7FF) return __uint_as_float(s | 0x7F800000u | (mant ? 0x400000u : 0u));
  const int e32 = e - 896;
  if (e32 >= 255) return __uint_as_float(s | 0x7F800000u);
  if (e32 >= 1) {
    unsigned int bits = ((unsigned int)e32 << 23) | (unsigned int)(mant >> 29);
    const unsigned int rem = (unsigned int)(mant & 0x1FFFFFFFull);
    if (rem > 0x10000000u || (rem == 0x10000000u && (bits & 1u))) bits += 1u;
    return __uint_as_float(s | bits);
  }
  if (e == 0) return __uint_as_float(s);  // binary64 subnormal: far below binary32
  const int shift = 30 - e32;             // 29 fraction bits + (1 - e32) denormalising
  if (shift > 53) return __uint_as_float(s);
  const unsigned long long full = mant | (1ull << 52);
  unsigned int bits = (unsigned int)(full >> shift);
  const unsigned long long rem = full & ((1ull << shift) - 1ull);
  const unsigned long long half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (bits & 1u))) bits += 1u;
  return __uint_as_float(s | bits);
}

template <typename T> __device__ __forceinline__ double to_f64(T v);
template <> __device__ __forceinline__ double to_f64<double>(double v) { return v; }
template <> __device__ __forceinline__ double to_f64<float>(float v) { return widen(v); }
template <typename T> __device__ __forceinline__ T from_f64(double v);
template <> __device__ __forceinline__ double from_f64<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_f64<float>(double v) { return narrow(v); }

}  // namespace etc

namespace etc {

// ---------------------------------------------------------------- double-float
// A value held as an unevaluated sum hi + lo of two binary32 numbers with
// |lo| <= ulp(hi)/2 ("double-float", a 48-bit significand): the FP32 pipe,
// 64 times faster than the FP64 pipe on B300, then does the FP64-class work of
// the mixed-precision matvec.  The algorithms are the error-free
// transformations TwoSum (Knuth) and TwoProduct by FMA, and the cascaded
// summation Sum2 of Ogita, Rump and Oishi (2005).

// Exact split of a binary64 value: hi = RN32(d), lo = RN32(d - hi), from the
// bit fields with integer operations only (no FP64 instruction).  Values whose
// remainder falls below the binary32 normal range (|d| < 2^-74), subnormal
// binary64 input, infinities and NaN keep lo = 0.
__device__ __forceinline__ float2 split_df(double d) {
  const float hi = narrow(d);
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7FF);
  const int be = e - 948;  // biased binary32 exponent of 2^(e - 1075)
  if (e - 896 < 1 || be < 1 || (__float_as_uint(hi) & 0x7F800000u) == 0x7F800000u)
    return make_float2(hi, 0.0f);
  const unsigned long long sig = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned int low = (unsigned int)(sig & 0x1FFFFFFFull);  // bits below hi's last bit
  const bool up = low > 0x10000000u || (low == 0x10000000u && ((sig >> 29) & 1ull));
  const int rem = up ? (int)low - 0x20000000 : (int)low;  // d - hi = rem * 2^(e - 1075)
  float lo = __int2float_rn(rem) * __int_as_float(be << 23);
  if (b >> 63) lo = -lo;
  return make_float2(hi, lo);
}

// s + t = a + b exactly, s = RN(a + b)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}

// Sum2 step: (s, e) <- (s, e) + sign * x * y for double-float x, y.  The
// product keeps hi*hi exactly (FMA) plus the two cross terms; lo*lo is below
// the format's precision.
template <int SIGN>
__device__ __forceinline__ void df_fma_acc(float2 x, float2 y, float& s, float& e) {
  float p = x.x * y.x;
  float pe = fma(x.x, y.x, -p);
  pe = fma(x.x, y.y, pe);
  pe = fma(x.y, y.x, pe);
  if (SIGN < 0) { p = -p; pe = -pe; }
  float t;
  two_sum(s, p, s, t);
  e += t + pe;
}

}  // namespace etc

namespace etc {

// ---------------------------------------------------------------- PCG vector storage
// The outer PCG vectors (x, r, w, q) are FP64 in the FP64 path; the mixed
// path keeps x, r, q as double-float pairs (float2) and the search direction w
// in FP32.  These overloads give the kernels one source for all of them.

// y + a x.  For double-float: TwoProduct of the high parts by FMA plus the
// cross terms, TwoSum with y's high part, then renormalisation.
__device__ __forceinline__ double vaxpy(double a, double x, double y) { return fma(a, x, y); }
__device__ __forceinline__ float2 vaxpy(float2 a, float2 x, float2 y) {
  const float p = a.x * x.x;
  float pe = fma(a.x, x.x, -p);
  pe = fma(a.x, x.y, pe);
  pe = fma(a.y, x.x, pe);
  float s, t;
  two_sum(y.x, p, s, t);
  t += y.y + pe;
  const float hi = s + t;
  return make_float2(hi, t - (hi - s));
}

template <typename V> struct Scalar;  // the scalar type a vector of V is scaled by
template <> struct Scalar<double> {
  using T = double;
  static __device__ __forceinline__ double from(double a) { return a; }
  static __device__ __forceinline__ double neg(double a) { return -a; }
};
template <> struct Scalar<float2> {
  using T = float2;
  static __device__ __forceinline__ float2 from(double a) { return split_df(a); }
  static __device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
};
template <> struct Scalar<float> {
  using T = float;
  static __device__ __forceinline__ float from(double a) { return narrow(a); }
  static __device__ __forceinline__ float neg(float a) { return -a; }
};

// FP32 search directions (the double-float path keeps w in FP32: it is only a
// direction, and x and r are updated with the same rounded w and its exact
// double-float product A w, so the recursive residual still tracks b - A x).
__device__ __forceinline__ float vaxpy(float a, float x, float y) { return fmaf(a, x, y); }

// Storage of x that goes with a storage of w: FP32 directions with double-float x.
template <typename TW> struct XOf { using T = TW; };
template <> struct XOf<float> { using T = float2; };
// x + alpha w with w in its own storage
__device__ __forceinline__ double xaxpy(double a, double w, double x) { return fma(a, w, x); }
__device__ __forceinline__ float2 xaxpy(float2 a, float2 w, float2 x) { return vaxpy(a, w, x); }
__device__ __forceinline__ float2 xaxpy(float2 a, float w, float2 x) {
  return vaxpy(a, make_float2(w, 0.f), x);
}

// A vector value as the FP64 or FP32 input of the preconditioner's transforms
// (double-float -> binary32: the high part, which is the nearest binary32).
template <typename R> __device__ __forceinline__ R vround(double v) { return from_f64<R>(v); }
template <typename R> __device__ __forceinline__ R vround(float2 v);
template <> __device__ __forceinline__ float vround<float>(float2 v) { return v.x; }

// ||v||^2 partial sums: FP64 for FP64 vectors; for double-float vectors the
// square of the high part in FP32 (the sum feeds the exit test only).
__device__ __forceinline__ void vsq_acc(double v, double& acc, float&) { acc = fma(v, v, acc); }
__device__ __forceinline__ void vsq_acc(float2 v, double&, float& accf) {
  accf = fma(v.x, v.x, accf);
}

// the value u (the transform's output, type R) as a vector element
template <typename V, typename R> __device__ __forceinline__ V vfrom(R u);
template <> __device__ __forceinline__ double vfrom<double, double>(double u) { return u; }
template <> __device__ __forceinline__ double vfrom<double, float>(float u) { return widen(u); }
template <> __device__ __forceinline__ float2 vfrom<float2, float>(float u) {
  return make_float2(u, 0.f);
}
template <> __device__ __forceinline__ float vfrom<float, float>(float u) { return u; }

// two consecutive elements, 16 bytes
template <typename V> struct VPair { V a, b; };
__device__ __forceinline__ VPair<double> ld_pair(const double* p) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  return {v.x, v.y};
}
__device__ __forceinline__ VPair<float2> ld_pair(const float2* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ VPair<float> ld_pair(const float* p) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  return {v.x, v.y};
}
__device__ __forceinline__ void st_pair(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void st_pair(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
__device__ __forceinline__ void st_pair(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
// element as FP64 (double-float: hi + lo rounded once)
__device__ __forceinline__ void store_f64(double* p, double v) { *p = v; }
__device__ __forceinline__ void store_f64(double* p, float2 v) { *p = widen(v.x) + widen(v.y); }

template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ double vzero<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ float vzero<float>() { return 0.f; }

}  // namespace etc

namespace etc {

// ---------------------------------------------------------------- tridiagonal solves
// (kernels.cu and tridiag_tma.cu)

// End of the tridiagonal kernels: block partials of rho (and of z_new . r_old
// for MODE 2), summed in block order by the last block, which forms beta.
template <int MODE>
__device__ __forceinline__ void tridiag_tail(double acc, double acc2, PcgState* st,
                                             double* partials, double w4, const double* kd,
                                             double kz_host, double* sh, int* flag_,
                                             const Blk& blk = hw_blk()) {
  int& flag = *flag_;
  double v[2];
  v[0] = block_sum(acc, sh);
  v[1] = (MODE == 2) ? block_sum(acc2, sh) : 0.0;
  if (publish_values(partials, 2, v, 2, &st->cnt[kCntRho], &flag, blk)) {
    const double wscale = w4 / (kd ? kd[2] : kz_host);
    double rho_new = 0.0, zr_old = 0.0;
    {
      // fixed-order sums of both columns
      const int nb = (int)nblocks(blk);
      double a0 = 0.0, a1 = 0.0;
      const int per = (nb + blockDim.x - 1) / blockDim.x;
      const int b0 = threadIdx.x * per;
      const int b1 = min(b0 + per, nb);
      int b = b0;
      for (; b + 4 <= b1; b += 4) {  // loads ahead of the in-order additions
        double2 t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          t[u] = __ldcg(reinterpret_cast<const double2*>(partials) + b + u);
#pragma unroll
        for (int u = 0; u < 4; ++u) { a0 += t[u].x; a1 += t[u].y; }
      }
      for (; b < b1; ++b) {
        a0 += __ldcg(partials + 2 * (size_t)b);
        a1 += __ldcg(partials + 2 * (size_t)b + 1);
      }
      rho_new = wscale * block_sum(a0, sh);
      zr_old = wscale * block_sum(a1, sh);
    }
    if (threadIdx.x == 0) {
      if (!(rho_new > 0.0) || !isfinite(rho_new)) {
        if (st->phase == 0 || !(rho_new == 0.0)) { st->status = kEBREAKDOWN; st->done = 1; }
      }
      if (st->phase == 0 || MODE == 3) {
        st->beta = 0.0;
        st->phase = 1;
      } else if (MODE == 1) {
        st->beta = rho_new / st->rho;
      } else {
        st->beta = (rho_new - zr_old) / st->rho;
        st->zq = zr_old;
      }
      st->rho = rho_new;
      if (!isfinite(st->beta)) { st->status = kEBREAKDOWN; st->done = 1; }
      st->cnt[kCntRho] = 0;
    }
  }
}

// FP32 solves with the pivots generated per column (k_tridiag_otf in
// kernels.cu, k_tridiag_tma in tridiag_tma.cu): the column's constants, one
// step of the forward recurrence, and the chunk length of the checkpoints.
constexpr int kTriChunk = 8;

struct TriCol {
  float sig;     // sigma
  float first;   // sigma + a_in (n2 = 1: the whole diagonal sigma + a_in + a_out)
  float last;    // sigma + a_out
};
// 1/d for the pivots (d >= 1 away from the corners, always > 0 and finite):
// the hardware approximation refined by one Newton-Raphson step
// r <- r + r (1 - d r), which leaves an error within about one ulp.  Both
// sweeps use this same function, so the regenerated pivots are bit-identical.
__device__ __forceinline__ float tri_rcp(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return fmaf(r, fmaf(-d, r, 1.0f), r);
}
// kappa_ref ratios kx/kz, ky/kz, 2 kin/kz, 2 kout/kz (one thread per block)
__device__ __forceinline__ void tri_coef(const double* kd, float* coef) {
  const double kz = kd[2];
  coef[0] = narrow(kd[0] / kz);
  coef[1] = narrow(kd[1] / kz);
  coef[2] = narrow(2.0 * kd[3] / kz);
  coef[3] = narrow(2.0 * kd[4] / kz);
}
// the constants of column (i, j) from the eigenvalue tables and the ratios
__device__ __forceinline__ TriCol tri_col(int i, int j, int n2, const double* lam0,
                                          const double* lam1, const float* coef) {
  TriCol a;
  a.sig = fmaf(narrow(lam0[i]), coef[0], narrow(lam1[j]) * coef[1]);
  a.first = a.sig + coef[2];
  a.last = a.sig + coef[3];
  if (n2 == 1) a.first = a.first + coef[3];
  return a;
}
// One plane of the forward recurrence: y_k = r_k + h_{k-1} y_{k-1}, then the
// pivot of plane k.  State before plane 0: e = h = y = 0.
__device__ __forceinline__ void tri_step(const TriCol& a, int k, int n2, float r, float& e,
                                         float& h, float& y) {
  y = fmaf(h, y, r);
  float d;
  if (n2 == 1) {
    d = a.first;
  } else if (k == n2 - 1) {
    d = fmaf(e, h, a.last);
  } else {
    e = fmaf(e, h, k == 0 ? a.first : a.sig);
    d = 1.0f + e;
  }
  h = tri_rcp(d);
}

}  // namespace etc
