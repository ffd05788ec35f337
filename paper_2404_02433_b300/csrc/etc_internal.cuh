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
  unsigned int cnt[8];  // arrival counters of the last-block reductions
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
  // each thread sums a contiguous chunk, then the chunks are added in order
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  for (int b = b0; b < b0 + per && b < nb; ++b) v += __ldcg(partials + (size_t)b * stride);
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

// ---------------------------------------------------------------- host launchers
struct Geometry {
  int n0, n1, n2;     // loading-frame sizes
  long long n;        // n0 * n1 * n2
  long long plane;    // n0 * n1
};

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
