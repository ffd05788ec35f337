// Double-float TPFA matvec fed by the Tensor Memory Accelerator.
//
// The same operator and arithmetic as k_matvec_df (kernels.cu): the
// face-difference form of Eq. (scaled bilinear forms),
//   (Aw)_c = sum_f T_f (w_c - w_f) + [k = 0] B_in w_c + [k = n2-1] B_out w_c,
// in double-float pairs on the FP32 pipe, summed by Sum2, with the partial
// w.q of Algorithm 1 (alpha = rho / w.q) in MODE 1.  Only the way the
// operands reach the threads differs.  A block owns a 32 x 8 column tile and
// marches over kchunk planes; for each plane, four tiled bulk-tensor copies
// land in a ring of kStages shared-memory stages:
//   T0 (x i0 .. i0+33, 8 rows)      the minus x faces and the plus face of the last column
//   T1 (32 columns, y j0 .. j0+8)   the minus y faces and the plus faces of the last row
//   T2 of plane k+1 (32 x 8)        the faces above the plane
//   w (x i0-4 .. i0+35, y j0-1 .. j0+8) the plane with a one-cell halo (FP32
//                                   search direction; x rounded down to a multiple
//                                   of 4: a copy's first x times 4 bytes must be
//                                   16-byte aligned)
// Copies that reach outside the box are filled with zeros by the hardware,
// which are exactly the Neumann faces (T = 0) and harmless finite neighbours.
// The block is warp-specialised: 4 consumer warps (two adjacent tile rows each) and one
// producer warp.  Each stage has a "full" mbarrier (completed by the copies'
// transaction bytes) and an "empty" one (one arrival per consumer warp).  The
// producer issues plane k into its stage once the consumers have released the
// stage's previous plane; each consumer warp waits for planes k and k+1 (the
// z neighbour), sums its row of plane k and releases that stage.  There is no
// block barrier in the loop; the copies of up to kStages-1 planes are in
// flight without holding registers.  Every wait is bounded: a wait that runs
// out sets status ETC_ECUDA and done in the solver state, the producer drains
// the block's copies (bounded again) and the block returns.  tx_extra (0 in
// use) adds bytes that no copy delivers to every stage's expected count: a
// test sets it (ETC_TEST_TMA_TX_EXTRA, read at create) so that the waits run
// out and the error path runs without any fault.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "etc_internal.cuh"
#include "launchers.h"
#include "tma.cuh"

namespace etc {

namespace {

constexpr int kStages = 4;
constexpr int kConsumers = 4;                     // warps
constexpr int kRowsPerWarp = 2;                   // adjacent tile rows 2w and 2w + 1
constexpr int kTileY = kConsumers * kRowsPerWarp; // 8
constexpr int kThreads = (kConsumers + 1) * 32;   // + one producer warp
// box extents (elements of 8 bytes)
constexpr int kT0X = 34, kT0Y = 8;
constexpr int kT1X = 32, kT1Y = 9;
constexpr int kT2X = 32, kT2Y = 8;
constexpr int kWX = 40, kWY = 10;  // w is FP32: x from i0-4 (16-byte aligned)
constexpr int kT0Bytes = kT0X * kT0Y * 8;   // 2176
constexpr int kT1Bytes = kT1X * kT1Y * 8;   // 2304
constexpr int kT2Bytes = kT2X * kT2Y * 8;   // 2048
constexpr int kWBytes = kWX * kWY * 4;      // 1600
constexpr int kTx = kT0Bytes + kT1Bytes + kT2Bytes + kWBytes;
constexpr int align128(int b) { return (b + 127) / 128 * 128; }
constexpr int kOffT1 = align128(kT0Bytes);
constexpr int kOffT2 = kOffT1 + align128(kT1Bytes);
constexpr int kOffW = kOffT2 + align128(kT2Bytes);
constexpr int kStageBytes = kOffW + align128(kWBytes);
// + the mbarriers, + slack to align the stages to 128 bytes at run time
constexpr int kSmemBytes = kStages * kStageBytes + 128 + 128;
static_assert(2 * kStages * 8 <= 128, "full and empty barriers fit behind the stages");
// The Sum2 step and the products of the double-float matvec, as in kernels.cu
__device__ __forceinline__ void two_sum_(float a, float b, float& s, float& t) {
  s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void acc_(float p, float pe, float& s, float& e) {
  float t;
  two_sum_(s, p, s, t);
  e += t + pe;
}
// p + pe ~ T (a - b) for FP32 a, b (the search direction): TwoSum gives the
// difference exactly as dh + dl
__device__ __forceinline__ void flux_f(float2 T, float a, float b, float& p, float& pe) {
  float dh, dl;
  two_sum_(a, -b, dh, dl);
  p = T.x * dh;
  pe = fma(T.x, dh, -p);
  pe = fma(T.x, dl, pe);
  pe = fma(T.y, dh, pe);
}
// (s, e) += x w for double-float x and FP32 w
__device__ __forceinline__ void prod_acc_f(float2 x, float w, float& s, float& e) {
  const float p = x.x * w;
  float pe = fma(x.x, w, -p);
  pe = fma(x.y, w, pe);
  acc_(p, pe, s, e);
}

}  // namespace

template <int MODE>
__global__ void __launch_bounds__(kThreads, 6)
    k_matvec_df_tma(const __grid_constant__ MatvecMaps mp, Geometry g, PcgState* st,
                    const float* __restrict__ w, float2* __restrict__ q,
                    const float2* __restrict__ T2, const float2* __restrict__ Bin,
                    const float2* __restrict__ Bout, double* partials, int par, int kchunk,
                    unsigned int tx_extra) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double sh[32];
  __shared__ int flag, failed;
  if (MODE == 1 && st->done) return;
  // the copies' destinations start on 128-byte boundaries
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + kStages * kStageBytes);
  unsigned long long* empty = full + kStages;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * kTileY;
  const int k0 = blockIdx.z * kchunk;
  const int k1 = min(k0 + kchunk, g.n2);
  const int kend = min(k1, g.n2 - 1);  // last plane loaded (k1 supplies w above k1-1)
  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, kConsumers);
    }
    mbar_init_fence();
  }
  __syncthreads();
  volatile int* vfailed = &failed;
  float ds = 0.f, dc = 0.f;
  if (warp == kConsumers) {
    // producer: plane k goes to stage (k - k0) mod kStages once the consumer
    // warps have released that stage's previous plane
    if (lane == 0) {
      int issued = 0;
      for (int k = k0; k <= kend; ++k) {
        const int u = k - k0;
        const unsigned int s = (unsigned int)(u % kStages);
        if (u >= kStages && !mbar_wait(empty + s, (unsigned int)(((u / kStages) - 1) & 1))) {
          *vfailed = 1;
          break;
        }
        if (*vfailed) break;
        unsigned char* sg = smem + s * kStageBytes;
        mbar_expect_tx(full + s, kTx + tx_extra);
        tma_load3(sg, &mp.T0, i0, j0, k, full + s);
        tma_load3(sg + kOffT1, &mp.T1, i0, j0, k, full + s);
        tma_load3(sg + kOffT2, &mp.T2, i0, j0, k + 1, full + s);
        tma_load3(sg + kOffW, &mp.w, i0 - 4, j0 - 1, k, full + s);
        ++issued;
      }
      // no copy may still be landing when the block exits (bounded)
      for (int u = max(0, issued - kStages); u < issued; ++u)
        (void)mbar_wait(full + u % kStages, (unsigned int)((u / kStages) & 1));
    }
    __syncwarp();
  } else {
    // consumer warp: tile rows r and r + kConsumers, one column per lane
    const int l = lane;
    const int i = i0 + l;
    const long long pl = g.plane;
    bool own[kRowsPerWarp];
    long long sidx[kRowsPerWarp];
    float fz[kRowsPerWarp], fze[kRowsPerWarp];
    float2* pq[kRowsPerWarp];
    int oT0[kRowsPerWarp], oT1[kRowsPerWarp], oT2[kRowsPerWarp], oW[kRowsPerWarp];
#pragma unroll
    for (int h = 0; h < kRowsPerWarp; ++h) {
      const int r = kRowsPerWarp * warp + h, j = j0 + r;
      own[h] = i < g.n0 && j < g.n1;
      sidx[h] = (long long)j * g.n0 + i;
      // flux through the face below plane k0: T2[k0] (w_{k0-1} - w_{k0})
      fz[h] = 0.f;
      fze[h] = 0.f;
      if (own[h] && k0 > 0) {
        const long long c = (long long)k0 * pl + sidx[h];
        flux_f(T2[c], w[c - pl], w[c], fz[h], fze[h]);
      }
      // this row's element offsets inside a stage (float2 units; w: float)
      oT0[h] = r * kT0X + l;
      oT1[h] = r * kT1X + l;
      oT2[h] = r * kT2X + l;
      oW[h] = (r + 1) * kWX + l + 4;
      pq[h] = q + (long long)k0 * pl + sidx[h];
    }
    unsigned int sc = 0, pc = 0;  // stage and parity of plane k
    bool seen = false;            // plane k's copies were seen complete (as plane k+1)
    for (int k = k0; k < k1; ++k) {
      const unsigned int sn = sc + 1 == kStages ? 0u : sc + 1;
      const unsigned int pn = sn == 0 ? pc ^ 1u : pc;
      // every lane waits (bounded) for planes k and k+1 (the z neighbour); a
      // stage seen complete stays so until this warp releases it
      bool ok = seen || mbar_wait(full + sc, pc);
      if (ok && k + 1 <= kend) ok = mbar_wait(full + sn, pn);
      seen = k + 1 <= kend;
      if (!__all_sync(0xffffffffu, ok) || *vfailed) {
        *vfailed = 1;
        break;
      }
      const unsigned char* sg = smem + sc * kStageBytes;
      const float* sWn = reinterpret_cast<const float*>(smem + sn * kStageBytes + kOffW);
#pragma unroll
      float yp = 0.f, ype = 0.f;  // flux through the face between this warp's rows
      for (int h = 0; h < kRowsPerWarp; ++h) {
        if (!own[h]) continue;
        const float2* sT0 = reinterpret_cast<const float2*>(sg) + oT0[h];
        const float2* sT1 = reinterpret_cast<const float2*>(sg + kOffT1) + oT1[h];
        const float2* sT2 = reinterpret_cast<const float2*>(sg + kOffT2) + oT2[h];
        const float* sW = reinterpret_cast<const float*>(sg + kOffW) + oW[h];
        const float wc = sW[0];
        const float wp = k + 1 <= kend ? sWn[oW[h]] : wc;
        float sv, ev, p, pe;
        flux_f(sT0[0], wc, sW[-1], sv, ev);
        flux_f(sT0[1], wc, sW[1], p, pe);
        acc_(p, pe, sv, ev);
        // the minus y face of the second row is the plus y face of the first,
        // whose flux (exact differences, so exactly negated) is reused
        if (h == 0) {
          flux_f(sT1[0], wc, sW[-kWX], p, pe);
        } else {
          p = -yp;
          pe = -ype;
        }
        acc_(p, pe, sv, ev);
        flux_f(sT1[kT1X], wc, sW[kWX], p, pe);
        yp = p;
        ype = pe;
        acc_(p, pe, sv, ev);
        acc_(-fz[h], -fze[h], sv, ev);
        flux_f(sT2[0], wc, wp, fz[h], fze[h]);
        acc_(fz[h], fze[h], sv, ev);
        if (k == 0) prod_acc_f(Bin[sidx[h]], wc, sv, ev);
        if (k == g.n2 - 1) prod_acc_f(Bout[sidx[h]], wc, sv, ev);
        float qh, ql;
        two_sum_(sv, ev, qh, ql);
        *pq[h] = make_float2(qh, ql);
        if (MODE == 1) prod_acc_f(make_float2(qh, ql), wc, ds, dc);
        pq[h] += pl;
      }
      // the warp is done with plane k's stage (plane k-1 no longer reads it)
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + sc);
      sc = sn;
      pc = pn;
    }
  }
  __syncthreads();
  if (failed) {
    if (threadIdx.x == 0) {
      st->status = kECUDA;
      st->done = 1;
    }
    return;
  }
  if (MODE == 1) {
    const double bs = block_sum(widen(ds) + widen(dc), sh);
    double v[1] = {bs};
    if (publish_values(partials, 1, v, 1, &st->cnt[kCntDot], &flag)) {
      const double dq = sum_partials(partials, (int)nblocks(), 1, sh);
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

namespace {

// esize 8: double-float pairs, 4: FP32
bool encode3(CUtensorMap* m, const void* base, int esize, int n0, int n1, int nz, int bx,
             int by) {
  const unsigned long long dim[3] = {(unsigned long long)n0, (unsigned long long)n1,
                                     (unsigned long long)nz};
  const unsigned long long stride[2] = {(unsigned long long)n0 * esize,
                                        (unsigned long long)n0 * n1 * esize};
  const unsigned int box[3] = {(unsigned int)bx, (unsigned int)by, 1};
  return tma_encode(m, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    3, base, dim, stride, box);
}

}  // namespace

bool matvec_tma_maps(const Geometry& g, const float2* T0, const float2* T1, const float2* T2,
                     const float* w, MatvecMaps* mp) {
  // row strides must be multiples of 16 bytes (n0 a multiple of 4 for the FP32
  // w) and the bases 16-byte aligned
  if (g.n0 % 4 != 0) return false;
  for (const void* p : {(const void*)T0, (const void*)T1, (const void*)T2, (const void*)w})
    if (reinterpret_cast<unsigned long long>(p) % 16 != 0) return false;
  std::memset(mp, 0, sizeof(*mp));
  return encode3(&mp->T0, T0, 8, g.n0, g.n1, g.n2, kT0X, kT0Y) &&
         encode3(&mp->T1, T1, 8, g.n0, g.n1, g.n2, kT1X, kT1Y) &&
         encode3(&mp->T2, T2, 8, g.n0, g.n1, g.n2 + 1, kT2X, kT2Y) &&  // + the zero plane
         encode3(&mp->w, w, 4, g.n0, g.n1, g.n2, kWX, kWY);
}

cudaError_t set_matvec_tma_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_matvec_df_tma<0>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_matvec_df_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kSmemBytes);
}

cudaError_t launch_matvec_df_tma(const Geometry& g, const MatvecMaps& mp, PcgState* st,
                                 const float* w, float2* q, const float2* T2, const float2* FB,
                                 double* partials, int par, int mode, cudaStream_t s,
                                 unsigned int tx_extra) {
  int kc;
  const dim3 grid = matvec_df_grid(g, &kc);
  const float2* Bout = FB + g.plane;
  if (mode == 1)
    k_matvec_df_tma<1><<<grid, kThreads, kSmemBytes, s>>>(mp, g, st, w, q, T2, FB, Bout, partials, par,
                                                     kc, tx_extra);
  else
    k_matvec_df_tma<0><<<grid, kThreads, kSmemBytes, s>>>(mp, g, st, w, q, T2, FB, Bout, partials, par,
                                                     kc, tx_extra);
  count_launch();
  return cudaGetLastError();
}

}  // namespace etc
