// FP32 tridiagonal solves of the flexible PCG (Sec. 3.2, Algorithm 3 step 2)
// with the operands staged by the Tensor Memory Accelerator.
//
// The arithmetic is that of k_tridiag_otf (kernels.cu): pivots generated per
// column by the positive recurrence of tri_step, the forward sweep keeping the
// state (e, y) at the start of every chunk of kTriChunk planes, the backward
// sweep regenerating each chunk's pivots and y from its checkpoint and solving
// down it; rho = r^.T^{-1}r^ and z_new.r_old by Parseval.  A block owns 128
// consecutive columns.  Instead of each thread loading its own planes, thread
// 0 issues one tiled bulk-tensor copy per chunk (128 columns x kTriChunk
// planes of r^; in the backward sweep also of r_old) into a ring of stages,
// chunks in the order they are used: the forward chunks 0 .. nch-1, then the
// backward chunks nch-1 .. 0, so the copies for the start of the backward
// sweep are already in flight at the end of the forward one.  Thread 0 waits
// (bounded) for the chunk in use, a block barrier hands it to every thread and
// frees the stage of the previous chunk.  Copies beyond the plane (the last
// block) or below n2 (the last chunk) are zero-filled.
// Two shapes of the ring, chosen per launch: 4 stages with 6 blocks per SM,
// or 3 stages with 8 blocks per SM (at most 64 registers).  The launcher takes
// the one that runs the grid in fewer waves of resident blocks, and on a tie
// the deeper ring: measured at 512^3 (2048 blocks) 0.428 -> 0.403 ms with 3
// stages; at 128^3..256^3 (under one wave either way) 4 stages were 3-5 %
// faster.  Both shapes do the same arithmetic, so their results are identical.
// Row strides of the maps are plane * 4 bytes: plane must be a multiple of 4.
#include <cuda.h>
#include <cuda_runtime.h>

#include "etc_internal.cuh"
#include "launchers.h"
#include "tma.cuh"

namespace etc {

namespace {

constexpr int kTriCols = 128;                            // columns per block
constexpr int kTriBox = kTriCols * kTriChunk * 4;        // bytes of one r^ (or r_old) box
constexpr int kTriStageBytes = 2 * kTriBox;              // r^ then r_old
// dynamic shared memory of a ring of `stages` stages, + barriers, + alignment
constexpr int tri_smem(int stages) { return stages * kTriStageBytes + 128 + 128; }

}  // namespace

template <int MODE, int STAGES, int MINB>
__global__ void __launch_bounds__(kTriCols, MINB)
    k_tridiag_tma(const __grid_constant__ CUtensorMap min_, const __grid_constant__ CUtensorMap mold,
                  Geometry g, PcgState* st, float* __restrict__ out, float2* __restrict__ ck,
                  const double* __restrict__ lam0, const double* __restrict__ lam1,
                  const double* __restrict__ kd, double w4, double* partials) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double sh[32];
  __shared__ float coef[4];
  __shared__ int flag, failed;
  if (st->done) return;
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(smem + STAGES * kTriStageBytes);
  const int n2 = g.n2;
  const int nch = (n2 + kTriChunk - 1) / kTriChunk;
  const int nuse = 2 * nch;  // chunk uses: forward 0..nch-1, backward nch-1..0
  const int s0 = blockIdx.x * kTriCols;
  // use u: its chunk and whether it is a backward use
  auto chunk_of = [&](int u) { return u < nch ? u : 2 * nch - 1 - u; };
  auto issue = [&](int u) {
    const int sidx = u % STAGES;
    unsigned char* sg = smem + sidx * kTriStageBytes;
    unsigned long long* b = bars + sidx;
    const int kb = chunk_of(u) * kTriChunk;
    const bool two = MODE == 2 && u >= nch;
    mbar_expect_tx(b, two ? 2 * kTriBox : kTriBox);
    tma_load2(sg, &min_, s0, kb, b);
    if (two) tma_load2(sg + kTriBox, &mold, s0, kb, b);
  };
  if (threadIdx.x == 0) {
    failed = 0;
    tri_coef(kd, coef);
    for (int sidx = 0; sidx < STAGES; ++sidx) mbar_init(bars + sidx, 1);
    mbar_init_fence();
    for (int u = 0; u < nuse && u < STAGES - 1; ++u) issue(u);
  }
  __syncthreads();
  const long long s = s0 + threadIdx.x;
  const bool own = s < g.plane;
  const int i = own ? (int)(s % g.n0) : 0, j = own ? (int)(s / g.n0) : 0;
  const TriCol a = tri_col(i, j, n2, lam0, lam1, coef);
  const long long pl = g.plane;
  float e = 0.f, h = 0.f, y = 0.f, part = 0.f, zn = 0.f, zr = 0.f;
  float2 cp = make_float2(0.f, 0.f);  // checkpoint of the backward chunk in use
  int u = 0;
  for (; u < nuse; ++u) {
    const int sidx = u % STAGES;
    if (threadIdx.x == 0 && !mbar_wait(bars + sidx, (unsigned int)((u / STAGES) & 1)))
      failed = 1;
    __syncthreads();
    if (failed) break;
    // every thread is past use u-1: its stage takes use u + STAGES - 1
    if (threadIdx.x == 0 && u + STAGES - 1 < nuse) issue(u + STAGES - 1);
    const float* sr = reinterpret_cast<const float*>(smem + sidx * kTriStageBytes) + threadIdx.x;
    const int ch = chunk_of(u);
    const int kb = ch * kTriChunk;
    if (u < nch) {  // forward sweep
      if (own && ch > 0) ck[(long long)(ch - 1) * pl + s] = make_float2(e, y);
      if (ch == nch - 1) cp = make_float2(e, y);  // the first backward chunk starts here
#pragma unroll
      for (int v = 0; v < kTriChunk; ++v) {
        const int k = kb + v;
        if (k < n2) {
          tri_step(a, k, n2, sr[v * kTriCols], e, h, y);
          part = fmaf(h * y, y, part);
        }
      }
    } else {  // backward sweep
      float2 cn = make_float2(0.f, 0.f);
      if (own && ch > 1) cn = ck[(long long)(ch - 2) * pl + s];  // the next chunk's state
      float ec = cp.x, yc = cp.y, hc = ch > 0 ? tri_rcp(1.0f + cp.x) : 0.f;
      float hv[kTriChunk], yv[kTriChunk];
#pragma unroll
      for (int v = 0; v < kTriChunk; ++v) {
        const int k = kb + v;
        if (k < n2) {
          tri_step(a, k, n2, sr[v * kTriCols], ec, hc, yc);
          hv[v] = hc;
          yv[v] = yc;
        }
      }
      const float* so = sr + kTriChunk * kTriCols;  // r_old of the chunk
#pragma unroll
      for (int v = kTriChunk - 1; v >= 0; --v) {
        const int k = kb + v;
        if (k < n2) {
          zn = hv[v] * (yv[v] + zn);
          if (own) out[(long long)k * pl + s] = zn;
          if (MODE == 2) zr = fmaf(zn, so[v * kTriCols], zr);
        }
      }
      cp = cn;
    }
  }
  if (failed) {
    if (threadIdx.x == 0) {
      // drain this block's copies still in flight (bounded), then report
      for (int uu = u; uu < nuse && uu < u + STAGES - 1; ++uu)
        (void)mbar_wait(bars + uu % STAGES, (unsigned int)((uu / STAGES) & 1));
      st->status = kECUDA;
      st->done = 1;
    }
    return;
  }
  double acc = 0.0, acc2 = 0.0;
  if (own) {
    const double wgt = (i == 0 ? 0.5 : 1.0) * (j == 0 ? 0.5 : 1.0);
    acc = wgt * widen(part);
    if (MODE == 2) acc2 = wgt * widen(zr);
  }
  tridiag_tail<MODE>(acc, acc2, st, partials, w4, kd, 1.0, sh, &flag);
}

bool tridiag_tma_map(const Geometry& g, const float* buf, CUtensorMap* m) {
  if (g.plane % 4 != 0 || reinterpret_cast<unsigned long long>(buf) % 16 != 0) return false;
  const unsigned long long dim[2] = {(unsigned long long)g.plane, (unsigned long long)g.n2};
  const unsigned long long stride[1] = {(unsigned long long)g.plane * 4};
  const unsigned int box[2] = {(unsigned int)kTriCols, (unsigned int)kTriChunk};
  return tma_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, buf, dim, stride, box);
}

namespace {

// the two ring shapes: 4 stages and 6 blocks per SM, 3 stages and 8
template <int MODE> constexpr auto kDeep = k_tridiag_tma<MODE, 4, 6>;
template <int MODE> constexpr auto kWide = k_tridiag_tma<MODE, 3, 8>;

template <typename K>
cudaError_t set_smem(K k, int stages) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, tri_smem(stages));
}

}  // namespace

cudaError_t set_tridiag_tma_attrs() {
  cudaError_t e = set_smem(kDeep<2>, 4);
  if (e == cudaSuccess) e = set_smem(kDeep<3>, 4);
  if (e == cudaSuccess) e = set_smem(kWide<2>, 3);
  if (e == cudaSuccess) e = set_smem(kWide<3>, 3);
  return e;
}

cudaError_t launch_tridiag_tma(const Geometry& g, const CUtensorMap& min_,
                               const CUtensorMap& mold, PcgState* st, float* out, float2* ck,
                               const double* lam0, const double* lam1, const double* kd,
                               double* partials, int mode, cudaStream_t s) {
  const unsigned int nb = (unsigned int)((g.plane + kTriCols - 1) / kTriCols);
  const double w4 = 4.0 / ((double)g.n0 * g.n1);
  // waves of resident blocks each shape needs for this grid (the shape's
  // residency is the same for both modes)
  static const int res_deep = resident_blocks(kDeep<2>, kTriCols, tri_smem(4));
  static const int res_wide = resident_blocks(kWide<2>, kTriCols, tri_smem(3));
  const long long waves_deep = res_deep > 0 ? (nb + res_deep - 1) / res_deep : 1;
  const long long waves_wide = res_wide > 0 ? (nb + res_wide - 1) / res_wide : waves_deep;
  if (waves_wide < waves_deep) {
    if (mode == 2)
      kWide<2><<<nb, kTriCols, tri_smem(3), s>>>(min_, mold, g, st, out, ck, lam0, lam1, kd, w4,
                                                 partials);
    else
      kWide<3><<<nb, kTriCols, tri_smem(3), s>>>(min_, mold, g, st, out, ck, lam0, lam1, kd, w4,
                                                 partials);
  } else {
    if (mode == 2)
      kDeep<2><<<nb, kTriCols, tri_smem(4), s>>>(min_, mold, g, st, out, ck, lam0, lam1, kd, w4,
                                                 partials);
    else
      kDeep<3><<<nb, kTriCols, tri_smem(4), s>>>(min_, mold, g, st, out, ck, lam0, lam1, kd, w4,
                                                 partials);
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace etc
