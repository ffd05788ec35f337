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

// Two-ended ("twisted") form of the same solves for grids that fit in one
// wave, where each SM holds a few warps and the time is the length of each
// column's recurrence.  The column is eliminated from both ends at once: the
// top chain runs the recurrence above over planes 0 .. m-1, the bottom chain
// its mirror image from plane n2-1 down to m+1,
//   y'_k = r_k + g_{k+1} y'_{k+1},  e'_k = sigma + e'_{k+1} g_{k+1} (e'_{n2-1} = sigma + a_out),
//   g_k = 1 / (1 + e'_k),
// both in the same thread, so their latencies overlap.  At the middle plane m
//   gamma = sigma + (m = 0 ? a_in : e_{m-1} h_{m-1}) + (m = n2-1 ? a_out : e'_{m+1} g_{m+1}),
//   y~ = r_m + h_{m-1} y_{m-1} + g_{m+1} y'_{m+1},   z_m = y~ / gamma,
// (the middle row of T z = r with z_{m-1} and z_{m+1} eliminated; every term
// is positive, as in the one-ended form), and the back-substitution runs
// outward: z_k = h_k (y_k + z_{k+1}) above m, z_k = g_k (y'_k + z_{k-1})
// below.  rho = r^.T^{-1}r^ is the sum of h_k y_k^2, g_k y'_k^2 and y~ z_m.
// The chunks go in pairs: use u < ntop takes top chunk u and bottom chunk
// nch-1-u, the backward uses take them in the opposite order, and m is the
// last plane of top chunk ntop-1 (ntop = ceil(nch/2)).  Checkpoints: the top
// chain's state at the start of chunk c in row c-1, the bottom chain's state
// on entering chunk c (from above) in row c; the rows do not overlap.
// Measured against the one-ended kernel at 128^3 / 160^3: 36.9 -> 34.8 us and
// 43.8 -> 41.0 us (each SMSP holds one warp there, and the time per plane is
// the warp's instruction sequence more than the recurrence's latency).
constexpr int kTwStages = 4;
constexpr int kTwStageBytes = 4 * kTriBox;  // top r^, bottom r^, top r_old, bottom r_old
constexpr int kTwSmem = kTwStages * kTwStageBytes + 128 + 128;

__device__ __forceinline__ void tw_step(float r, float c0, float& e, float& h, float& y) {
  y = fmaf(h, y, r);
  e = fmaf(e, h, c0);
  h = tri_rcp(1.0f + e);
}

template <int MODE>
__global__ void __launch_bounds__(kTriCols, 3)
    k_tridiag_tw(const __grid_constant__ CUtensorMap min_, const __grid_constant__ CUtensorMap mold,
                 Geometry g, PcgState* st, float* __restrict__ out, float2* __restrict__ ck,
                 const double* __restrict__ lam0, const double* __restrict__ lam1,
                 const double* __restrict__ kd, double w4, double* partials) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double sh[32];
  __shared__ float coef[4];
  __shared__ int flag, failed;
  if (st->done) return;
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + kTwStages * kTwStageBytes);
  const int n2 = g.n2;
  const int nch = (n2 + kTriChunk - 1) / kTriChunk;
  const int ntop = (nch + 1) / 2, nbot = nch - ntop;
  const int m = min(kTriChunk * ntop, n2) - 1;
  const int nuse = 2 * ntop;
  const int s0 = blockIdx.x * kTriCols;
  auto top_of = [&](int u) { return u < ntop ? u : 2 * ntop - 1 - u; };
  auto bot_of = [&](int u) {
    const int q = u < ntop ? u : u - ntop;
    return q < nbot ? (u < ntop ? nch - 1 - q : ntop + q) : -1;
  };
  auto issue = [&](int u) {
    const int sidx = u % kTwStages;
    unsigned char* sg = smem + sidx * kTwStageBytes;
    unsigned long long* b = bars + sidx;
    const int ct = top_of(u), cb = bot_of(u);
    const bool two = MODE == 2 && u >= ntop;
    mbar_expect_tx(b, (cb >= 0 ? 2u : 1u) * (two ? 2u : 1u) * kTriBox);
    tma_load2(sg, &min_, s0, ct * kTriChunk, b);
    if (cb >= 0) tma_load2(sg + kTriBox, &min_, s0, cb * kTriChunk, b);
    if (two) {
      tma_load2(sg + 2 * kTriBox, &mold, s0, ct * kTriChunk, b);
      if (cb >= 0) tma_load2(sg + 3 * kTriBox, &mold, s0, cb * kTriChunk, b);
    }
  };
  if (threadIdx.x == 0) {
    failed = 0;
    tri_coef(kd, coef);
    for (int sidx = 0; sidx < kTwStages; ++sidx) mbar_init(bars + sidx, 1);
    mbar_init_fence();
    for (int u = 0; u < nuse && u < kTwStages - 1; ++u) issue(u);
  }
  __syncthreads();
  const long long s = s0 + threadIdx.x;
  const bool own = s < g.plane;
  const int i = own ? (int)(s % g.n0) : 0, j = own ? (int)(s / g.n0) : 0;
  const TriCol a = tri_col(i, j, n2, lam0, lam1, coef);
  const long long pl = g.plane;
  float et = 0.f, ht = 0.f, yt = 0.f;  // top chain
  float eb = 0.f, hb = 0.f, yb = 0.f;  // bottom chain
  float part = 0.f, rm = 0.f, zm = 0.f, zt = 0.f, zb = 0.f, zr = 0.f;
  int u = 0;
  for (; u < nuse; ++u) {
    const int sidx = u % kTwStages;
    if (threadIdx.x == 0 && !mbar_wait(bars + sidx, (unsigned int)((u / kTwStages) & 1)))
      failed = 1;
    __syncthreads();
    if (failed) break;
    if (threadIdx.x == 0 && u + kTwStages - 1 < nuse) issue(u + kTwStages - 1);
    const float* rt = reinterpret_cast<const float*>(smem + sidx * kTwStageBytes) + threadIdx.x;
    const float* rb = rt + kTriBox / 4;
    const int ct = top_of(u), cb = bot_of(u);
    const int kt = ct * kTriChunk, kb = cb * kTriChunk;
    if (u < ntop) {  // elimination towards the middle
      if (own && ct > 0) ck[(long long)(ct - 1) * pl + s] = make_float2(et, yt);
      if (own && cb >= 0 && cb < nch - 1) ck[(long long)cb * pl + s] = make_float2(eb, yb);
#pragma unroll
      for (int v = 0; v < kTriChunk; ++v) {
        const int k = kt + v;
        if (k < m) {
          tw_step(rt[v * kTriCols], k == 0 ? a.first : a.sig, et, ht, yt);
          part = fmaf(ht * yt, yt, part);
        } else if (k == m) {
          rm = rt[v * kTriCols];
        }
        const int w = kTriChunk - 1 - v, k2 = kb + w;
        if (cb >= 0 && k2 > m && k2 < n2) {
          tw_step(rb[w * kTriCols], k2 == n2 - 1 ? a.last : a.sig, eb, hb, yb);
          part = fmaf(hb * yb, yb, part);
        }
      }
      if (u == ntop - 1) {  // both chains have reached the middle plane
        const float t = m == 0 ? coef[2] : et * ht;
        const float b = m == n2 - 1 ? coef[3] : eb * hb;
        const float gam = a.sig + t + b;
        const float ym = fmaf(hb, yb, fmaf(ht, yt, rm));
        zm = ym * tri_rcp(gam);
        part = fmaf(ym, zm, part);
        zt = zm;
        zb = zm;
      }
    } else {  // back-substitution away from the middle
      float2 c1 = make_float2(0.f, 0.f), c2 = make_float2(0.f, 0.f);
      if (own && ct > 0) c1 = ck[(long long)(ct - 1) * pl + s];
      if (own && cb >= 0 && cb < nch - 1) c2 = ck[(long long)cb * pl + s];
      float e1 = c1.x, y1 = c1.y, h1 = ct > 0 ? tri_rcp(1.0f + c1.x) : 0.f;
      float e2 = c2.x, y2 = c2.y, h2 = (cb >= 0 && cb < nch - 1) ? tri_rcp(1.0f + c2.x) : 0.f;
      float hv1[kTriChunk], yv1[kTriChunk], hv2[kTriChunk], yv2[kTriChunk];
#pragma unroll
      for (int v = 0; v < kTriChunk; ++v) {
        const int k = kt + v;
        if (k < m) {
          tw_step(rt[v * kTriCols], k == 0 ? a.first : a.sig, e1, h1, y1);
          hv1[v] = h1;
          yv1[v] = y1;
        }
        const int w = kTriChunk - 1 - v, k2 = kb + w;
        if (cb >= 0 && k2 > m && k2 < n2) {
          tw_step(rb[w * kTriCols], k2 == n2 - 1 ? a.last : a.sig, e2, h2, y2);
          hv2[w] = h2;
          yv2[w] = y2;
        }
      }
      const float* ot = rt + 2 * kTriBox / 4;  // r_old of the top chunk
      const float* ob = rt + 3 * kTriBox / 4;  // r_old of the bottom chunk
#pragma unroll
      for (int v = 0; v < kTriChunk; ++v) {
        const int w = kTriChunk - 1 - v, k = kt + w;
        if (k < m) {
          zt = hv1[w] * (yv1[w] + zt);
          if (own) out[(long long)k * pl + s] = zt;
          if (MODE == 2) zr = fmaf(zt, ot[w * kTriCols], zr);
        } else if (k == m) {
          if (own) out[(long long)k * pl + s] = zm;
          if (MODE == 2) zr = fmaf(zm, ot[w * kTriCols], zr);
        }
        const int k2 = kb + v;
        if (cb >= 0 && k2 > m && k2 < n2) {
          zb = hv2[v] * (yv2[v] + zb);
          if (own) out[(long long)k2 * pl + s] = zb;
          if (MODE == 2) zr = fmaf(zb, ob[v * kTriCols], zr);
        }
      }
    }
  }
  if (failed) {
    if (threadIdx.x == 0) {
      for (int uu = u; uu < nuse && uu < u + kTwStages - 1; ++uu)
        (void)mbar_wait(bars + uu % kTwStages, (unsigned int)((uu / kTwStages) & 1));
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
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tridiag_tw<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTwSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tridiag_tw<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTwSmem);
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
  static const int res_tw = resident_blocks(k_tridiag_tw<2>, kTriCols, kTwSmem);
  if (res_tw > 0 && (int)nb <= res_tw) {  // one wave: the two-ended form
    if (mode == 2)
      k_tridiag_tw<2><<<nb, kTriCols, kTwSmem, s>>>(min_, mold, g, st, out, ck, lam0, lam1, kd,
                                                    w4, partials);
    else
      k_tridiag_tw<3><<<nb, kTriCols, kTwSmem, s>>>(min_, mold, g, st, out, ck, lam0, lam1, kd,
                                                    w4, partials);
    count_launch();
    return cudaGetLastError();
  }
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
