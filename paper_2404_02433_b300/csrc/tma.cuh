// Tensor Memory Accelerator helpers shared by the bulk-tensor kernels:
// mbarrier initialisation, transaction-count arrival, bounded waits, tiled
// 2-D/3-D copies into shared memory, and the host-side tensor-map encoder
// (cuTensorMapEncodeTiled, reached through the runtime's driver entry point,
// so the library needs no link against the driver library).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace etc {

// A wait gives up after 0.5 s of wall time (a plane's copies take
// microseconds), with an iteration cap as a second bound.
constexpr unsigned long long kWaitNs = 500000000ull;
constexpr unsigned int kWaitPolls = 1u << 24;

__device__ __forceinline__ unsigned int smem_addr(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// one test of the phase; the thread may be suspended up to ~2 us meanwhile
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(2000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long wall_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the phase of the given parity; false when it ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned int parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = wall_ns();
  for (unsigned int it = 0; it < kWaitPolls; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (wall_ns() - t0 > kWaitNs) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
      "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load2(void* dst, const CUtensorMap* map, int x, int y,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiled tma_encoder() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// Tiled map of a dense tensor (dims and byte strides of the outer dims; box
// extents in elements); no interleave or swizzle, zero fill outside.  False
// when the encoder is unavailable or rejects the arguments.
inline bool tma_encode(CUtensorMap* m, CUtensorMapDataType type, unsigned int rank,
                       const void* base, const unsigned long long* dim,
                       const unsigned long long* stride, const unsigned int* box) {
  const EncodeTiled enc = tma_encoder();
  if (!enc) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t bx[5], es[5];
  for (unsigned int i = 0; i < rank; ++i) {
    d[i] = dim[i];
    bx[i] = box[i];
    es[i] = 1;
    if (i + 1 < rank) st[i] = stride[i];
  }
  return enc(m, type, rank, const_cast<void*>(base), d, st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace etc
