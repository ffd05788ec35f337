// Measurement support: the FP64 fused multiply-add rate of the device.
//
// The FP64 path of the solver is bound by the FP64 pipe, so its roofline
// fraction needs that pipe's peak.  The figure derived from unit counts and
// the maximum clock is an upper bound; this probe measures what dependent-free
// DFMA streams reach on the running clock: every thread of 148 x 8 blocks of
// 256 threads keeps eight independent FMA chains a <- a x + y, so the pipe
// never waits on a result.
#include <cuda_runtime.h>

#include "../../include/etc.h"
#include "launchers.h"

namespace etc {
namespace {

constexpr int kChains = 8;
constexpr int kProbeBlocks = 148 * 8;
constexpr int kProbeThreads = 256;

__device__ double g_probe_sink;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, double x, double y) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.0) g_probe_sink = s;  // never true; keeps the chains live
}

}  // namespace
}  // namespace etc

using namespace etc;

extern "C" etc_status etc_fp64_fma_rate(int iters, double* tflops, void* stream) {
  if (iters < 1 || !tflops) return ETC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  etc_status st = ETC_ECUDA;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    // x < 1 and y > 0: every chain converges to y / (1 - x), no overflow
    k_fma_probe<<<kProbeBlocks, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-6);  // warm-up
    count_launch();
    cudaEventRecord(e0, s);
    k_fma_probe<<<kProbeBlocks, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-6);
    count_launch();
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
      const double flops = 2.0 * kChains * (double)iters * kProbeBlocks * kProbeThreads;
      *tflops = flops / (ms * 1e-3) / 1e12;
      st = ETC_OK;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}
