// Reference-preconditioner apply without any allocation.
//
// Some callers cannot allocate device memory: their device memory belongs to
// another allocator (a framework's caching pool that reserves the whole GPU, or
// a host application that budgets memory itself and forbids third-party
// allocations), or they cannot afford the device-wide synchronisation that
// cudaFree may cause.  This entry point serves them.  Its working memory is a
// file-scope __device__ array of fixed size, present on every GPU that loads
// the library until the process exits; the caller passes only the input and
// the output.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/etc.h"
#include "dct_device.cuh"
#include "etc_internal.cuh"
#include "launchers.h"

namespace etc {
namespace {

// Largest problem: 2^20 cells, each of n0 and n1 at most 2048.
constexpr long long kStaticMaxCells = 1LL << 20;
constexpr int kStaticMaxAxis = 2048;
// Cosine tables of one axis: tw 2m + fpost 4(m+1) + ipre 4(m+1) + cosq 4n + lam n.
constexpr long long kTableDoubles = 10LL * kStaticMaxAxis + 16;
// transform buffer + pivot table + tables of two axes (about 16.3 MiB)
constexpr long long kScratchDoubles = 2 * kStaticMaxCells + 2 * kTableDoubles;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, found once per device.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    e = set_smem_attrs<double>();
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Stockham radices of length m (same rule as the allocating path).
bool static_factor(int m, int* rad, int* nst) {
  int e2 = 0, e3 = 0, e5 = 0, v = m;
  while (v % 2 == 0) { v /= 2; ++e2; }
  while (v % 3 == 0) { v /= 3; ++e3; }
  while (v % 5 == 0) { v /= 5; ++e5; }
  if (v != 1) return false;
  int k = 0;
  while (e2 >= 3) { rad[k++] = 8; e2 -= 3; }
  if (e2 == 2) rad[k++] = 4;
  if (e2 == 1) {
    if (k > 0 && rad[k - 1] == 8) { rad[k - 1] = 4; rad[k++] = 4; }
    else rad[k++] = 2;
  }
  for (int i = 0; i < e3; ++i) rad[k++] = 3;
  for (int i = 0; i < e5; ++i) rad[k++] = 5;
  if (k > kMaxStages) return false;
  *nst = k;
  return true;
}

// Cosine tables of one axis, computed on the device (sincospi of exact
// rational multiples of pi), laid out like the host-built tables.
__global__ void k_static_tables(int n, int m, int fft, double* tw, double* fpost, double* ipre,
                                double* cosq, double* lam) {
  const int total = 4 * n + 4 * (m + 1);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    if (t < 4 * n) {
      cosq[t] = cospi((double)t / (2.0 * n));
      if (t < n) {
        const double s = sinpi((double)t / (2.0 * n));
        lam[t] = 4.0 * s * s;
      }
      if (fft && t < m) {
        double s, c;
        sincospi(-2.0 * t / m, &s, &c);
        tw[2 * t] = c;
        tw[2 * t + 1] = s;
      }
    } else if (fft) {
      const int k = t - 4 * n;
      if (k <= m) {
        double s, c;
        sincospi((double)k / (2.0 * n), &s, &c);
        fpost[4 * k + 0] = c / 2;
        fpost[4 * k + 1] = s / 2;
        fpost[4 * k + 2] = cospi(5.0 * k / (2.0 * n)) / 2;
        fpost[4 * k + 3] = sinpi(5.0 * k / (2.0 * n)) / 2;
        ipre[4 * k + 0] = c / (2.0 * m);
        ipre[4 * k + 1] = s / (2.0 * m);
        ipre[4 * k + 2] = cospi(2.0 * k / n);
        ipre[4 * k + 3] = sinpi(2.0 * k / n);
      }
    }
  }
}

// Carve one axis' tables out of `base` and queue their computation.
cudaError_t static_plan(int n, double* base, DctPlan<double>* p, const double** lam,
                        cudaStream_t s) {
  DctShape sh;
  sh.n = n;
  sh.m = n / 2;
  sh.nst = 0;
  for (int i = 0; i < kMaxStages; ++i) sh.radix[i] = 0;
  sh.fft = (n % 2 == 0) && static_factor(sh.m, sh.radix, &sh.nst);
  if (!sh.fft) sh.nst = 0;
  const int m = sh.m;
  double* tw = base;
  double* fpost = tw + 2 * (long long)m;
  double* ipre = fpost + 4 * (long long)(m + 1);
  double* cosq = ipre + 4 * (long long)(m + 1);
  double* lm = cosq + 4 * (long long)n;
  p->s = sh;
  p->t.tw = tw;
  p->t.fpost = fpost;
  p->t.ipre = ipre;
  p->t.cosq = cosq;
  *lam = lm;
  const int total = 4 * n + 4 * (m + 1);
  k_static_tables<<<(total + 255) / 256, 256, 0, s>>>(n, m, sh.fft, tw, fpost, ipre, cosq, lm);
  return cudaGetLastError();
}

}  // namespace
}  // namespace etc

using namespace etc;

extern "C" etc_status etc_apply_reference_inverse_static(int n0, int n1, int n2,
                                                         const double* kref, const double* r,
                                                         double* z, void* stream) {
  set_thread_error("");
  auto reject = [](const char* msg) { set_thread_error(msg); return ETC_EINVAL; };
  if (n0 < 1 || n1 < 1 || n2 < 1)
    return reject("etc_apply_reference_inverse_static: n0, n1, n2 must be >= 1");
  const long long n = (long long)n0 * n1 * n2;
  if (n0 > kStaticMaxAxis || n1 > kStaticMaxAxis || n > kStaticMaxCells)
    return reject("etc_apply_reference_inverse_static: beyond the fixed scratch "
                  "(n0, n1 <= 2048 and n0*n1*n2 <= 2^20 cells)");
  if (!kref || !r || !z) return reject("etc_apply_reference_inverse_static: NULL argument");
  for (int i = 0; i < 5; ++i)
    if (!(kref[i] > 0.0) || !std::isfinite(kref[i]))
      return reject("etc_apply_reference_inverse_static: kref values must be finite and > 0");
  if (z < r + n && r < z + n)
    return reject("etc_apply_reference_inverse_static: r and z overlap");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* base = nullptr;
  if (const cudaError_t se = scratch_address(&base); se != cudaSuccess) {
    char msg[192];
    std::snprintf(msg, sizeof msg,
                  "etc_apply_reference_inverse_static: device set-up of the scratch failed: %s",
                  cudaGetErrorString(se));
    set_thread_error(msg);
    return ETC_ECUDA;
  }
  double* t = base;
  double* h = base + kStaticMaxCells;
  double* tab0 = base + 2 * kStaticMaxCells;
  double* tab1 = tab0 + kTableDoubles;
  Geometry g;
  g.n0 = n0; g.n1 = n1; g.n2 = n2;
  g.plane = (long long)n0 * n1;
  g.n = n;
  DctPlan<double> p0, p1;
  const double *lam0 = nullptr, *lam1 = nullptr;
  // A failed step reports itself and the CUDA error in etc_last_error(NULL).
  auto cuda_fail = [](const char* step, cudaError_t e) {
    char msg[192];
    std::snprintf(msg, sizeof msg, "etc_apply_reference_inverse_static: %s failed: %s", step,
                  cudaGetErrorString(e));
    set_thread_error(msg);
    return ETC_ECUDA;
  };
  cudaError_t e;
  // Every scratch element read below is written earlier in this same call:
  // the tables and pivots fully, the transform buffer by the first pass.
  if ((e = static_plan(n0, tab0, &p0, &lam0, s)) != cudaSuccess)
    return cuda_fail("axis-0 cosine tables", e);
  if ((e = static_plan(n1, tab1, &p1, &lam1, s)) != cudaSuccess)
    return cuda_fail("axis-1 cosine tables", e);
  if ((e = launch_pivots<double>(g, lam0, lam1, nullptr, kref, h, s)) != cudaSuccess)
    return cuda_fail("pivot table", e);
  if ((e = launch_fwd_x<double, double>(g, p0, nullptr, nullptr, nullptr, nullptr, nullptr, r, t,
                                        nullptr, 0, 0.0, 2, s)) != cudaSuccess)
    return cuda_fail("forward transform, axis 0", e);
  if ((e = launch_dct_y<double>(g, p1, nullptr, t, 0, 0, s)) != cudaSuccess)
    return cuda_fail("forward transform, axis 1", e);
  if ((e = launch_tridiag<double>(g, nullptr, t, h, nullptr, kref[2], nullptr, 0, nullptr,
                                  nullptr, s)) != cudaSuccess)
    return cuda_fail("tridiagonal solves", e);
  if ((e = launch_dct_y<double>(g, p1, nullptr, t, 1, 0, s)) != cudaSuccess)
    return cuda_fail("backward transform, axis 1", e);
  if ((e = launch_inv_x<double, double>(g, p0, nullptr, t, z, nullptr, kref[2], 0, 0, s)) !=
      cudaSuccess)
    return cuda_fail("backward transform, axis 0", e);
  return ETC_OK;
}
