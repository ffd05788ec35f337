// Dispatch of the register-resident transforms (fast_kernels.cuh) by line
// length; the per-length launchers are instantiated in fast_sizes_*.cu.
#include "fast_kernels.cuh"

namespace etc {

bool fast_len(int n) {
  return n == 32 || n == 64 || n == 96 || n == 128 || n == 160 || n == 192 || n == 256 ||
         n == 384 || n == 512 || n == 1024;
}
int fast_threads_per_line(int n) { return fast_p(n / 2); }

namespace {
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
}  // namespace

ETC_FAST_SIZES(ETC_FAST_EXTERN)


template <typename R>
bool fast_x_ok(const Geometry& g, const DctPlan<R>& p, const void* a, const void* b,
               const void* c, const void* d) {
  return p.t.tw4 != nullptr && fast_len(g.n0) && p.s.n == g.n0 && aligned16(a) &&
         aligned16(b) && aligned16(c) && aligned16(d);
}
template bool fast_x_ok<double>(const Geometry&, const DctPlan<double>&, const void*,
                                const void*, const void*, const void*);
template bool fast_x_ok<float>(const Geometry&, const DctPlan<float>&, const void*, const void*,
                               const void*, const void*);

template <typename R>
bool fast_y_ok(const Geometry& g, const DctPlan<R>& p) {
  return p.t.tw4 != nullptr && fast_len(g.n1) && p.s.n == g.n1;
}
template bool fast_y_ok<double>(const Geometry&, const DctPlan<double>&);
template bool fast_y_ok<float>(const Geometry&, const DctPlan<float>&);

template <typename R, typename V>
cudaError_t launch_fast_fwd_x(const Geometry& g, const DctPlan<R>& p, PcgState* st, V* x,
                              const V* w, const V* q, V* r, const double* rin, R* t,
                              double* partials, int par, double rtol2, int mode,
                              cudaStream_t s, int nt) {
#define FWD(N)                                                                               \
  case N:                                                                                    \
    return fwd_x_n<R, N, V>(g, p.t, st, x, w, q, r, rin, t, partials, par, rtol2, mode, s, nt);
  switch (g.n0) {
    FWD(32) FWD(64) FWD(96) FWD(128) FWD(160) FWD(192) FWD(256) FWD(384) FWD(512) FWD(1024)
    default: return cudaErrorInvalidValue;
  }
#undef FWD
}
template cudaError_t launch_fast_fwd_x<double, double>(const Geometry&, const DctPlan<double>&,
                                                       PcgState*, double*, const double*,
                                                       const double*, double*, const double*,
                                                       double*, double*, int, double, int,
                                                       cudaStream_t, int);
template cudaError_t launch_fast_fwd_x<float, double>(const Geometry&, const DctPlan<float>&,
                                                      PcgState*, double*, const double*,
                                                      const double*, double*, const double*,
                                                      float*, double*, int, double, int,
                                                      cudaStream_t, int);
template cudaError_t launch_fast_fwd_x<float, float2>(const Geometry&, const DctPlan<float>&,
                                                      PcgState*, float2*, const float2*,
                                                      const float2*, float2*, const double*,
                                                      float*, double*, int, double, int,
                                                      cudaStream_t, int);

template <typename R, typename TZ>
cudaError_t launch_fast_inv_x(const Geometry& g, const DctPlan<R>& p, PcgState* st, const R* t,
                              TZ* z, const double* kd, double kz_host, int check, int mode,
                              cudaStream_t s, typename XOf<TZ>::T* x, int par, int nt) {
#define INV(N)                                                                      \
  case N:                                                                           \
    return inv_x_n<R, TZ, N>(g, p.t, st, t, z, kd, kz_host, check, mode, s, x, par, nt);
  switch (g.n0) {
    INV(32) INV(64) INV(96) INV(128) INV(160) INV(192) INV(256) INV(384) INV(512) INV(1024)
    default: return cudaErrorInvalidValue;
  }
#undef INV
}
template cudaError_t launch_fast_inv_x<double, double>(const Geometry&, const DctPlan<double>&,
                                                       PcgState*, const double*, double*,
                                                       const double*, double, int, int,
                                                       cudaStream_t, double*, int, int);
template cudaError_t launch_fast_inv_x<float, double>(const Geometry&, const DctPlan<float>&,
                                                      PcgState*, const float*, double*,
                                                      const double*, double, int, int,
                                                      cudaStream_t, double*, int, int);
template cudaError_t launch_fast_inv_x<float, float>(const Geometry&, const DctPlan<float>&,
                                                     PcgState*, const float*, float*,
                                                     const double*, double, int, int,
                                                     cudaStream_t, float2*, int, int);

template <typename R>
cudaError_t launch_fast_y(const Geometry& g, const DctPlan<R>& p, const PcgState* st, R* t,
                          int inverse, int check, cudaStream_t s) {
#define YN(N) \
  case N: return y_n<R, N>(g, p.t, st, t, inverse, check, s);
  switch (g.n1) {
    YN(32) YN(64) YN(96) YN(128) YN(160) YN(192) YN(256) YN(384) YN(512) YN(1024)
    default: return cudaErrorInvalidValue;
  }
#undef YN
}
template cudaError_t launch_fast_y<double>(const Geometry&, const DctPlan<double>&,
                                           const PcgState*, double*, int, int, cudaStream_t);
template cudaError_t launch_fast_y<float>(const Geometry&, const DctPlan<float>&,
                                          const PcgState*, float*, int, int, cudaStream_t);

template <typename R>
cudaError_t launch_q_fast_fwd_x(const Geometry& g, const DctTables<R>& tb, const QueueLaunch& ql,
                                int par, int nt) {
  cudaError_t e = cudaErrorInvalidValue;
#define QX(N) \
  case N: e = q_x_n<R, N>(g, tb, ql, par, 0, nt); break;
  switch (g.n0) {
    QX(32) QX(64) QX(96) QX(128) QX(160) QX(192) QX(256) QX(384) QX(512) QX(1024)
    default: return e;
  }
#undef QX
  count_launch();
  return e;
}
template <typename R>
cudaError_t launch_q_fast_inv_x(const Geometry& g, const DctTables<R>& tb,
                                const QueueLaunch& ql, int par, int nt) {
  cudaError_t e = cudaErrorInvalidValue;
#define QX(N) \
  case N: e = q_x_n<R, N>(g, tb, ql, par, 1, nt); break;
  switch (g.n0) {
    QX(32) QX(64) QX(96) QX(128) QX(160) QX(192) QX(256) QX(384) QX(512) QX(1024)
    default: return e;
  }
#undef QX
  count_launch();
  return e;
}
template <typename R>
cudaError_t launch_q_fast_y(const Geometry& g, const DctTables<R>& tb, const QueueLaunch& ql,
                            int inverse, int buf, int par) {
  if (g.n1 == 1) return cudaSuccess;  // a length-1 transform is the identity
  cudaError_t e = cudaErrorInvalidValue;
#define QY(N) \
  case N: e = q_y_n<R, N>(g, tb, ql, inverse, buf, par); break;
  switch (g.n1) {
    QY(32) QY(64) QY(96) QY(128) QY(160) QY(192) QY(256) QY(384) QY(512) QY(1024)
    default: return e;
  }
#undef QY
  count_launch();
  return e;
}
template cudaError_t launch_q_fast_fwd_x<double>(const Geometry&, const DctTables<double>&,
                                                 const QueueLaunch&, int, int);
template cudaError_t launch_q_fast_fwd_x<float>(const Geometry&, const DctTables<float>&,
                                                const QueueLaunch&, int, int);
template cudaError_t launch_q_fast_inv_x<double>(const Geometry&, const DctTables<double>&,
                                                 const QueueLaunch&, int, int);
template cudaError_t launch_q_fast_inv_x<float>(const Geometry&, const DctTables<float>&,
                                                const QueueLaunch&, int, int);
template cudaError_t launch_q_fast_y<double>(const Geometry&, const DctTables<double>&,
                                             const QueueLaunch&, int, int, int);
template cudaError_t launch_q_fast_y<float>(const Geometry&, const DctTables<float>&,
                                            const QueueLaunch&, int, int, int);

template <typename R>
cudaError_t set_fast_attrs() {
  cudaError_t e = cudaSuccess;
#define AT(N) \
  if (e == cudaSuccess) e = attrs_n<R, N>();
  AT(32) AT(64) AT(96) AT(128) AT(160) AT(192) AT(256) AT(384) AT(512) AT(1024)
#undef AT
  return e;
}
template cudaError_t set_fast_attrs<double>();
template cudaError_t set_fast_attrs<float>();

}  // namespace etc

