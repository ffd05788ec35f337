// Dispatch of the block-floating-point transforms of the FP64 path
// (fixed_kernels.cuh) by line length; the per-length launchers are
// instantiated in fixed_sizes_*.cu.
#include "fixed_kernels.cuh"

namespace etc {

bool fx_len(int n) { return fx_len_c(n); }
int fx_threads_per_line(int n) { return fx_p(n / 2); }
int fxp_table_int4(int m) { return fxp::fx_table_int4(m); }
bool fxp_has_y3(int m) { return fxp::fx_has_y3(m); }

ETC_FX_SIZES(ETC_FX_EXTERN)
ETC_FX_Y3_SIZES(ETC_FX_Y3_EXTERN)

bool fx_y3_ok(const Geometry& g, const DctPlan<double>& p) {
  return fx_y_ok(g, p) && fxp::fx_has_y3(g.n1 / 2) && g.n1 % 2 == 0;
}
cudaError_t launch_fx_y3(const Geometry& g, const DctPlan<double>& p, const PcgState* st,
                         double* t, int inverse, int check, cudaStream_t s) {
  switch (g.n1) {
    case 256: return fx_y3_n<256>(g, p.t, st, t, inverse, check, s);
    case 512: return fx_y3_n<512>(g, p.t, st, t, inverse, check, s);
    case 1024: return fx_y3_n<1024>(g, p.t, st, t, inverse, check, s);
    default: return cudaErrorInvalidValue;
  }
}

namespace {
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
}  // namespace

bool fx_x_ok(const Geometry& g, const DctPlan<double>& p, const void* a, const void* b,
             const void* c, const void* d) {
  return p.t.fxq != nullptr && fx_len(g.n0) && p.s.n == g.n0 && aligned16(a) && aligned16(b) &&
         aligned16(c) && aligned16(d);
}
bool fx_y_ok(const Geometry& g, const DctPlan<double>& p) {
  return p.t.fxq != nullptr && fx_len(g.n1) && p.s.n == g.n1;
}

cudaError_t launch_fx_fwd_x(const Geometry& g, const DctPlan<double>& p, PcgState* st, double* x,
                            const double* w, const double* q, double* r, const double* rin,
                            double* t, double* partials, int par, double rtol2, int mode,
                            cudaStream_t s, int nt) {
#define FWD(N) \
  case N: return fx_fwd_x_n<N>(g, p.t, st, x, w, q, r, rin, t, partials, par, rtol2, mode, s, nt);
  switch (g.n0) {
    FWD(32) FWD(64) FWD(96) FWD(128) FWD(160) FWD(192) FWD(256) FWD(384) FWD(512)
    FWD(1024)
    default: return cudaErrorInvalidValue;
  }
#undef FWD
}

cudaError_t launch_fx_inv_x(const Geometry& g, const DctPlan<double>& p, PcgState* st,
                            const double* t, double* z, const double* kd, double kz_host,
                            int check, int mode, cudaStream_t s, int nt) {
#define INV(N) \
  case N: return fx_inv_x_n<N>(g, p.t, st, t, z, kd, kz_host, check, mode, s, nt);
  switch (g.n0) {
    INV(32) INV(64) INV(96) INV(128) INV(160) INV(192) INV(256) INV(384) INV(512)
    INV(1024)
    default: return cudaErrorInvalidValue;
  }
#undef INV
}

cudaError_t launch_fx_y(const Geometry& g, const DctPlan<double>& p, const PcgState* st,
                        double* t, int inverse, int check, cudaStream_t s) {
#define YN(N) \
  case N: return fx_y_n<N>(g, p.t, st, t, inverse, check, s);
  switch (g.n1) {
    YN(32) YN(64) YN(96) YN(128) YN(160) YN(192) YN(256) YN(384) YN(512) YN(1024)
    default: return cudaErrorInvalidValue;
  }
#undef YN
}

cudaError_t launch_q_fx_x(const Geometry& g, const DctPlan<double>& p, const QueueLaunch& ql,
                          int par, int inverse, int nt) {
  cudaError_t e = cudaErrorInvalidValue;
#define QX(N) \
  case N: e = q_fx_x_n<N>(g, p.t, ql, par, inverse, nt); break;
  switch (g.n0) {
    QX(32) QX(64) QX(96) QX(128) QX(160) QX(192) QX(256) QX(384) QX(512) QX(1024)
    default: return e;
  }
#undef QX
  count_launch();
  return e;
}
cudaError_t launch_q_fx_y(const Geometry& g, const DctPlan<double>& p, const QueueLaunch& ql,
                          int inverse) {
  if (g.n1 == 1) return cudaSuccess;  // a length-1 transform is the identity
  cudaError_t e = cudaErrorInvalidValue;
#define QY(N) \
  case N: e = q_fx_y_n<N>(g, p.t, ql, inverse); break;
  switch (g.n1) {
    QY(32) QY(64) QY(96) QY(128) QY(160) QY(192) QY(256) QY(384) QY(512) QY(1024)
    default: return e;
  }
#undef QY
  count_launch();
  return e;
}

cudaError_t set_fx_attrs() {
  cudaError_t e = cudaSuccess;
#define AT(N) \
  if (e == cudaSuccess) e = fx_attrs_n<N>();
  ETC_FX_SIZES(AT)
#undef AT
#define AT3(N) \
  if (e == cudaSuccess) e = fx_y3_attrs_n<N>();
  ETC_FX_Y3_SIZES(AT3)
#undef AT3
  return e;
}

}  // namespace etc
