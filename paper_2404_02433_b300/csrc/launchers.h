// Host-side launchers of the kernels in kernels.cu (internal to libetc).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "etc_internal.cuh"

namespace etc {

// Reason of the calling thread's last failed call that has no handle (what
// etc_last_error(NULL) returns); defined with the C ABI.
void set_thread_error(const char* msg);

cudaError_t launch_kappa_stats(const double* a, long long n, double* partials, PcgState* st,
                               int slot, cudaStream_t s);
cudaError_t launch_permute(const double* in, double* out, int d0, int d1, int d2, long long s0,
                           long long s1, long long s2, cudaStream_t s);
cudaError_t launch_faces(const Geometry& g, double ih0, double ih1, double ih2, const double* k0,
                         const double* k1, const double* k2, double* T0, double* T1, double* T2,
                         double* D, double* Bin, double* Bout, double* partials, PcgState* st,
                         cudaStream_t s);
// The diagonal D from the faces and Bin/Bout, and the double-float copies of
// T0, T1, T2 (with the extra plane) and of Bin, Bout (FB: 2 planes).
cudaError_t launch_diag_split(const Geometry& g, const double* T0, const double* T1,
                              const double* T2, const double* Bin, const double* Bout, double* D,
                              float2* F0, float2* F1, float2* F2, float2* FB, cudaStream_t s);
unsigned int faces_blocks(const Geometry& g);
// kref_dev (device, may be NULL) takes precedence over kref_host (host, 5 values).
template <typename R>
cudaError_t launch_pivots(const Geometry& g, const double* lam0, const double* lam1,
                          const double* kref_dev, const double* kref_host, R* h, cudaStream_t s);
cudaError_t launch_select_kref(PcgState* st, int mode, const double* user, cudaStream_t s);
cudaError_t launch_state_reset(PcgState* st, int maxit, cudaStream_t s);
cudaError_t launch_loop_control(PcgState* st, cudaGraphConditionalHandle handle,
                                cudaStream_t s);
cudaError_t launch_init(const Geometry& g, const double* Bin, const double* Bout, double pin,
                        double pout, double* r, double* x, double* w0, cudaStream_t s,
                        const double* pin_f = nullptr, const double* pout_f = nullptr,
                        const double* src = nullptr);
// x0 of a homogeneous medium (linear in k) and ||b||^2 of r = b into st->bb_given.
cudaError_t launch_init_linear(const Geometry& g, double pin, double pout, const double* r,
                               double* x, double* partials, PcgState* st, cudaStream_t s);
cudaError_t launch_sub(long long n, double* r, const double* q, cudaStream_t s);  // r -= q
cudaError_t launch_matvec(const Geometry& g, PcgState* st, const double* w, double* q,
                          const double* T0, const double* T1, const double* T2, const double* D,
                          double* partials, int par, int mode, cudaStream_t s);
// Mixed-precision matvec on double-float faces and Dirichlet planes (FB as in
// launch_diag_split) and q, with the FP32 search direction w (which needs n0
// zero guard elements on both sides); mode 1 as k_matvec.
cudaError_t launch_matvec_df(const Geometry& g, PcgState* st, const float* w, float2* q,
                             const float2* T0, const float2* T1, const float2* T2,
                             const float2* FB, double* partials, int par, int mode,
                             cudaStream_t s);
// The same matvec with its operands staged by tiled bulk-tensor copies
// (matvec_tma.cu).  The maps describe T0, T1, T2 (with its zero plane) of one
// loading frame as [n2][n1][n0] arrays of 8-byte pairs and w as FP32; they
// exist when n0 is a multiple of 4 and the bases are 16-byte aligned
// (matvec_tma_maps returns false otherwise, and launch_matvec_df serves that
// frame).
struct MatvecMaps {
  CUtensorMap T0, T1, T2, w;
};
bool matvec_tma_maps(const Geometry& g, const float2* T0, const float2* T1, const float2* T2,
                     const float* w, MatvecMaps* mp);
cudaError_t set_matvec_tma_attrs();
cudaError_t launch_matvec_df_tma(const Geometry& g, const MatvecMaps& mp, PcgState* st,
                                 const float* w, float2* q, const float2* T2, const float2* FB,
                                 double* partials, int par, int mode, cudaStream_t s,
                                 unsigned int tx_extra = 0);
// FP32 tridiagonal solves of the flexible PCG (modes 2 and 3 of
// launch_tridiag_otf) with r^ and r_old staged by tiled bulk-tensor copies
// (tridiag_tma.cu).  The maps view an FP32 field as [n2][plane]; they exist
// when plane is a multiple of 4 and the base 16-byte aligned.
bool tridiag_tma_map(const Geometry& g, const float* buf, CUtensorMap* m);
cudaError_t set_tridiag_tma_attrs();
cudaError_t launch_tridiag_tma(const Geometry& g, const CUtensorMap& min_,
                               const CUtensorMap& mold, PcgState* st, float* out, float2* ck,
                               const double* lam0, const double* lam1, const double* kd,
                               double* partials, int mode, cudaStream_t s);
// grid and planes per thread of both double-float matvec kernels
dim3 matvec_df_grid(const Geometry& g, int* kchunk);
void count_launch();  // one more library kernel launched
cudaError_t launch_split_df(const double* a, float2* b, long long n, cudaStream_t s);
// FP64 values to double-float pairs in place.
cudaError_t launch_split_inplace(double* a, long long n, cudaStream_t s);
// V: storage of x, w, q, r (double, or float2 double-float pairs with
// R = float); x += alpha w happens here for FP64 storage only (mode 1);
// rin (mode 2) is FP64.
template <typename R, typename V>
cudaError_t launch_fwd_x(const Geometry& g, const DctPlan<R>& p, PcgState* st, V* x, const V* w,
                         const V* q, V* r, const double* rin, R* t, double* partials, int par,
                         double rtol2, int mode, cudaStream_t s, int L = 0);
template <typename R>
cudaError_t launch_dct_y(const Geometry& g, const DctPlan<R>& p, const PcgState* st, R* t,
                         int inverse, int check, cudaStream_t s, int TI = 0);
// kd (device kref, may be NULL) supplies kappa_ref^z, else kz_host.
template <typename R>
cudaError_t launch_tridiag(const Geometry& g, PcgState* st, R* t, const R* h, const double* kd,
                           double kz_host, double* partials, int mode, R* rnew, const R* rold,
                           cudaStream_t s);
// FP32 tridiagonal solves with the pivots generated per column (mixed paths):
// r^ from in, z to out (may be in), checkpoints in ck (tridiag_ck_pairs(g)
// pairs), kd the device kref; mode as launch_tridiag, rold for mode 2.
cudaError_t launch_tridiag_otf(const Geometry& g, PcgState* st, const float* in, float* out,
                               float2* ck, const double* lam0, const double* lam1,
                               const double* kd, double* partials, int mode, const float* rold,
                               cudaStream_t s);
size_t tridiag_ck_pairs(const Geometry& g);
// mode 2 with x: also x += alpha[par] w (old w) before w is replaced.  x is
// stored as XOf<TZ> (double-float when the directions w are FP32).
template <typename R, typename TZ>
cudaError_t launch_inv_x(const Geometry& g, const DctPlan<R>& p, PcgState* st, const R* t, TZ* z,
                         const double* kd, double kz_host, int check, int mode, cudaStream_t s,
                         int L = 0, typename XOf<TZ>::T* x = nullptr, int par = 0);
// End of a solve: the x += alpha w still due (see PcgState::xpend), then for
// double-float storage (df = 1: w is the FP32 direction wf) x back to FP64 in
// place; df = 0: FP64 x and w.
cudaError_t launch_finish_x(const Geometry& g, const PcgState* st, double* x, const double* w,
                            const float* wf, int df, cudaStream_t s);
cudaError_t launch_flux(const Geometry& g, const double* x, const double* T0, const double* T1,
                        const double* T2, const double* Bin, const double* Bout, double pin,
                        double pout, double* partials, PcgState* st, cudaStream_t s);
cudaError_t launch_true_residual(const Geometry& g, const double* x, const double* T0,
                                 const double* T1, const double* T2, const double* D,
                                 const double* Bin, const double* Bout, double pin, double pout,
                                 double* partials, PcgState* st, cudaStream_t s,
                                 const double* pin_f = nullptr, const double* pout_f = nullptr,
                                 const double* src = nullptr);
cudaError_t launch_widen(const float* a, double* b, long long n, cudaStream_t s);
cudaError_t launch_gradient(const Geometry& g, const double* x, const double* lam,
                            const double* k0, const double* k1, const double* k2, double ih0,
                            double ih1, double ih2, const double* T0, const double* T1,
                            const double* T2, double pin, double pout, double cJ, double* G0,
                            double* G1, double* G2, int summed, cudaStream_t s);
cudaError_t launch_convert(const float* fin, double* dout, const double* din, float* fout,
                           long long n, cudaStream_t s);
template <typename R>
cudaError_t set_smem_attrs();

// Register-resident transforms for line lengths 32..512 (fast_kernels.cu).
// The launch_fwd_x / launch_dct_y / launch_inv_x entry points route to them
// when fast_*_ok holds and the tile argument is 0 (default) or negative:
// axis 0, -1 = blocks of 256 threads, -2 = blocks of 128; axis 1, -1.
bool fast_len(int n);
int fast_threads_per_line(int n);  // P of the split n/2 = P * Q
template <typename R>
bool fast_x_ok(const Geometry& g, const DctPlan<R>& p, const void* a, const void* b,
               const void* c, const void* d);
template <typename R>
bool fast_y_ok(const Geometry& g, const DctPlan<R>& p);
template <typename R, typename V>
cudaError_t launch_fast_fwd_x(const Geometry& g, const DctPlan<R>& p, PcgState* st, V* x,
                              const V* w, const V* q, V* r, const double* rin, R* t,
                              double* partials, int par, double rtol2, int mode,
                              cudaStream_t s, int nt);
template <typename R, typename TZ>
cudaError_t launch_fast_inv_x(const Geometry& g, const DctPlan<R>& p, PcgState* st, const R* t,
                              TZ* z, const double* kd, double kz_host, int check, int mode,
                              cudaStream_t s, typename XOf<TZ>::T* x, int par, int nt);
template <typename R>
cudaError_t launch_fast_y(const Geometry& g, const DctPlan<R>& p, const PcgState* st, R* t,
                          int inverse, int check, cudaStream_t s);
template <typename R>
cudaError_t set_fast_attrs();

// Block-floating-point transforms of the FP64 path for the power-of-two line
// lengths 32..512 (fixed_kernels.cuh): tiles -3 (axis 0, blocks of 256
// threads), -4 (axis 0, blocks of 128) and -3 (axis 1) of launch_fwd_x /
// launch_inv_x / launch_dct_y with R = double, where fx_*_ok holds.
bool fx_len(int n);
int fx_threads_per_line(int n);  // P of their split n/2 = P * Q
int fxp_table_int4(int m);       // int4 entries of their constant table
bool fxp_has_y3(int m);          // a three-stage axis-1 kernel for n = 2 m
bool fx_x_ok(const Geometry& g, const DctPlan<double>& p, const void* a, const void* b,
             const void* c, const void* d);
bool fx_y_ok(const Geometry& g, const DctPlan<double>& p);
cudaError_t launch_fx_fwd_x(const Geometry& g, const DctPlan<double>& p, PcgState* st, double* x,
                            const double* w, const double* q, double* r, const double* rin,
                            double* t, double* partials, int par, double rtol2, int mode,
                            cudaStream_t s, int nt);
cudaError_t launch_fx_inv_x(const Geometry& g, const DctPlan<double>& p, PcgState* st,
                            const double* t, double* z, const double* kd, double kz_host,
                            int check, int mode, cudaStream_t s, int nt);
cudaError_t launch_fx_y(const Geometry& g, const DctPlan<double>& p, const PcgState* st,
                        double* t, int inverse, int check, cudaStream_t s);
// The three-stage axis-1 kernels (n1 = 256, 512, 1024): tile -4 of axis 1.
bool fx_y3_ok(const Geometry& g, const DctPlan<double>& p);
cudaError_t launch_fx_y3(const Geometry& g, const DctPlan<double>& p, const PcgState* st,
                         double* t, int inverse, int check, cudaStream_t s);
cudaError_t set_fx_attrs();

unsigned long long launch_count();

// ---------------------------------------------------------------- batch work queue
// Persistent launches over the solves of one batch class (BatchQueue): the
// queue, the per-solve addresses, the launch slot of the loop-body pass, the
// number of solves of the class (bounds the grid) and the stream.
struct QueueLaunch {
  BatchQueue* q;
  const BatchSolve* bs;
  int slot;
  int nsolves;
  cudaStream_t s;
};

// Blocks of a persistent launch: as many as the SMs hold at once, at most one
// per item.
template <typename K>
unsigned int persistent_grid(K kernel, int threads, size_t smem, long long items) {
  int occ = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) !=
          cudaSuccess || occ < 1)
    occ = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1)
    sms = 148;
  long long g = (long long)sms * occ;
  if (g > items) g = items;
  return (unsigned int)(g < 1 ? 1 : g);
}

// Loop control of a class (init: the initial list before the loop).
cudaError_t launch_queue_control(BatchQueue* q, const BatchSolve* bs,
                                 cudaGraphConditionalHandle handle, int init, cudaStream_t s);
// The iteration's kernels over the class: FP64 matvec (mode 1), double-float
// matvec (mode 1), FP64 tridiagonal solves (mode 1), FP32 tridiagonal solves
// of the flexible PCG (mode 2, r^ in rhat[par], r_old in rhat[par ^ 1]).
cudaError_t launch_q_matvec(const Geometry& g, const QueueLaunch& ql, int par);
cudaError_t launch_q_matvec_df(const Geometry& g, const QueueLaunch& ql, int par);
cudaError_t launch_q_tridiag(const Geometry& g, const QueueLaunch& ql);
cudaError_t launch_q_tridiag_otf(const Geometry& g, const QueueLaunch& ql, const double* lam0,
                                 const double* lam1, int par);
// Register-resident transforms over the class (lengths with fast_len):
// axis-0 forward with the residual update (FP64: x, w, q, r and t64; mixed:
// the double-float q, r and rhat[par]), axis 1 in place (buf 0: t64, 1:
// rhat[par], 2: t32), axis-0 backward with w <- z + beta w (FP64: t64 into w;
// mixed: t32 into wf, with x += alpha w).  nt: 256 or 128 threads (axis 0).
template <typename R>
cudaError_t launch_q_fast_fwd_x(const Geometry& g, const DctTables<R>& tb, const QueueLaunch& ql,
                                int par, int nt);
template <typename R>
cudaError_t launch_q_fast_y(const Geometry& g, const DctTables<R>& tb, const QueueLaunch& ql,
                            int inverse, int buf, int par);
template <typename R>
cudaError_t launch_q_fast_inv_x(const Geometry& g, const DctTables<R>& tb,
                                const QueueLaunch& ql, int par, int nt);

// The block-floating-point transforms over an FP64 class (fx_len lengths):
// axis 0 forward (inverse = 0) or backward (1) with blocks of nt threads, and
// axis 1.
cudaError_t launch_q_fx_x(const Geometry& g, const DctPlan<double>& p, const QueueLaunch& ql,
                          int par, int inverse, int nt);
cudaError_t launch_q_fx_y(const Geometry& g, const DctPlan<double>& p, const QueueLaunch& ql,
                          int inverse);

// Grid sizes of the reduction kernels (to size the partials buffer).
unsigned int matvec_blocks(const Geometry& g);
unsigned int matvec_df_blocks(const Geometry& g);
unsigned int fwd_x_blocks(const Geometry& g, int elem_bytes);
unsigned int tridiag_blocks(const Geometry& g);
// Shared memory of the transform tiles (rows L / columns TI per block).
size_t smem_x_bytes(int n0, int L, int elem_bytes);
size_t smem_y_bytes(int n1, int TI, int elem_bytes);
size_t smem_limit();

}  // namespace etc
