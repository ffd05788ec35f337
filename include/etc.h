/*
 * libetc -- effective thermal conductivity of a voxel RVE on one B300 GPU.
 *
 * C ABI of the hot path of Ye, Fu & Chung, "A fast cosine transformation
 * accelerated method for predicting effective thermal conductivity"
 * (arXiv 2404.02433):
 *   - the problem (Sec. 2.1): -div(K grad p) = 0 on an Lx x Ly x Lz box with an
 *     orthotropic diagonal K = diag(kx, ky, kz) > 0 per voxel, p = p_in on one
 *     face, p = p_out on the opposite face, zero flux on the other four;
 *   - its TPFA discretisation (Sec. 2.2, Eq. scaled bilinear forms): one unknown
 *     per voxel, harmonic-mean face conductances, half-cell Dirichlet faces;
 *   - PCG (Algorithm 1) preconditioned by the homogeneous reference operator
 *     (Eq. refer bilinear forms), whose parameters come from the linear
 *     programme of Algorithm 2 and which is inverted by 2-D cosine transforms
 *     plus tridiagonal solves (Algorithm 3);
 *   - the effective conductivity from the outflow (Eq. effective formula dis).
 *
 * Conventions common to every entry point:
 *   - Voxel arrays are dense float64 in C order [nz][ny][nx] (x fastest), the
 *     index set I_h of Sec. 2.2.  Pointers may be device, pinned-host or
 *     pageable-host memory (the library copies with cudaMemcpyDefault).
 *   - dir is the loading direction: 0 = x, 1 = y, 2 = z.  Internally the medium
 *     is permuted so that the loading axis is the slowest ("loading frame"):
 *     dir z keeps (x, y, z); dir y uses (x, z, y); dir x uses (y, z, x), listed
 *     fastest to slowest.  Component entry points marked "loading frame" take
 *     and return arrays in that permuted layout, [n2][n1][n0].
 *   - Every function returns an etc_status, never throws and never exits.
 *     Arguments are validated on the host before any GPU work; a rejected call
 *     returns ETC_EINVAL and changes nothing.  After ETC_ECUDA the handle should
 *     be destroyed.  etc_last_error(handle) gives a one-line reason;
 *     etc_last_error(NULL) gives the reason for the calling thread's last call
 *     of etc_create_rve, etc_batch_create or etc_apply_reference_inverse_static
 *     ("" if it succeeded).
 *   - Test hooks read at etc_create_rve from the environment (both unset in
 *     use): ETC_FAIL_ALLOC_AFTER=k fails the handle's (k+1)-th device allocation
 *     (ETC_ENOMEM, clean teardown); ETC_TEST_TMA_TX_EXTRA=b makes the
 *     bulk-tensor matvec's waits expect b bytes that no copy delivers, so they
 *     run out and the mixed solve ends with ETC_ECUDA, without any fault.
 *     ETC_FORCE_TILES="fx,ix,y" (read whenever the transform tiles are chosen)
 *     replaces the tuned tiles by these candidates: rows per block of the
 *     axis-0 forward and backward transforms (1..64, or -1 / -2 for the
 *     register-resident kernels in blocks of 256 / 128 threads, or, FP64
 *     only, -3 / -4 for the block-floating-point kernels in blocks of 256 /
 *     128 threads) and columns per block of the axis-1 transforms (1..32, or
 *     -1, or, FP64 only, -3, or -4 for the three-stage kernels of lengths
 *     256, 512, 1024); a candidate the shape or precision does not
 *     allow gives ETC_EINVAL.  It lets a test run every kernel the tuner may
 *     pick.
 *   - A handle is used from one host thread at a time.  All its GPU work is
 *     ordered on the stream given to etc_create_rve; calls that return numbers
 *     to the host synchronise that stream before returning.
 */
#ifndef ETC_H
#define ETC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct etc_rve etc_rve;
typedef int etc_status;

enum {
  ETC_OK = 0,
  ETC_EINVAL = 1,      /* bad argument (size, length, kappa, p_in == p_out, dir) */
  ETC_ENOMEM = 2,      /* device or pinned-host allocation failed */
  ETC_ECUDA = 3,       /* a CUDA runtime call failed, or a bounded device wait for
                          bulk-tensor copies ran out (0.5 s; the solve stops) */
  ETC_ENOCONV = 4,     /* maxit reached; results hold the last iterate */
  ETC_EBREAKDOWN = 5,  /* non-finite or non-positive PCG scalar */
  ETC_ESTATE = 6       /* call out of order (e.g. solution of an unsolved dir) */
};

/* Arithmetic of a solve.  The mixed forms run Algorithm 3 in FP32 inside a
 * flexible (Polak-Ribiere) PCG; their scalars and reductions are FP64. */
enum {
  ETC_PREC_FP64 = 0,      /* everything in FP64: plain PCG (Algorithm 1) */
  ETC_PREC_MIXED = 1,     /* x, r, q and the operator in double-float (pairs of
                             FP32 values, 48-bit significand) on the FP32 pipe; the
                             search direction w in FP32 */
  ETC_PREC_MIXED_F64 = 2  /* x, r, w, q and the operator in FP64 */
};

/* How the five reference parameters of Eq. (refer bilinear forms) are chosen. */
enum {
  ETC_REF_LP = 0,      /* optimum of the LP of Algorithm 2 (centred optimal point) */
  ETC_REF_ONES = 1,    /* all equal to 1 (the paper's "one" setting, Sec. 4.4) */
  ETC_REF_USER = 2     /* values given to etc_set_reference_params */
};

/* Initial guess of PCG (Algorithm 1 leaves it open). */
enum {
  ETC_INIT_ZERO = 0,   /* x0 = 0 (r0 = b) */
  ETC_INIT_LINEAR = 1  /* x0 = p_in + (p_out - p_in) (k + 1/2) / n along the loading axis:
                          the exact TPFA solution of a homogeneous medium; costs one
                          product with A.  Solves with per-face data or a source
                          (etc_solve_general) start from 0. */
};

/* Options of a solve.  Fill with etc_default_opts before setting fields
 * (fields may be added at the end). */
typedef struct {
  double rtol;         /* exit when ||r||_2 <= rtol ||b||_2 (Eq. exit); default 1e-8 */
  int maxit;           /* iteration cap; default 5000 */
  int precision;       /* ETC_PREC_*; default ETC_PREC_FP64 */
  int true_residual;   /* 1: also compute ||b - A p|| / ||b|| at exit; default 1 */
  int batch_queue;     /* etc_batch_create only: 1 = work-queue loops per class of
                          equal sizes (persistent kernels), 0 = a device-driven loop
                          per solve; default 0 (see etc_batch_create) */
  int init;            /* ETC_INIT_ZERO (default) or ETC_INIT_LINEAR; a guess that
                          already meets the exit test ends with 0 iterations */
} etc_opts;

typedef struct {
  int iters;           /* PCG iterations (products with A after the initial residual) */
  int status;          /* ETC_OK, ETC_ENOCONV or ETC_EBREAKDOWN */
  double relres;       /* ||r|| / ||b|| of the recursively updated residual */
  double true_relres;  /* ||b - A p|| / ||b||, or -1 if not computed */
  double kref[5];      /* reference parameters used: x, y, z, in, out of the
                          loading frame, in units of kappa / h^2 (Sec. 2.2) */
  double cond_bound;   /* Lambda''/Lambda' of Lemma 3.1 for kref */
  double kappa_in;     /* effective conductivity from the inflow face */
  double column[3];    /* K[:, dir] in physical axes x, y, z (see etc_effective_tensor) */
  double t_setup_ms;   /* faces, LP, pivot tables */
  double t_solve_ms;   /* PCG loop and post-processing */
  double kappa_energy; /* effective conductivity from the energy of the solution,
                          L h E / (n0 n1 (p_in - p_out)^2) with E = p.Ap - 2 b.p +
                          sum B_in p_in^2 + sum B_out p_out^2 summed as its positive
                          face terms; equal to kappa_eff at the exact solution, with
                          an error quadratic in the solve error; -1 unless the true
                          residual is computed (opts->true_residual) */
} etc_info;

/* Fill *opts with the defaults listed in etc_opts. */
etc_status etc_default_opts(etc_opts* opts);

/*
 * Create an RVE handle: copies the voxel conductivities (Sec. 2.2, arrays
 * kappa^x, kappa^y, kappa^z on I_h) and allocates every device buffer the
 * solve needs (about 14 doubles per voxel).
 *   nx, ny, nz  >= 1 voxels per axis; lx, ly, lz > 0 box lengths (h = L / N).
 *   kx          nx*ny*nz doubles; ky, kz the same, or NULL / equal to kx for an
 *               isotropic medium (one array is then stored).  Every value must
 *               be finite and > 0 (Sec. 2.1), else ETC_EINVAL.  The caller keeps
 *               ownership; the arrays may be freed once this call returns.
 *   stream      cudaStream_t to order all work of the handle (NULL = legacy).
 *   out         receives the handle; unchanged on error.
 */
etc_status etc_create_rve(int nx, int ny, int nz, double lx, double ly, double lz,
                          const double* kx, const double* ky, const double* kz,
                          void* stream, etc_rve** out);

/* Release every resource of the handle (NULL is accepted). */
etc_status etc_destroy_rve(etc_rve* rve);

/*
 * Choose how kappa_ref is set for loading direction dir (Algorithm 2).
 *   mode     ETC_REF_LP (default), ETC_REF_ONES or ETC_REF_USER.
 *   kref_in  5 positive values (x, y, z, in, out of the loading frame, units of
 *            kappa / h^2), read for ETC_REF_USER only.
 *   kref_out if not NULL, receives the parameters that the next solve of dir
 *            will use (this runs the face assembly of dir on the GPU).
 */
etc_status etc_set_reference_params(etc_rve* rve, int dir, int mode, const double* kref_in,
                                    double* kref_out);

/*
 * Solve the TPFA system for loading direction dir with p = p_in on the low face
 * and p_out on the high face of that axis (Sec. 2.1), by PCG from the initial
 * guess opts->init (default 0), and return the effective conductivity
 * kappa_eff (Eq. effective formula dis,
 * outflow side).  opts may be NULL (defaults).  info may be NULL.
 * p_in == p_out is rejected (Sec. 2.1).  ETC_ENOCONV still fills kappa_eff and
 * info from the last iterate.
 */
etc_status etc_solve_direction(etc_rve* rve, int dir, double p_in, double p_out,
                               const etc_opts* opts, double* kappa_eff, etc_info* info);

/*
 * Solve -div(K grad p) = source with p = p_in_face on the low face and
 * p_out_face on the high face of loading direction dir, zero flux elsewhere
 * (Sec. 4.1, the data of the smooth test of Table 2).  Face values follow Eq.
 * (flux) face by face; the source enters the second equation of the mixed
 * system with one value per voxel (taken at the voxel centre by the caller).
 *   p_in_face, p_out_face  n0*n1 doubles each in the loading-frame plane layout
 *                          [n1][n0] (see etc_loading_dims), or NULL for zero;
 *   source                 nx*ny*nz doubles, ORIGINAL layout, or NULL for zero;
 *                          pointers may be device or host memory.
 * At least one of the three must be given.  The solution is read with
 * etc_get_solution(dir); info (may be NULL) carries iterations and residuals,
 * its kappa fields are 0 (the ETC needs constant face data).
 */
etc_status etc_solve_general(etc_rve* rve, int dir, const double* p_in_face,
                             const double* p_out_face, const double* source,
                             const etc_opts* opts, etc_info* info);

/* Copy the solution p of the last solve of dir into dst (nx*ny*nz doubles, the
 * ORIGINAL [nz][ny][nx] layout, device or host memory).  ETC_ESTATE if dir has
 * not been solved. */
etc_status etc_get_solution(etc_rve* rve, int dir, double* dst);

/*
 * Three solves (dir = x, y, z, p_in = 1, p_out = 0) giving the 3x3 tensor
 * K[a*3 + b] = L^b <v_a> / (p_in - p_out) under load b, where <v_a> is the
 * volume average of the cell-averaged a-face fluxes of Eq. (flux) (Neumann faces
 * carry zero flux).  The diagonal is the outflow formula of Eq. (effective
 * formula dis).  The off-diagonal entries are this library's definition: the
 * paper defers the full tensor to a citation (Sec. 2.1).  info may be NULL,
 * else receives 3 records.
 */
etc_status etc_effective_tensor(etc_rve* rve, const etc_opts* opts, double* K,
                                etc_info* info);

/*
 * Adjoint gradient of kappa_eff (Eq. effective formula dis, loading direction
 * dir, Dirichlet data p_in, p_out) with respect to the logarithm of every voxel
 * conductivity -- not in the paper; derived from its Sec. 2.2 discretisation.
 * Runs the forward solve, one adjoint solve of the same operator (A symmetric;
 * right-hand side dJ/dp = c b_out on the outflow plane, i.e. Dirichlet data
 * (0, c) with c = L h / (n0 n1 (p_in - p_out))) and one gradient pass using the
 * face derivatives dT/dlog kappa_a = T kappa~_b / (kappa~_a + kappa~_b).
 *   per_component 0: grad has nx*ny*nz doubles, sum over the three components
 *                    (the derivative for an isotropic medium kappa = exp(theta));
 *                 1: grad has 3*nx*ny*nz doubles: components x, y, z in turn.
 *   grad         ORIGINAL [nz][ny][nx] layout, device or host memory.
 *   kappa_eff    receives the forward value (may be NULL).
 *   info         NULL or 2 records: forward solve, adjoint solve.
 * The solution of dir is kept as after etc_solve_direction.
 */
etc_status etc_gradient(etc_rve* rve, int dir, double p_in, double p_out, const etc_opts* opts,
                        int per_component, double* grad, double* kappa_eff, etc_info* info);

/*
 * Batches: the full tensors of many RVEs in one CUDA graph (the three loading
 * directions of Sec. 2.1 for every RVE, p_in = 1, p_out = 0).
 * By default (opts->batch_queue == 0) every handle gets a branch that runs
 * its three directions in turn, each as a device-driven solve: face
 * assembly, LP optimum and pivots on the device, the initial apply, a graph
 * WHILE node whose body runs two PCG iterations and ends the loop once the
 * device `done` flag is set (or after maxit/2 + 4 passes), then the flux
 * sums.  Branches of different handles run concurrently.
 * With opts->batch_queue == 1 the handles are grouped into classes of equal
 * sizes.  A class whose loading frames all have register-resident transform
 * lengths (32, 64, 96, 128, 160, 192, 256, 384, 512, 1024 on axes 0 and 1),
 * in FP64 or ETC_PREC_MIXED, runs per direction: every member's start in
 * parallel branches, then ONE graph WHILE loop for the whole class whose body
 * runs two PCG iterations of every member still iterating -- each kernel of
 * the iteration one persistent launch whose blocks take (solve, block) items
 * from a device work queue, finished solves dropped from the queue by the
 * loop control -- and ends when no member is left (or each after maxit/2 + 4
 * passes), then every member's flux sums.  Other handles get per-solve
 * branches.  (Measured on B300 the per-solve branches are faster: see the
 * design notes.)  The handles must be distinct, must outlive the batch, and
 * must not be used by other calls while a run is in progress; their
 * reference modes are read at creation.
 *   etc_batch_run launches the graph, waits, and fills K (count * 9 doubles,
 *   handle i's tensor at K + 9 i, layout as etc_effective_tensor) and, if not
 *   NULL, info (count * 3 records; t_solve_ms is the whole batch) and ms (the
 *   batch time).  Returns the first non-OK solve status, else ETC_OK.
 */
typedef struct etc_batch etc_batch;
etc_status etc_batch_create(int count, etc_rve* const* rves, const etc_opts* opts,
                            etc_batch** out);
etc_status etc_batch_run(etc_batch* batch, double* K, etc_info* info, double* ms);
etc_status etc_batch_destroy(etc_batch* batch);
/* Number of the batch's handles whose solves run in work-queue loops (0 for
 * NULL). */
int etc_batch_queued(const etc_batch* batch);
/* create + run + destroy. */
etc_status etc_effective_tensor_batch(int count, etc_rve* const* rves, const etc_opts* opts,
                                      double* K, etc_info* info);

/*
 * Convergence history of the last solve on the handle (any direction or
 * call): the relative residual ||r_i||_2 / ||b||_2 of Eq. (exit) after
 * iteration i, i = 0 (the initial residual, 1) .. iters, as the paper plots
 * it (Sec. 4.2).  The residual-update kernel writes ||r_i||^2 into a device
 * ring of the last 8192 iterations; this call copies the last min(cap,
 * iters + 1, 8192) values into out (host memory, cap doubles), sets *first to
 * the iteration of out[0] and *count to the number written.  Synchronises the
 * handle's stream.  ETC_ESTATE if no solve has run.
 */
etc_status etc_residual_history(etc_rve* rve, double* out, int cap, int* first, int* count);

/* Loading-frame sizes (n0, n1, n2) of direction dir. */
etc_status etc_loading_dims(const etc_rve* rve, int dir, int* dims3);

/*
 * Component entry points (loading frame of dir, device pointers, n0*n1*n2
 * doubles each, in/out must not overlap).  They run the same kernels as the
 * solve and exist so that each kernel can be checked on its own.
 */

/* q = A w: the TPFA operator of Eq. (scaled bilinear forms) for direction dir. */
etc_status etc_apply_operator(etc_rve* rve, int dir, const double* w, double* q);

/* q = A w by the double-float operator of the mixed path (ETC_PREC_MIXED): w
 * is FP32 (n0*n1*n2 floats, the search direction's storage there), q is
 * returned as the FP64 value of each double-float pair (hi + lo, exact), and,
 * if wq is not NULL, *wq = w.q as that kernel's reduction forms it (the
 * denominator of alpha in Algorithm 1).  It runs the kernel a mixed solve of
 * dir runs (the bulk-tensor form where n0 is a multiple of 4).  Uses the
 * handle's work buffers; synchronises the handle's stream. */
etc_status etc_apply_operator_df(etc_rve* rve, int dir, const float* w, double* q, double* wq);

/* z = A_ref^{-1} r by Algorithm 3 with the kref that the next solve of dir uses;
 * precision = ETC_PREC_FP64, or one of the mixed forms (FP32 transforms and
 * solves: the kernels of the flexible PCG's initial apply, including the
 * bulk-tensor tridiagonal solves where the plane is a multiple of 4).  The
 * transform tiles are those a solve of dir in that precision uses. */
etc_status etc_apply_preconditioner(etc_rve* rve, int dir, int precision, const double* r,
                                    double* z);

/* Per plane k, the 2-D transform over axes 0 and 1 of the loading frame:
 * inverse == 0 applies Eq. (forward DCT) along both axes, inverse == 1 applies
 * Eq. (backward DCT) along both axes (FP64, with the tiles of an FP64 solve). */
etc_status etc_dct_planes(etc_rve* rve, int dir, int inverse, const double* in, double* out);

/*
 * Measurement support.  etc_profile_iteration runs the initial preconditioner
 * apply of dir and then `iters` PCG iterations with a CUDA event between
 * consecutive kernels on the handle's stream, and writes the mean time in ms
 * of each kernel of the iteration to ms[0..5]: matvec, forward DCT axis 0 (with
 * the x/r update), forward DCT axis 1, tridiagonal solves, backward DCT axis 1,
 * backward DCT axis 0.  It leaves dir marked unsolved.
 */
etc_status etc_profile_iteration(etc_rve* rve, int dir, int precision, int iters, double* ms);

/*
 * The transform kernels a solve of dir in `precision` uses, as chosen by the
 * tile autotuner (or forced by ETC_FORCE_TILES): tiles[0] the axis-0 forward
 * pass, tiles[1] the axis-0 backward pass, tiles[2] the axis-1 passes.
 * Values: L > 0 rows (axis 0) or columns (axis 1) per block of the generic
 * kernels; -1/-2 the register-resident floating-point kernels (axis-0 blocks
 * of 256/128 threads); -3/-4 the FP64 path's block-floating-point kernels
 * (integer arithmetic, axis-0 blocks of 256/128 threads; on axis 1, -3 the
 * two-stage and -4 the three-stage kernels); 0 the
 * default of the generic kernels (no autotuning).  tiles: host array of 3 ints
 * written on ETC_OK.  May run the autotuner (timed launches on the handle's
 * stream) when dir/precision has no recorded choice yet in the process.
 */
etc_status etc_transform_tiles(etc_rve* rve, int dir, int precision, int* tiles);

/* Test support: the integer-pipe conversions the mixed path uses, element-wise
 * on device arrays of n values: d_out = (double) f_in exactly, f_out = f_in
 * rounded to nearest even.  Synchronises the stream. */
etc_status etc_convert_check(const float* f_in, double* d_out, const double* d_in, float* f_out,
                             long long n, void* stream);

/* Test support: the double-float split the mixed-precision matvec uses
 * (Algorithm 1's A w on the FP32 pipe), element-wise on n device values d:
 * hilo[2i] = hi = d rounded to binary32 (nearest even), hilo[2i+1] = lo = d - hi
 * rounded to binary32; lo = 0 when |d| < 2^-74, for binary64 subnormals, and
 * where hi is infinite or NaN.  hilo: 2n floats, 8-byte aligned.  Synchronises
 * the stream. */
etc_status etc_split_check(const double* d, float* hilo, long long n, void* stream);

/* Kernels launched by this library since the process started (all handles). */
unsigned long long etc_kernel_launches(void);

/* Measurement support (not in the paper): the FP64 fused multiply-add rate of
 * the current device on the clock it runs at, in TFLOP/s (an FMA counts 2).
 * 148 x 8 blocks of 256 threads each keep eight independent FMA chains for
 * `iters` steps; one warm-up launch, then one launch timed with CUDA events on
 * `stream`.  This is the measured peak the FP64 kernels' roofline fractions
 * are quoted against, next to the figure derived from unit counts and the
 * maximum clock.  Synchronises the stream; ETC_EINVAL for iters < 1 or a NULL
 * tflops. */
etc_status etc_fp64_fma_rate(int iters, double* tflops, void* stream);

/*
 * z = A_ref^{-1} r without allocating anything (the paper has no counterpart;
 * it is a service for callers that cannot allocate device memory: those whose
 * GPU memory is owned by another allocator -- a framework pool that reserves
 * the device, an embedding application with its own memory budget -- and those
 * that cannot accept the device synchronisation cudaFree may cause).
 * Same operation as etc_apply_preconditioner in FP64, but without a handle:
 *   n0, n1, n2  loading-frame sizes, r and z in that layout ([n2][n1][n0]);
 *               limits: n0, n1 <= 2048 and n0*n1*n2 <= 2^20 cells, else
 *               ETC_EINVAL, with the limits in etc_last_error(NULL).
 *   kref        5 reference parameters (x, y, z, in, out; finite, > 0), host.
 *   r, z        device pointers, n0*n1*n2 doubles each, not overlapping.
 *   stream      cudaStream_t the work is queued on; the call does not wait.
 * Working memory is a fixed __device__ array of about 16.3 MiB inside the
 * library, held by every GPU that loads it until the process exits.  No
 * cudaMalloc, cudaFree or allocating library routine is called.  The first
 * call on each device looks up that array's device address (and sets kernel
 * attributes) with the device current; make that first call before any stream
 * capture.  The address and attributes are kept for the life of the process:
 * resetting a device (cudaDeviceReset) after its first call is not supported.
 * ETC_ECUDA names the failed step and the CUDA error in etc_last_error(NULL).  All calls share the array and it keeps the last call's contents
 * (each call writes every element it reads), so calls that overlap on the GPU
 * -- on different streams, or from different host threads -- race.
 */
etc_status etc_apply_reference_inverse_static(int n0, int n1, int n2, const double* kref,
                                              const double* r, double* z, void* stream);

const char* etc_status_string(etc_status status);
const char* etc_last_error(const etc_rve* rve);

#ifdef __cplusplus
}
#endif

#endif /* ETC_H */
