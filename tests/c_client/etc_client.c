/*
 * A plain C99 caller of libetc (include/etc.h): no CUDA headers, no Python.
 *
 * Without arguments it runs the host-side checks that need no GPU: default
 * options, argument validation before any GPU work, status strings.  With
 * --gpu it also solves a homogeneous orthotropic medium from host arrays
 * (the library copies with cudaMemcpyDefault).  There the reference operator
 * equals the TPFA operator, so PCG converges in one iteration, and the exact
 * TPFA solution is linear: the effective tensor is diag(kx, ky, kz) and the
 * middle voxel of each loading line holds the mean of p_in and p_out.
 * Exit status 0 on success, otherwise the number of the failed check.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "etc.h"

static int close_rel(double a, double b, double tol) { return fabs(a - b) <= tol * fabs(b); }

static int host_checks(void) {
  etc_opts o;
  etc_rve* h = NULL;
  double one = 1.0, k = 0.0;
  if (etc_default_opts(&o) != ETC_OK || o.maxit != 5000 || o.rtol != 1e-8) return 10;
  if (etc_default_opts(NULL) != ETC_EINVAL) return 11;
  if (etc_create_rve(0, 4, 4, 1.0, 1.0, 1.0, &one, NULL, NULL, NULL, &h) != ETC_EINVAL || h)
    return 12;
  if (etc_create_rve(4, 4, 4, 1.0, -1.0, 1.0, &one, NULL, NULL, NULL, &h) != ETC_EINVAL || h)
    return 13;
  if (etc_create_rve(4, 4, 4, 1.0, 1.0, 1.0, NULL, NULL, NULL, NULL, &h) != ETC_EINVAL) return 14;
  if (etc_solve_direction(NULL, 0, 1.0, 0.0, NULL, &k, NULL) != ETC_EINVAL) return 15;
  if (etc_destroy_rve(NULL) != ETC_OK) return 16;
  if (strcmp(etc_status_string(ETC_OK), "ok") != 0) return 17;
  return 0;
}

static int gpu_checks(void) {
  const int nx = 12, ny = 10, nz = 14;
  const size_t n = (size_t)nx * ny * nz;
  const double comp[3] = {2.0, 3.5, 0.7};
  double* kap[3];
  double K[9];
  etc_info info[3];
  etc_opts o;
  etc_rve* h = NULL;
  int rc = 0;
  for (int a = 0; a < 3; ++a) {
    kap[a] = malloc(n * sizeof(double));
    if (!kap[a]) return 20;
    for (size_t c = 0; c < n; ++c) kap[a][c] = comp[a];
  }
  etc_default_opts(&o);
  o.rtol = 1e-12;
  if (etc_create_rve(nx, ny, nz, 1.0, 1.0, 1.0, kap[0], kap[1], kap[2], NULL, &h) != ETC_OK) {
    rc = 21;
    goto done;
  }
  if (etc_effective_tensor(h, &o, K, info) != ETC_OK) { rc = 22; goto done; }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      if (a == b && !close_rel(K[3 * a + b], comp[a], 1e-12)) { rc = 23; goto done; }
      if (a != b && fabs(K[3 * a + b]) > 1e-12) { rc = 24; goto done; }
    }
  for (int b = 0; b < 3; ++b)
    if (info[b].iters != 1 || info[b].status != ETC_OK) { rc = 25; goto done; }
  {
    /* load along z, p_in = 3, p_out = 1: p is linear in k, so the mean of the
       two middle planes (nz even) is 2 */
    double kz = 0.0;
    double* p = malloc(n * sizeof(double));
    if (!p) { rc = 26; goto done; }
    if (etc_solve_direction(h, 2, 3.0, 1.0, &o, &kz, NULL) != ETC_OK ||
        etc_get_solution(h, 2, p) != ETC_OK) {
      free(p);
      rc = 27;
      goto done;
    }
    const size_t plane = (size_t)nx * ny, i = 5, j = 4;
    const double mid = 0.5 * (p[(nz / 2 - 1) * plane + j * nx + i] + p[(nz / 2) * plane + j * nx + i]);
    free(p);
    if (!close_rel(kz, comp[2], 1e-12) || fabs(mid - 2.0) > 1e-12) { rc = 28; goto done; }
  }
  {
    double km = 0.0;
    o.precision = ETC_PREC_MIXED;
    o.rtol = 1e-8;
    if (etc_solve_direction(h, 0, 1.0, 0.0, &o, &km, NULL) != ETC_OK ||
        !close_rel(km, comp[0], 1e-7)) {
      rc = 29;
      goto done;
    }
  }
done:
  if (rc && h) fprintf(stderr, "libetc: %s\n", etc_last_error(h));
  etc_destroy_rve(h);
  for (int a = 0; a < 3; ++a) free(kap[a]);
  return rc;
}

int main(int argc, char** argv) {
  int rc = host_checks();
  if (rc == 0 && argc > 1 && strcmp(argv[1], "--gpu") == 0) rc = gpu_checks();
  printf(rc ? "etc_client: check %d failed\n" : "etc_client: ok\n", rc);
  return rc;
}
