/* A plain C consumer of the C ABI in kfbim.h, compiled as C99 and as C++17 and
 * run on the host (no GPU) by test_abi_c.py.  It builds a host-only context
 * for the sphere of radius 0.5 at N = 32 on [-1, 1]^3 and prints, one
 * "key value" pair per line: the sizes, the table sizes, the number of
 * primary flags, the largest distance of a control point from the sphere, the
 * number of Omega cells, the control points per component (kfbim_control_points)
 * with the largest deviation of their normals from the sphere's, the number of
 * jump points (kfbim_jump_points), the status of a solver call on the
 * host-only context and of a setup whose grid size is not a power of two.
 * Exits non-zero when a call that must succeed fails. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "kfbim.h"

/* The sphere of radius *(double*)user about the origin as a CALLBACK level
 * set, with the built-in sphere's arithmetic. */
static double sphere_F(const double x[3], void* user) {
  return sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) - *(const double*)user;
}

static void sphere_derivs(const double x[3], double g[3], double H[9], void* user) {
  const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  int i, j;
  (void)user;
  for (i = 0; i < 3; ++i) g[i] = x[i] / r;
  for (i = 0; i < 3; ++i)
    for (j = 0; j < 3; ++j) H[3 * i + j] = ((i == j) - g[i] * g[j]) / r;
}

static int fail(const char* what, int st) {
  fprintf(stderr, "%s: status %d\n", what, st);
  return 1;
}

int main(void) {
  kfbim_options opt;
  kfbim_geometry geom;
  kfbim_grid grid;
  kfbim_ctx* ctx = NULL;
  int64_t n_points = 0, n_primary = 0, fit_nnz = 0, corr_rows = 0, corr_nnz = 0, i;
  int N = 0, st, st_apply, st_bad, n_cells = 0;
  double* xyz;
  int32_t *comp, *axis, *primary;
  uint8_t* side;
  int64_t n_flagged = 0;
  double dist = 0.0;

  kfbim_default_options(&opt);
  memset(&geom, 0, sizeof geom);
  geom.kind = KFBIM_SPHERE;
  geom.rot[0] = geom.rot[4] = geom.rot[8] = 1.0;
  geom.params[0] = 0.5;
  grid.N = 32;
  grid.lo = -1.0;
  grid.hi = 1.0;

  st = kfbim_setup_host(&geom, &grid, &opt, &ctx);
  if (st != KFBIM_OK || !ctx) return fail("kfbim_setup_host", st);
  st = kfbim_sizes(ctx, &n_points, &n_primary, &N);
  if (st != KFBIM_OK) return fail("kfbim_sizes", st);
  st = kfbim_table_sizes(ctx, &fit_nnz, &corr_rows, &corr_nnz);
  if (st != KFBIM_OK) return fail("kfbim_table_sizes", st);

  xyz = (double*)malloc(sizeof(double) * 3 * (size_t)n_points);
  comp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_points);
  axis = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_points);
  primary = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_points);
  side = (uint8_t*)malloc((size_t)N * N * N);
  if (!xyz || !comp || !axis || !primary || !side) return fail("malloc", -6);
  st = kfbim_points(ctx, xyz, comp, axis, primary);
  if (st != KFBIM_OK) return fail("kfbim_points", st);
  for (i = 0; i < n_points; ++i) {
    const double r = sqrt(xyz[3 * i] * xyz[3 * i] + xyz[3 * i + 1] * xyz[3 * i + 1] +
                          xyz[3 * i + 2] * xyz[3 * i + 2]);
    if (comp[i] < 1 || comp[i] > 3 || axis[i] < 0 || axis[i] > 2) return fail("kfbim_points ranges", -1);
    if (fabs(r - 0.5) > dist) dist = fabs(r - 0.5);
    n_flagged += primary[i] != 0;
  }
  st = kfbim_sides(ctx, 0, side);
  if (st != KFBIM_OK) return fail("kfbim_sides", st);
  for (i = 0; i < (int64_t)N * N * N; ++i) n_cells += side[i] != 0;

  /* the density unknowns per component with their normals, and the jump points */
  {
    int64_t per[3] = {0, 0, 0}, total = 0, nj = 0;
    double ndev = 0.0;
    int c;
    for (c = 1; c <= 3; ++c) {
      double *cx, *cn;
      st = kfbim_control_points(ctx, c, &per[c - 1], NULL, NULL);
      if (st != KFBIM_OK) return fail("kfbim_control_points (count)", st);
      cx = (double*)malloc(sizeof(double) * 3 * (size_t)(per[c - 1] + 1));
      cn = (double*)malloc(sizeof(double) * 3 * (size_t)(per[c - 1] + 1));
      if (!cx || !cn) return fail("malloc", -6);
      st = kfbim_control_points(ctx, c, &per[c - 1], cx, cn);
      if (st != KFBIM_OK) return fail("kfbim_control_points", st);
      for (i = 0; i < per[c - 1]; ++i) {
        int a;
        for (a = 0; a < 3; ++a) {
          const double dv = fabs(cn[3 * i + a] - cx[3 * i + a] / 0.5);
          if (dv > ndev) ndev = dv;
        }
      }
      total += per[c - 1];
      free(cx);
      free(cn);
    }
    st = kfbim_jump_points(ctx, &nj, NULL);
    if (st != KFBIM_OK) return fail("kfbim_jump_points", st);
    printf("control_points_total %lld\ncontrol_points_1 %lld\nnormal_deviation %.3e\njump_points %lld\n",
           (long long)total, (long long)per[0], ndev, (long long)nj);
    if (kfbim_control_points(ctx, 4, &nj, NULL, NULL) != KFBIM_E_INVALID) return fail("kfbim_control_points(4)", 0);
  }

  /* a solver call on a host-only context is refused, with a message */
  st_apply = kfbim_apply(ctx, NULL, NULL, NULL);
  if (!kfbim_last_error(ctx) || !kfbim_last_error(ctx)[0]) return fail("kfbim_last_error", st_apply);
  st = kfbim_destroy(ctx);
  if (st != KFBIM_OK) return fail("kfbim_destroy", st);

  /* the same sphere through the CALLBACK kind: identical sizes and points */
  {
    kfbim_geometry cb;
    kfbim_ctx* cctx = NULL;
    double radius = 0.5;
    int64_t cn = 0, cprim = 0;
    double* cxyz;
    memset(&cb, 0, sizeof cb);
    cb.kind = KFBIM_CALLBACK;
    cb.F = sphere_F;
    cb.derivs = sphere_derivs;
    cb.user = &radius;
    st = kfbim_setup_host(&cb, &grid, &opt, &cctx);
    if (st != KFBIM_OK || !cctx) return fail("kfbim_setup_host (callback)", st);
    st = kfbim_sizes(cctx, &cn, &cprim, NULL);
    if (st != KFBIM_OK) return fail("kfbim_sizes (callback)", st);
    cxyz = (double*)malloc(sizeof(double) * 3 * (size_t)cn);
    if (!cxyz) return fail("malloc", -6);
    st = kfbim_points(cctx, cxyz, NULL, NULL, NULL);
    if (st != KFBIM_OK) return fail("kfbim_points (callback)", st);
    printf("callback_equal %d\n",
           cn == n_points && cprim == n_primary && memcmp(cxyz, xyz, sizeof(double) * 3 * (size_t)cn) == 0);
    free(cxyz);
    kfbim_destroy(cctx);
  }

  /* N = 24 is not a power of two: refused, *ctx set to NULL */
  grid.N = 24;
  ctx = (kfbim_ctx*)&grid;
  st_bad = kfbim_setup_host(&geom, &grid, &opt, &ctx);
  if (ctx != NULL) return fail("kfbim_setup_host left *ctx set", st_bad);

  printf("n_points %lld\nn_primary %lld\nN %d\n", (long long)n_points, (long long)n_primary, N);
  printf("options_size %d\nrelax %.17g\n", (int)sizeof(kfbim_options), opt.relax);
  printf("fit_nnz %lld\ncorr_rows %lld\ncorr_nnz %lld\n", (long long)fit_nnz, (long long)corr_rows,
         (long long)corr_nnz);
  printf("primary_flags %lld\nmax_distance %.3e\nomega_cells %d\n", (long long)n_flagged, dist, n_cells);
  printf("status_apply %d\nstatus_bad_grid %d\n", st_apply, st_bad);
  free(xyz);
  free(comp);
  free(axis);
  free(primary);
  free(side);
  return 0;
}
