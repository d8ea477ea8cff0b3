/* A plain C99 user of include/lsms.h: the host-only entry points and the create/last_error path,
 * compiled by tests/test_c_abi_cpu.py with gcc -std=c99 -pedantic and linked against liblsms.so.
 * Prints one "name value..." line per result (values with 17 significant digits), which the test
 * compares with the Python binding's. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lsms.h"

static void put(const char* name, const double* v, int n) {
  int i;
  printf("%s", name);
  for (i = 0; i < n; ++i) printf(" %.17g", v[i]);
  printf("\n");
}

int main(void) {
  const double pi = 3.14159265358979323846;
  double k1 = 2.0 * pi, k2 = 3.0 * pi, k3 = 4.0 * pi, kp = 2.4 * pi, radius = 0.25;
  int p = 6, rc, n, i;
  double s[2 * 13], nodes[2 * 256], weights[2 * 256], status[1];
  lsms_contour contour = {256, 0.2, 40.0, 16, 0};
  lsms_ctx* ctx = NULL;
  double centres[6] = {0.0, -1.0, 0.6, -1.0, 0.3, -0.3};
  double ds[2] = {0.7, 2.0};
  double lam[4] = {0.5, -0.1, 2.7, -0.1}, resp[2 * 2 * 12];
  double curve[6 * 64];

  rc = lsms_build_contour(&contour, k1, k2, k3, nodes, weights);
  status[0] = rc;
  put("build_contour_rc", status, 1);
  put("nodes_head", nodes, 8);
  put("weights_tail", weights + 2 * 252, 8);

  rc = lsms_scattering_diagonal(p, k2, kp, radius, s);
  status[0] = rc;
  put("mie_rc", status, 1);
  put("mie", s, 2 * (2 * p + 1));
  rc = lsms_scattering_diagonal_c(p, k2, kp, 0.5, radius, s);
  put("mie_absorbing", s, 2 * (2 * p + 1));
  rc = lsms_pec_scattering_diagonal(p, k2, radius, s);
  put("pec", s, 2 * (2 * p + 1));
  status[0] = lsms_scattering_diagonal_c(p, k2, kp, -0.5, radius, s);     /* Im kp < 0: rejected */
  put("mie_absorbing_bad_rc", status, 1);

  status[0] = lsms_check_geometry(2.0, radius, 3, centres);
  put("geometry_ok", status, 1);
  centres[2] = 0.54;                                                     /* gap below 0.2 R */
  status[0] = lsms_check_geometry(2.0, radius, 3, centres);
  put("geometry_close", status, 1);

  rc = lsms_layer_response(4, (const double[]){1.0, 0.0, 2.5, 0.0, 3.0, 0.0, 1.5, 0.0}, ds, 3, 2, lam, resp);
  status[0] = rc;
  put("layer_response_rc", status, 1);
  put("layer_response", resp, 2 * 2 * 12);

  /* a circle of radius 0.2 as an inclusion: x, y, x', y', x'', y'' at t_j = 2 pi j / 64 */
  n = 64;
  for (i = 0; i < n; ++i) {
    double t = 2.0 * pi * i / n, c = 0.2 * cos(t), sn = 0.2 * sin(t);
    curve[6 * i + 0] = c;
    curve[6 * i + 1] = sn;
    curve[6 * i + 2] = -sn;
    curve[6 * i + 3] = c;
    curve[6 * i + 4] = -c;
    curve[6 * i + 5] = -sn;
  }
  {
    double* m = (double*)malloc(sizeof(double) * 2 * 5 * 5);
    status[0] = lsms_inclusion_scattering_matrix(2, k2, kp, radius, n, curve, m);
    put("inclusion_rc", status, 1);
    put("inclusion", m, 2 * 5 * 5);
    status[0] = lsms_inclusion_scattering_matrix_c(2, k2, kp, 0.5, radius, n, curve, m);
    put("inclusion_absorbing", m, 2 * 5 * 5);
    free(m);
  }

  /* without a GPU, creating a context fails with LSMS_ERR_CUDA and a message */
  rc = lsms_create(k1, k2, k3, 2.0, kp, radius, p, &contour, LSMS_FP64, &ctx);
  status[0] = rc;
  put("create_rc", status, 1);
  printf("create_error %s\n", rc ? lsms_last_error(NULL) : "");
  if (ctx) lsms_destroy(ctx);
  return 0;
}
