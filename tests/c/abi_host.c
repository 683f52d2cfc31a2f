/* C99 client of include/pc.h: compiles as plain C against the header, links
 * libpc.so and calls the entry points that need no GPU (pc_default_options,
 * pc_estimate_bytes, pc_check_domain, pc_create's error return).  Prints one
 * line per check and exits non-zero on the first failure. */
#include <stdio.h>
#include <stdlib.h>

#include "pc.h"

static int fail(const char *what) {
  fprintf(stderr, "FAIL %s\n", what);
  return 1;
}

int main(void) {
  pc_options o;
  pc_default_options(&o);
  if (o.precision != PC_PREC_MIXED || o.exec != PC_EXEC_PERSISTENT || o.polish != -1) return fail("defaults");
  printf("defaults precision=%d exec=%d kappa=%g polish_tol=%g\n", o.precision, o.exec, o.filter_kappa, o.polish_tol);

  const int32_t widths[4] = {3, 64, 64, 1};
  const int64_t est = pc_estimate_bytes(3, widths);
  if (est <= 0) return fail("estimate");
  printf("estimate %lld bytes\n", (long long)est);
  if (pc_estimate_bytes(0, widths) != -1) return fail("estimate of a bad network");

  /* the triangle {x >= -1, y >= -1, x + y <= 0} with its 3 vertices and 3 edges */
  const double A[6] = {-1, 0, 0, -1, 1, 1};
  const double c[3] = {1, 1, 0};
  const double X0[6] = {-1, -1, 1, -1, -1, 1};
  const int32_t E0[6] = {0, 1, 0, 2, 1, 2};
  if (pc_check_domain(2, 3, A, c, 3, X0, 3, E0) != PC_OK) return fail("triangle");
  const double Xout[6] = {-1, -1, 1.5, -1, -1, 1}; /* vertex 1 outside x + y <= 0 */
  if (pc_check_domain(2, 3, A, c, 3, Xout, 3, E0) != PC_ERR_INVALID) return fail("vertex outside");
  printf("domain checks ok\n");

  if (pc_create(NULL, 0, &o) != PC_ERR_INVALID) return fail("pc_create(NULL)");
  printf("ok\n");
  return 0;
}
