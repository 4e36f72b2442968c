/* Plain-C client of the library's ABI (no C++, no torch): the header compiles
 * as C11, and the entry points that need no GPU behave as include/ok.h says.
 * Prints "ok" and returns 0 on success, else the number of the failed check. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "ok.h"

#define CHECK(n, cond)                                  \
  do {                                                  \
    if (!(cond)) {                                      \
      fprintf(stderr, "check %d failed: %s\n", n, #cond); \
      return n;                                         \
    }                                                   \
  } while (0)

int main(void) {
  ok_opts o;
  ok_default_opts(&o);
  CHECK(1, o.restart == 30 && o.q_A == 10 && o.n_V == 5 && o.precision == OK_FP64);
  CHECK(2, sizeof(ok_opts) == 96 && sizeof(ok_params) == 40);
  CHECK(3, strncmp(ok_version(), "ok-gb300", 8) == 0);

  /* host-side validation: rejected before any device work */
  ok_params p = {0.04, 100.0, 0.0, 1.0, 1e-4};
  ok_grid* g = (ok_grid*)1;
  CHECK(4, ok_grid_create(4, 8, &p, &o, &g) == OK_ERR_INVALID_ARG && g == NULL);
  CHECK(5, strstr(ok_last_error(), "dim") != NULL);
  CHECK(6, ok_grid_create(2, 8, &p, &o, NULL) == OK_ERR_INVALID_ARG);

  /* eigenvalues of [[2, 3], [1, 4]] are 1 and 5; of [[0, -1], [1, 0]] are +-i */
  double H[4] = {2.0, 1.0, 3.0, 4.0}; /* column-major */
  double re[2], im[2];
  CHECK(7, ok_hessenberg_eigenvalues(2, H, 2, re, im) == OK_SUCCESS);
  double lo = re[0] < re[1] ? re[0] : re[1], hi = re[0] < re[1] ? re[1] : re[0];
  CHECK(8, fabs(lo - 1.0) < 1e-14 && fabs(hi - 5.0) < 1e-14 && im[0] == 0.0 && im[1] == 0.0);
  double R[4] = {0.0, 1.0, -1.0, 0.0};
  CHECK(9, ok_hessenberg_eigenvalues(2, R, 2, re, im) == OK_SUCCESS);
  CHECK(10, re[0] == 0.0 && re[1] == 0.0 && fabs(fabs(im[0]) - 1.0) < 1e-15 && im[0] == -im[1]);

  /* Givens restoration: one column (a, b) reduced to (r, 0) by c = a/r, s = b/r */
  double a = 3.0, b = 4.0, r = 5.0, c = a / r, s = b / r;
  double col[2] = {r, 0.0};
  CHECK(11, ok_givens_unrotate(1, col, 2, &c, &s) == OK_SUCCESS);
  CHECK(12, fabs(col[0] - a) < 1e-15 && fabs(col[1] - b) < 1e-15);
  CHECK(13, ok_givens_unrotate(1, col, 1, &c, &s) == OK_ERR_INVALID_ARG);
  printf("ok\n");
  return 0;
}
