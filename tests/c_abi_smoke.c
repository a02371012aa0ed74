/* Plain C use of the boundary (no C++ and no Python): include the header,
 * link the library, call it.  Without a device a grid cannot be created and
 * the call says so; the device-free compile check of the run-time stage
 * kernels succeeds. */
#include <stdio.h>
#include <string.h>

#include "hj.h"

int main(void) {
  int n[4] = {41, 41, 41, 41};
  double lo[4] = {-5.0, -2.0, -0.35, -1.5}, hi[4] = {5.0, 2.0, 0.35, 1.5};
  hj_grid g = NULL;
  hj_status st = hj_grid_create(&g, 4, n, lo, hi, NULL);
  printf("grid_create %d %s\n", (int)st, st == HJ_OK ? "" : hj_last_error());
  if (st == HJ_OK) hj_grid_destroy(g);
  hj_status jc = hj_jit_check(4, n, HJ_QUAD_X4, HJ_WENO5, 256);
  printf("jit_check %d\n", (int)jc);
  hj_status bad = hj_jit_check(4, n, HJ_QUAD_X4, 3, 256);
  printf("jit_check_bad %d %s\n", (int)bad, hj_last_error());
  printf("launches %llu\n", (unsigned long long)hj_kernel_launches());
  return (jc == HJ_OK && bad == HJ_ERR_ARG) ? 0 : 1;
}
