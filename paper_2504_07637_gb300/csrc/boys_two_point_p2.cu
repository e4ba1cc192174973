// Two-point (Trick B) instantiations for n_max = 22..27 (closed forms at n_top and at n_top(n_max/2);
// split across translation units to build in parallel).
#include "boys_f64.cuh"

int boys_two_point_dispatch_p2(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_TWO_CASE(22)
    BOYS_F64_TWO_CASE(23)
    BOYS_F64_TWO_CASE(24)
    BOYS_F64_TWO_CASE(25)
    BOYS_F64_TWO_CASE(26)
    BOYS_F64_TWO_CASE(27)
    default:
      return -1;
  }
}
