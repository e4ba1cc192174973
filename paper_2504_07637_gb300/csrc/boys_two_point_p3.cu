// Two-point (Trick B) instantiations for n_max = 28..32 (closed forms at n_top and at n_top(n_max/2);
// split across translation units to build in parallel).
#include "boys_f64.cuh"

int boys_two_point_dispatch_p3(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_TWO_CASE(28)
    BOYS_F64_TWO_CASE(29)
    BOYS_F64_TWO_CASE(30)
    BOYS_F64_TWO_CASE(31)
    BOYS_F64_TWO_CASE(32)
    default:
      return -1;
  }
}
