// Two-point (Trick B) instantiations for n_max = 33..36 (closed forms at n_top and at n_top(n_max/2);
// split across translation units to build in parallel).
#include "boys_f64.cuh"

int boys_two_point_dispatch_p4(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_TWO_CASE(33)
    BOYS_F64_TWO_CASE(34)
    BOYS_F64_TWO_CASE(35)
    BOYS_F64_TWO_CASE(36)
    default:
      return -1;
  }
}
