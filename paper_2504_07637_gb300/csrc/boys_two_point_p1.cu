// Two-point (Trick B) instantiations for n_max = 15..21 (closed forms at n_top and at n_top(n_max/2);
// split across translation units to build in parallel).
#include "boys_f64.cuh"

int boys_two_point_dispatch_p1(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_TWO_CASE(15)
    BOYS_F64_TWO_CASE(16)
    BOYS_F64_TWO_CASE(17)
    BOYS_F64_TWO_CASE(18)
    BOYS_F64_TWO_CASE(19)
    BOYS_F64_TWO_CASE(20)
    BOYS_F64_TWO_CASE(21)
    default:
      return -1;
  }
}
