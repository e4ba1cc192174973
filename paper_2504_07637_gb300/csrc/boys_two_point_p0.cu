// Two-point (Trick B) instantiations for n_max = 2..14 (closed forms at n_top and at n_top(n_max/2);
// split across translation units to build in parallel).
#include "boys_f64.cuh"

int boys_two_point_dispatch_p0(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_TWO_CASE(2)
    BOYS_F64_TWO_CASE(3)
    BOYS_F64_TWO_CASE(4)
    BOYS_F64_TWO_CASE(5)
    BOYS_F64_TWO_CASE(6)
    BOYS_F64_TWO_CASE(7)
    BOYS_F64_TWO_CASE(8)
    BOYS_F64_TWO_CASE(9)
    BOYS_F64_TWO_CASE(10)
    BOYS_F64_TWO_CASE(11)
    BOYS_F64_TWO_CASE(12)
    BOYS_F64_TWO_CASE(13)
    BOYS_F64_TWO_CASE(14)
    default:
      return -1;
  }
}
