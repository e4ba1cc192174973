// Two-point (Trick B) instantiations for n_max = 21..36: closed forms at n_top and at n_top(n_max/2).
#include "boys_f64.cuh"

int boys_two_point_dispatch_p1(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_TWO_CASE(21)
    BOYS_F64_TWO_CASE(22)
    BOYS_F64_TWO_CASE(23)
    BOYS_F64_TWO_CASE(24)
    BOYS_F64_TWO_CASE(25)
    BOYS_F64_TWO_CASE(26)
    BOYS_F64_TWO_CASE(27)
    BOYS_F64_TWO_CASE(28)
    BOYS_F64_TWO_CASE(29)
    BOYS_F64_TWO_CASE(30)
    BOYS_F64_TWO_CASE(31)
    BOYS_F64_TWO_CASE(32)
    BOYS_F64_TWO_CASE(33)
    BOYS_F64_TWO_CASE(34)
    BOYS_F64_TWO_CASE(35)
    BOYS_F64_TWO_CASE(36)
    default:
      return -1;
  }
}
