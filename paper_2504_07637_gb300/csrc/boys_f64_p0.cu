// FP64 forward instantiations for n_max = 0..12 (split across translation units to build in parallel).
#include "boys_f64.cuh"

int boys_f64_dispatch_p0(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_CASE(0)
    BOYS_F64_CASE(1)
    BOYS_F64_CASE(2)
    BOYS_F64_CASE(3)
    BOYS_F64_CASE(4)
    BOYS_F64_CASE(5)
    BOYS_F64_CASE(6)
    BOYS_F64_CASE(7)
    BOYS_F64_CASE(8)
    BOYS_F64_CASE(9)
    BOYS_F64_CASE(10)
    BOYS_F64_CASE(11)
    BOYS_F64_CASE(12)
    default:
      return -1;
  }
}
