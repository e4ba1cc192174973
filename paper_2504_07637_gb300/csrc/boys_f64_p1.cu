// FP64 forward instantiations for n_max = 13..20 (split across translation units to build in parallel).
#include "boys_f64.cuh"

int boys_f64_dispatch_p1(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_CASE(13)
    BOYS_F64_CASE(14)
    BOYS_F64_CASE(15)
    BOYS_F64_CASE(16)
    BOYS_F64_CASE(17)
    BOYS_F64_CASE(18)
    BOYS_F64_CASE(19)
    BOYS_F64_CASE(20)
    default:
      return -1;
  }
}
