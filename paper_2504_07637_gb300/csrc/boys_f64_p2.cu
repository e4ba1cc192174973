// FP64 forward instantiations for n_max = 21..26 (split across translation units to build in parallel).
#include "boys_f64.cuh"

int boys_f64_dispatch_p2(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_CASE(21)
    BOYS_F64_CASE(22)
    BOYS_F64_CASE(23)
    BOYS_F64_CASE(24)
    BOYS_F64_CASE(25)
    BOYS_F64_CASE(26)
    default:
      return -1;
  }
}
