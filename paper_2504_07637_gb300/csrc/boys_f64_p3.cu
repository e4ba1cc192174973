// FP64 forward instantiations for n_max = 27..31 (split across translation units to build in parallel).
#include "boys_f64.cuh"

int boys_f64_dispatch_p3(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_CASE(27)
    BOYS_F64_CASE(28)
    BOYS_F64_CASE(29)
    BOYS_F64_CASE(30)
    BOYS_F64_CASE(31)
    default:
      return -1;
  }
}
