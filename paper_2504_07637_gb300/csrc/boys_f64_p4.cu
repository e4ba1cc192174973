// FP64 forward instantiations for n_max = 32..36 (split across translation units to build in parallel).
#include "boys_f64.cuh"

int boys_f64_dispatch_p4(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_CASE(32)
    BOYS_F64_CASE(33)
    BOYS_F64_CASE(34)
    BOYS_F64_CASE(35)
    BOYS_F64_CASE(36)
    default:
      return -1;
  }
}
