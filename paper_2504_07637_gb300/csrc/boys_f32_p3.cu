// FP32 forward instantiations for n_max = 27..36 (split across translation units to build in parallel).
#include "boys_f32.cuh"

int boys_f32_dispatch_p3(int n_max, const float *x, int64_t count, float *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F32_CASE(27)
    BOYS_F32_CASE(28)
    BOYS_F32_CASE(29)
    BOYS_F32_CASE(30)
    BOYS_F32_CASE(31)
    BOYS_F32_CASE(32)
    BOYS_F32_CASE(33)
    BOYS_F32_CASE(34)
    BOYS_F32_CASE(35)
    BOYS_F32_CASE(36)
    default:
      return -1;
  }
}
