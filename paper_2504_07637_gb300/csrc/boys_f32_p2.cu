// FP32 forward instantiations for n_max = 17..26 (split across translation units to build in parallel).
#include "boys_f32.cuh"

int boys_f32_dispatch_p2(int n_max, const float *x, int64_t count, float *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F32_CASE(17)
    BOYS_F32_CASE(18)
    BOYS_F32_CASE(19)
    BOYS_F32_CASE(20)
    BOYS_F32_CASE(21)
    BOYS_F32_CASE(22)
    BOYS_F32_CASE(23)
    BOYS_F32_CASE(24)
    BOYS_F32_CASE(25)
    BOYS_F32_CASE(26)
    default:
      return -1;
  }
}
