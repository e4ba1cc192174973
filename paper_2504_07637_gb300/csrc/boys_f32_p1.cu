// FP32 forward instantiations for n_max = 9..16 (split across translation units to build in parallel).
#include "boys_f32.cuh"

int boys_f32_dispatch_p1(int n_max, const float *x, int64_t count, float *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F32_CASE(9)
    BOYS_F32_CASE(10)
    BOYS_F32_CASE(11)
    BOYS_F32_CASE(12)
    BOYS_F32_CASE(13)
    BOYS_F32_CASE(14)
    BOYS_F32_CASE(15)
    BOYS_F32_CASE(16)
    default:
      return -1;
  }
}
