// FP32 forward instantiations for n_max = 0..8 (split across translation units to build in parallel).
#include "boys_f32.cuh"

int boys_f32_dispatch_p0(int n_max, const float *x, int64_t count, float *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F32_CASE(0)
    BOYS_F32_CASE(1)
    BOYS_F32_CASE(2)
    BOYS_F32_CASE(3)
    BOYS_F32_CASE(4)
    BOYS_F32_CASE(5)
    BOYS_F32_CASE(6)
    BOYS_F32_CASE(7)
    BOYS_F32_CASE(8)
    default:
      return -1;
  }
}
