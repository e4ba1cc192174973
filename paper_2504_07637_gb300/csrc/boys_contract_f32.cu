// FP32 fused-contraction instantiations for n_max = 0..16: out = sum_m c_m F_m(x).
#include "boys_f32.cuh"

int boys_contract_f32_dispatch(int n_max, const float *x, int64_t count, const float *c, int64_t c_row,
                               int64_t c_col, float *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F32_CONTRACT_CASE(0)
    BOYS_F32_CONTRACT_CASE(1)
    BOYS_F32_CONTRACT_CASE(2)
    BOYS_F32_CONTRACT_CASE(3)
    BOYS_F32_CONTRACT_CASE(4)
    BOYS_F32_CONTRACT_CASE(5)
    BOYS_F32_CONTRACT_CASE(6)
    BOYS_F32_CONTRACT_CASE(7)
    BOYS_F32_CONTRACT_CASE(8)
    BOYS_F32_CONTRACT_CASE(9)
    BOYS_F32_CONTRACT_CASE(10)
    BOYS_F32_CONTRACT_CASE(11)
    BOYS_F32_CONTRACT_CASE(12)
    BOYS_F32_CONTRACT_CASE(13)
    BOYS_F32_CONTRACT_CASE(14)
    BOYS_F32_CONTRACT_CASE(15)
    BOYS_F32_CONTRACT_CASE(16)
    default:
      return -1;
  }
}
