// Fused-contraction instantiations for n_max = 0..18: out = sum_m c_m F_m(x), rows kept in registers.
#include "boys_f64.cuh"

int boys_contract_dispatch_p0(int n_max, const double *x, int64_t count, const double *c, int64_t c_row,
                               int64_t c_col, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_CONTRACT_CASE(0)
    BOYS_F64_CONTRACT_CASE(1)
    BOYS_F64_CONTRACT_CASE(2)
    BOYS_F64_CONTRACT_CASE(3)
    BOYS_F64_CONTRACT_CASE(4)
    BOYS_F64_CONTRACT_CASE(5)
    BOYS_F64_CONTRACT_CASE(6)
    BOYS_F64_CONTRACT_CASE(7)
    BOYS_F64_CONTRACT_CASE(8)
    BOYS_F64_CONTRACT_CASE(9)
    BOYS_F64_CONTRACT_CASE(10)
    BOYS_F64_CONTRACT_CASE(11)
    BOYS_F64_CONTRACT_CASE(12)
    BOYS_F64_CONTRACT_CASE(13)
    BOYS_F64_CONTRACT_CASE(14)
    BOYS_F64_CONTRACT_CASE(15)
    BOYS_F64_CONTRACT_CASE(16)
    BOYS_F64_CONTRACT_CASE(17)
    BOYS_F64_CONTRACT_CASE(18)
    default:
      return -1;
  }
}
