// Fused-contraction instantiations for n_max = 19..36: out = sum_m c_m F_m(x), rows kept in registers.
#include "boys_f64.cuh"

int boys_contract_dispatch_p1(int n_max, const double *x, int64_t count, const double *c, int64_t c_row,
                               int64_t c_col, double *out, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_CONTRACT_CASE(19)
    BOYS_F64_CONTRACT_CASE(20)
    BOYS_F64_CONTRACT_CASE(21)
    BOYS_F64_CONTRACT_CASE(22)
    BOYS_F64_CONTRACT_CASE(23)
    BOYS_F64_CONTRACT_CASE(24)
    BOYS_F64_CONTRACT_CASE(25)
    BOYS_F64_CONTRACT_CASE(26)
    BOYS_F64_CONTRACT_CASE(27)
    BOYS_F64_CONTRACT_CASE(28)
    BOYS_F64_CONTRACT_CASE(29)
    BOYS_F64_CONTRACT_CASE(30)
    BOYS_F64_CONTRACT_CASE(31)
    BOYS_F64_CONTRACT_CASE(32)
    BOYS_F64_CONTRACT_CASE(33)
    BOYS_F64_CONTRACT_CASE(34)
    BOYS_F64_CONTRACT_CASE(35)
    BOYS_F64_CONTRACT_CASE(36)
    default:
      return -1;
  }
}
