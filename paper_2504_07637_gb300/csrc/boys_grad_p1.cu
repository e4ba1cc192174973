// Backward (recompute mode) instantiations for n_max = 18..35: the forward of order n_max+1 is
// re-evaluated and folded into grad_x = -sum_m g_m F_{m+1}.
#include "boys_f64.cuh"

int boys_grad_dispatch_p1(int n_max, const double *x, int64_t count, const double *g, int64_t g_row,
                           int64_t g_col, double *grad, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_GRAD_CASE(18)
    BOYS_F64_GRAD_CASE(19)
    BOYS_F64_GRAD_CASE(20)
    BOYS_F64_GRAD_CASE(21)
    BOYS_F64_GRAD_CASE(22)
    BOYS_F64_GRAD_CASE(23)
    BOYS_F64_GRAD_CASE(24)
    BOYS_F64_GRAD_CASE(25)
    BOYS_F64_GRAD_CASE(26)
    BOYS_F64_GRAD_CASE(27)
    BOYS_F64_GRAD_CASE(28)
    BOYS_F64_GRAD_CASE(29)
    BOYS_F64_GRAD_CASE(30)
    BOYS_F64_GRAD_CASE(31)
    BOYS_F64_GRAD_CASE(32)
    BOYS_F64_GRAD_CASE(33)
    BOYS_F64_GRAD_CASE(34)
    BOYS_F64_GRAD_CASE(35)
    default:
      return -1;
  }
}
