// Backward (recompute mode) instantiations for n_max = 0..17: the forward of order n_max+1 is
// re-evaluated and folded into grad_x = -sum_m g_m F_{m+1}.
#include "boys_f64.cuh"

int boys_grad_dispatch_p0(int n_max, const double *x, int64_t count, const double *g, int64_t g_row,
                           int64_t g_col, double *grad, cudaStream_t s) {
  switch (n_max) {
    BOYS_F64_GRAD_CASE(0)
    BOYS_F64_GRAD_CASE(1)
    BOYS_F64_GRAD_CASE(2)
    BOYS_F64_GRAD_CASE(3)
    BOYS_F64_GRAD_CASE(4)
    BOYS_F64_GRAD_CASE(5)
    BOYS_F64_GRAD_CASE(6)
    BOYS_F64_GRAD_CASE(7)
    BOYS_F64_GRAD_CASE(8)
    BOYS_F64_GRAD_CASE(9)
    BOYS_F64_GRAD_CASE(10)
    BOYS_F64_GRAD_CASE(11)
    BOYS_F64_GRAD_CASE(12)
    BOYS_F64_GRAD_CASE(13)
    BOYS_F64_GRAD_CASE(14)
    BOYS_F64_GRAD_CASE(15)
    BOYS_F64_GRAD_CASE(16)
    BOYS_F64_GRAD_CASE(17)
    default:
      return -1;
  }
}
