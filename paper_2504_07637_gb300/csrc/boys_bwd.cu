// Backward from saved forward rows: grad_x[i] = -sum_{m=0}^{n_max} g[i, m] F_{m+1}(x_i)
// (dF_m/dx = -F_{m+1}, from differentiating Eq. "fn" under the integral).
// One thread per row; each warp reads 32 consecutive rows of F (contiguous
// for a row-major [count, ld_F] array), and a broadcast gradient (row stride
// 0) is served from L1.  The n_max+1 fused multiply-adds per row run on the
// FP64 pipe, which sets the pace together with HBM.
#include "boys_common.cuh"

namespace {

__global__ void __launch_bounds__(256) grad_saved_kernel(const double *__restrict__ F, int64_t ld_F,
                                                         const double *__restrict__ g, int64_t g_row, int64_t g_col,
                                                         int64_t count, int terms, double *__restrict__ grad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double *Fi = F + i * ld_F + 1;
    const double *gi = g + i * g_row;
    double acc = 0.0;
#pragma unroll 4
    for (int m = 0; m < terms; ++m) acc = fma(__ldg(gi + m * g_col), __ldg(Fi + m), acc);
    grad[i] = -acc;
  }
}

}  // namespace

int boys_grad_saved_launch(const double *F, int64_t ld_F, const double *g, int64_t g_row, int64_t g_col,
                           int64_t count, int n_max, double *grad, cudaStream_t s) {
  static std::atomic<int> cache[boys::kMaxCachedDevices];
  const int grid_cap = boys::device_setup(grad_saved_kernel, 256, 0, 0, true, cache);
  if (grid_cap == 0) return BOYS_ERR_CUDA;
  const int64_t blocks = (count + 255) / 256;
  const int grid = (int)(blocks < grid_cap ? blocks : grid_cap);
  grad_saved_kernel<<<grid, 256, 0, s>>>(F, ld_F, g, g_row, g_col, count, n_max + 1, grad);
  return cudaPeekAtLastError() == cudaSuccess ? BOYS_OK : BOYS_ERR_CUDA;
}
