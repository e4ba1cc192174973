// FP64 forward path: one argument per thread, rows staged in shared memory
// and written out as contiguous 16-byte stores.
#pragma once

#include "boys_coeffs_f64.inc"
#include "boys_common.cuh"

namespace boys {

// F_0..F_{NMAX} at one argument, evaluating the approximation of order NTOP.
//
// Below the cut-off z_{NTOP,53} (Sec. 2):
//   Q   = q0 + q1 x + q2 x^2 u(x)/v(x)           (Eq. "pqz", root products of Eqs. "pz"/"qz")
//   D   = x + Q^NTOP sqrt(Q) e^{-x}               (the bracket of Eq. "fq")
//   F_NTOP = c_NTOP (1/D)^NTOP sqrt(1/D)          (Eq. "fq": half-integer power as s^n sqrt(s))
//   F_{m-1} = (2x F_m + e^{-x}) / (2m-1)          (Eq. "r", reusing the same e^{-x})
// Above it, the asymptote of Eq. "limf1" holds for every m <= NTOP to within
// 2^-53 (the neglected part R(m+1/2, x) decreases with m), so the row is
// F_0 = c_0 / sqrt(x), F_m = F_{m-1} (m - 1/2) / x, computed upward so that
// high orders underflow gracefully for huge x.
template <int NTOP, int NMAX>
__device__ __forceinline__ void f64_row(const double x, double (&F)[NMAX + 1]) {
  static_assert(NTOP >= NMAX && NTOP <= NMAX + 1, "NTOP is NMAX or NMAX+1");
  using Tab = BoysF64<NTOP>;
  if (x <= Tab::kCutoff) {
    double u, v;
    Tab::uv(x, u, v);
    const double r = u / v;
    const double p = (Tab::kQ2 * x) * x;
    const double q = fma(p, r, fma(Tab::kQ1, x, Tab::kQ0));
    const double e = exp(-x);
    const double T = (ipow<NTOP>(q) * sqrt(q)) * e;
    const double D = x + T;
    const double w = 1.0 / D;
    double f = (Tab::kC * ipow<NTOP>(w)) * sqrt(w);
    const double tx = x + x;
#pragma unroll
    for (int m = NTOP; m >= 1; --m) {
      if (m <= NMAX) F[m] = f;
      f = fma(tx, f, e) * (1.0 / double(2 * m - 1));
    }
    F[0] = f;
    if (!(x >= 0.0)) {  // negative arguments are outside the domain
#pragma unroll
      for (int m = 0; m <= NMAX; ++m) F[m] = __longlong_as_double(0x7ff8000000000000LL);
    }
  } else {
    // x > cut-off, +inf or NaN (NaN propagates through rsqrt)
    const double y = 1.0 / x;
    double f = 0.88622692545275801365 * rsqrt(x);  // c_0 = sqrt(pi)/2
    F[0] = f;
#pragma unroll
    for (int m = 1; m <= NMAX; ++m) {
      f = f * ((double(m) - 0.5) * y);
      F[m] = f;
    }
  }
}

template <int NMAX, int BLOCK>
__global__ void __launch_bounds__(BLOCK) f64_plain_kernel(const double *__restrict__ x, int64_t count,
                                                          double *__restrict__ out) {
  constexpr int NTOP = f64_top_order(NMAX);
  constexpr int W = NMAX + 1;
  __shared__ __align__(16) double tile[BLOCK * W];
  const int64_t ntiles = (count + BLOCK - 1) / BLOCK;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t base = t * BLOCK;
    const int64_t i = base + threadIdx.x;
    double F[W];
    const double xi = i < count ? __ldg(x + i) : 0.0;
    f64_row<NTOP, NMAX>(xi, F);
#pragma unroll
    for (int m = 0; m < W; ++m) tile[threadIdx.x * W + m] = F[m];
    __syncthreads();
    const int nel = (int)((count - base) < BLOCK ? (count - base) : BLOCK);
    store_tile<double, BLOCK>(out + base * W, tile, nel * W);
    __syncthreads();
  }
}

template <int NMAX>
int launch_f64_plain(const double *x, int64_t count, double *out, cudaStream_t s) {
  constexpr int BLOCK = 128;
  auto k = f64_plain_kernel<NMAX, BLOCK>;
  static int grid_cap = 0;
  const int64_t tiles = (count + BLOCK - 1) / BLOCK;
  if (grid_cap == 0) grid_cap = persistent_grid(k, BLOCK, 0, INT64_MAX);
  const int grid = (int)(tiles < grid_cap ? tiles : grid_cap);
  k<<<grid, BLOCK, 0, s>>>(x, count, out);
  return cudaPeekAtLastError() == cudaSuccess ? BOYS_OK : BOYS_ERR_CUDA;
}

}  // namespace boys

// Dispatch one n_max in [LO, HI] to its instantiation; returns -1 if not in range.
#define BOYS_F64_CASE(k) \
  case k:                \
    return boys::launch_f64_plain<k>(x, count, out, s);
