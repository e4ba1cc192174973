// Throughput microbenchmarks for the ALU roofline of the Boys kernels: how
// many FP64 / FP32 operations of each kind the GPU retires per second.  Each
// thread runs 8 independent dependency chains so the pipes, not latency,
// set the rate.
#include <math.h>
#include <stdint.h>

#include "../../include/boys_microbench.h"
#include "boys_common.cuh"
#include "boys_f64.cuh"

namespace {

constexpr int kChains = 8;

template <int OP>
__global__ void __launch_bounds__(256) micro_kernel(int64_t iters, double *sink) {
  __shared__ double tab64[64];
  if (threadIdx.x < 64) tab64[threadIdx.x] = boys::kExp2Frac64[threadIdx.x];
  __syncthreads();
  double a[kChains];
  float f[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    f[c] = 1.0f + 1e-3f * (threadIdx.x + c);
  }
  const double ka = 0.9999999, kb = 1e-7;
  const float fa = 0.9999f, fb = 1e-4f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if constexpr (OP == BOYS_MICRO_DFMA) a[c] = fma(a[c], ka, kb);
      if constexpr (OP == BOYS_MICRO_DEXP) a[c] = exp(-a[c]) + 0.5;
      if constexpr (OP == BOYS_MICRO_DEXP_LIB) a[c] = boys::exp_neg(a[c], tab64) + 0.5;
      if constexpr (OP == BOYS_MICRO_DSQRT) a[c] = sqrt(a[c]) + 0.25;
      if constexpr (OP == BOYS_MICRO_DRSQRT) a[c] = rsqrt(a[c]) + 0.25;
      if constexpr (OP == BOYS_MICRO_DDIV) a[c] = 1.5 / a[c] + 0.25;
      if constexpr (OP == BOYS_MICRO_FFMA) f[c] = fmaf(f[c], fa, fb);
      if constexpr (OP == BOYS_MICRO_FEXP2) f[c] = exp2f(-f[c]) + 0.5f;
      if constexpr (OP == BOYS_MICRO_FSQRT) f[c] = sqrtf(f[c]) + 0.25f;
      if constexpr (OP == BOYS_MICRO_FDIV) f[c] = 1.5f / f[c] + 0.25f;
      if constexpr (OP == BOYS_MICRO_FRSQRT) f[c] = rsqrtf(f[c]) + 0.25f;
    }
  }
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += a[c] + (double)f[c];
  if (acc == 123.456) sink[0] = acc;  // never true; keeps the chains live
}

// FMA-only kernel with C independent chains per thread
template <int C>
__global__ void __launch_bounds__(256) dfma_chains_kernel(int64_t iters, double *sink) {
  double a[C];
#pragma unroll
  for (int c = 0; c < C; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  const double ka = 0.9999999, kb = 1e-7;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < C; ++c) a[c] = fma(a[c], ka, kb);
  }
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < C; ++c) acc += a[c];
  if (acc == 123.456) sink[0] = acc;  // never true; keeps the chains live
}

template <int C>
int launch_chains(int64_t iters, double *sink, int blocks, cudaStream_t s) {
  dfma_chains_kernel<C><<<blocks, 256, 0, s>>>(iters, sink);
  return cudaPeekAtLastError() == cudaSuccess ? BOYS_OK : BOYS_ERR_CUDA;
}

template <int OP>
int launch(int64_t iters, double *sink, int blocks, cudaStream_t s) {
  micro_kernel<OP><<<blocks, 256, 0, s>>>(iters, sink);
  return cudaPeekAtLastError() == cudaSuccess ? BOYS_OK : BOYS_ERR_CUDA;
}

}  // namespace

extern "C" int boys_microbench_launch(int op, int64_t iters, double *sink, int blocks, void *stream) {
  if (iters < 0 || blocks < 1 || !sink) return BOYS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (op) {
    case BOYS_MICRO_DFMA: return launch<BOYS_MICRO_DFMA>(iters, sink, blocks, s);
    case BOYS_MICRO_DEXP: return launch<BOYS_MICRO_DEXP>(iters, sink, blocks, s);
    case BOYS_MICRO_DSQRT: return launch<BOYS_MICRO_DSQRT>(iters, sink, blocks, s);
    case BOYS_MICRO_DRSQRT: return launch<BOYS_MICRO_DRSQRT>(iters, sink, blocks, s);
    case BOYS_MICRO_DDIV: return launch<BOYS_MICRO_DDIV>(iters, sink, blocks, s);
    case BOYS_MICRO_FFMA: return launch<BOYS_MICRO_FFMA>(iters, sink, blocks, s);
    case BOYS_MICRO_FEXP2: return launch<BOYS_MICRO_FEXP2>(iters, sink, blocks, s);
    case BOYS_MICRO_FSQRT: return launch<BOYS_MICRO_FSQRT>(iters, sink, blocks, s);
    case BOYS_MICRO_FDIV: return launch<BOYS_MICRO_FDIV>(iters, sink, blocks, s);
    case BOYS_MICRO_FRSQRT: return launch<BOYS_MICRO_FRSQRT>(iters, sink, blocks, s);
    case BOYS_MICRO_DEXP_LIB: return launch<BOYS_MICRO_DEXP_LIB>(iters, sink, blocks, s);
    default: return BOYS_ERR_ARG;
  }
}

extern "C" int boys_microbench_ops_per_thread_iter(void) { return kChains; }

extern "C" int boys_microbench_dfma(int chains, int64_t iters, double *sink, int blocks, void *stream) {
  if (iters < 0 || blocks < 1 || !sink) return BOYS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (chains) {
    case 1: return launch_chains<1>(iters, sink, blocks, s);
    case 2: return launch_chains<2>(iters, sink, blocks, s);
    case 4: return launch_chains<4>(iters, sink, blocks, s);
    case 8: return launch_chains<8>(iters, sink, blocks, s);
    case 16: return launch_chains<16>(iters, sink, blocks, s);
    default: return BOYS_ERR_ARG;
  }
}

namespace {

// Integer-pipe chains: per thread 8 independent chains of one instruction
// kind, written as inline PTX so that the front end cannot fold them.  The
// counted unit is the warp instruction; which pipe each kind occupies is
// read from ncu's per-pipe instruction counters, not assumed.
template <int KIND>
__global__ void __launch_bounds__(256) micro_int_kernel(int64_t iters, uint32_t k1, uint32_t k2, double *sink) {
  uint32_t a[kChains];
  uint64_t w[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    a[c] = threadIdx.x * 0x9e3779b9u + 17u * c + 1u;
    w[c] = ((uint64_t)a[c] << 17) | c;
  }
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if constexpr (KIND == BOYS_MICRO_INT_MADWIDE) {
        // w = lo(w) k1 + w: one 32 x 32 -> 64-bit multiply-add
        asm("{\n\t.reg .u32 l, h;\n\tmov.b64 {l, h}, %0;\n\tmad.wide.u32 %0, l, %1, %0;\n\t}" : "+l"(w[c]) : "r"(k1));
      }
      if constexpr (KIND == BOYS_MICRO_INT_MADLO) {
        asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(k1), "r"(k2));
      }
      if constexpr (KIND == BOYS_MICRO_INT_ALU) {
        // an add and an exclusive or alternate, so no two fuse into one
        // three-input instruction
        asm("add.u32 %0, %0, %1;\n\txor.b32 %0, %0, %2;" : "+r"(a[c]) : "r"(k1), "r"(k2));
      }
      if constexpr (KIND == BOYS_MICRO_INT_SHIFT64) {
        // 64-bit shift by a run-time amount, then an or: the aligned sum's shift
        asm("{\n\t.reg .u64 t;\n\tshr.b64 t, %0, %1;\n\tor.b64 %0, t, %2;\n\t}"
            : "+l"(w[c])
            : "r"(k1 & 7u), "l"((uint64_t)k2 << 40));
      }
    }
  }
  // a 64-bit mix of every chain (a plain sum of 32-bit values has a range
  // the compiler can bound, and would drop the chains as dead code)
  uint64_t acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc = (acc ^ a[c] ^ w[c]) * 0x9e3779b97f4a7c15ull;
  if (acc == 0x123456789abcdefull) sink[0] = (double)acc;  // (practically) never true; keeps the chains live
}

template <int KIND>
int launch_int(int64_t iters, double *sink, int blocks, cudaStream_t s) {
  micro_int_kernel<KIND><<<blocks, 256, 0, s>>>(iters, 0x9e3779b1u, 0x7f4a7c15u, sink);
  return cudaPeekAtLastError() == cudaSuccess ? BOYS_OK : BOYS_ERR_CUDA;
}

}  // namespace

extern "C" int boys_microbench_int(int kind, int64_t iters, double *sink, int blocks, void *stream) {
  if (iters < 0 || blocks < 1 || !sink) return BOYS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (kind) {
    case BOYS_MICRO_INT_MADWIDE: return launch_int<BOYS_MICRO_INT_MADWIDE>(iters, sink, blocks, s);
    case BOYS_MICRO_INT_MADLO: return launch_int<BOYS_MICRO_INT_MADLO>(iters, sink, blocks, s);
    case BOYS_MICRO_INT_ALU: return launch_int<BOYS_MICRO_INT_ALU>(iters, sink, blocks, s);
    case BOYS_MICRO_INT_SHIFT64: return launch_int<BOYS_MICRO_INT_SHIFT64>(iters, sink, blocks, s);
    default: return BOYS_ERR_ARG;
  }
}

extern "C" int boys_microbench_int_insts_per_chain_iter(int kind) {
  switch (kind) {
    case BOYS_MICRO_INT_MADWIDE: return 1;
    case BOYS_MICRO_INT_MADLO: return 1;
    case BOYS_MICRO_INT_ALU: return 2;
    case BOYS_MICRO_INT_SHIFT64: return 2;
    default: return -1;
  }
}

namespace {
__global__ void exp_neg_kernel(const double *__restrict__ x, int64_t n, double *__restrict__ out) {
  __shared__ double tab64[64];
  if (threadIdx.x < 64) tab64[threadIdx.x] = boys::kExp2Frac64[threadIdx.x];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = boys::exp_neg(x[i], tab64);
}
}  // namespace

extern "C" int boys_debug_exp_neg(const double *x, int64_t n, double *out, void *stream) {
  if (n < 0) return BOYS_ERR_COUNT;
  if (n == 0) return BOYS_OK;
  if (!x || !out) return BOYS_ERR_NULL;
  const int64_t blocks = (n + 255) / 256;
  exp_neg_kernel<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, out);
  return cudaPeekAtLastError() == cudaSuccess ? BOYS_OK : BOYS_ERR_CUDA;
}
