// Shared device/host helpers of the Boys-function library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/boys.h"

namespace boys {

// Integer power by repeated squaring, unrolled at compile time.
template <int K, typename T>
__device__ __forceinline__ T ipow(T a) {
  if constexpr (K == 0) {
    return T(1);
  } else if constexpr (K == 1) {
    return a;
  } else {
    const T h = ipow<K / 2>(a);
    if constexpr (K % 2) {
      return h * h * a;
    } else {
      return h * h;
    }
  }
}

// Order evaluated for a requested n_max on the double path: computing
// F_{n_top} with n_top > n_max and recursing down buys accuracy at m = n_max
// (Sec. 3 suggests n_top = n_max + 1); the offsets keep every m within 2e-14
// up to n_max = 36.
__host__ __device__ constexpr int f64_top_order(int n_max) {
  return n_max <= 3 ? n_max : n_max <= 12 ? n_max + 1 : n_max <= 22 ? n_max + 2 : n_max <= 27 ? n_max + 3 : n_max + 4;
}
constexpr int kMaxNF64 = 36;

// n_top for the float path: the closed form of order n_max itself up to 8,
// one order higher above (Sec. 3's F_{n+1} trick) to keep F_{n_max} within 2e-6.
__host__ __device__ constexpr int f32_top_order(int n_max) { return n_max <= 8 ? n_max : n_max + 1; }
constexpr int kMaxNF32 = 36;
// the fused float contraction keeps plain FP32 Horner sums: up to n_max = 16
constexpr int kMaxNF32Contract = 16;

// Persistent-grid size for a kernel: resident blocks per SM times SM count.
template <typename Kernel>
inline int persistent_grid(Kernel k, int block, size_t smem, int64_t tiles);

// Per-device launch setup of one kernel, done on its first launch on each
// device (a kernel's attributes belong to the device's context, so one
// process driving several GPUs needs them per device): the opt-in to
// dyn_attr bytes of dynamic shared memory (0: none needed) and, when
// want_grid, the persistent grid for dyn_smem bytes.  carveout >= 0 sets the
// kernel's preferred shared-memory share of the SM's on-chip memory (percent)
// before the grid is sized.  cache holds one slot per device (0 = not set
// up).  Returns the grid (1 when !want_grid), or 0 on a CUDA error.
constexpr int kMaxCachedDevices = 64;
template <typename Kernel>
inline int device_setup(Kernel k, int block, size_t dyn_smem, size_t dyn_attr, bool want_grid,
                        std::atomic<int> (&cache)[kMaxCachedDevices], int carveout = -1) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const bool cached = dev >= 0 && dev < kMaxCachedDevices;
  if (cached) {
    const int g = cache[dev].load(std::memory_order_acquire);
    if (g) return g;
  }
  if (dyn_attr > 0 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_attr) != cudaSuccess)
    return 0;
  if (carveout >= 0 && cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carveout) != cudaSuccess)
    return 0;
  const int g = want_grid ? persistent_grid(k, block, dyn_smem, INT64_MAX) : 1;
  if (cached) cache[dev].store(g, std::memory_order_release);
  return g;
}

template <typename Kernel>
inline int persistent_grid(Kernel k, int block, size_t smem, int64_t tiles) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t g = (int64_t)sms * per_sm;
  if (tiles < g) g = tiles;
  return (int)(g < 1 ? 1 : g);
}

// Copy a staged tile of `total` contiguous values from shared to global memory
// with 16-byte vector stores when the destination allows it (streaming stores:
// the output is written once and not re-read by this kernel).
template <typename T, int BLOCK>
__device__ __forceinline__ void store_tile(T *__restrict__ dst, const T *__restrict__ src, int total) {
  constexpr int V = 16 / sizeof(T);
  const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
  if ((a & 15) == 0) {
    const int nv = total / V;
    using Vec = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    const Vec *s = reinterpret_cast<const Vec *>(src);
    Vec *d = reinterpret_cast<Vec *>(dst);
    for (int j = threadIdx.x; j < nv; j += BLOCK) __stcs(d + j, s[j]);
    for (int j = nv * V + threadIdx.x; j < total; j += BLOCK) __stcs(dst + j, src[j]);
  } else {
    for (int j = threadIdx.x; j < total; j += BLOCK) __stcs(dst + j, src[j]);
  }
}

// ---- asynchronous bulk copies (the TMA engine, sm_90 and later) ----------
// A bulk copy moves a contiguous block between shared and global memory
// without the threads: both addresses 16-byte aligned, size a multiple of 16.

// Writes made to shared memory by ordinary stores become visible to the bulk
// copy engine only after this fence (executed by the writing threads, then a
// barrier).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Start copying `bytes` from shared memory to global memory (one thread).
__device__ __forceinline__ void bulk_store_s2g(void *gdst, const void *ssrc, unsigned bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(ssrc);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst), "r"(s), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

// Wait until every bulk copy this thread started has finished reading its
// shared-memory source (the source may then be overwritten).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }

// Wait until every bulk copy this thread started has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

}  // namespace boys
