// FP32 forward path: HBM-bound (4 bytes in, 4 (n_max+1) bytes out per
// argument), so the design minimises issued instructions and overlaps
// memory with arithmetic:
//  * every argument of a tile first gets the cheap asymptote row, computed in
//    place in lane order; the arguments below the cut-off (about 30% on
//    integral-like inputs, spread at random) are listed in shared memory and
//    only they run the closed form (~6x the asymptote's cost in float-float
//    arithmetic), densely, overwriting their rows;
//  * the tile's rows leave as one asynchronous bulk copy (TMA engine), so the
//    block moves on to the next tile while the copy drains;
//  * the next tile's arguments are loaded into registers during the current
//    tile's arithmetic.
#pragma once

#include "boys_common.cuh"
#include "boys_f32_row.cuh"

namespace boys {

static __constant__ float kExp2Frac32ff[64] = BOYS_EXP2_FRAC32_FF;

// n_top for the float path: the closed form of order n_max itself up to 8,
// one order higher above (Sec. 3's F_{n+1} trick) to keep F_{n_max} within 2e-6.
__host__ __device__ constexpr int f32_top_order(int n_max) { return n_max <= 8 ? n_max : n_max + 1; }
constexpr int kMaxNF32 = 16;
static_assert(f32_top_order(kMaxNF32) <= BOYS_F32_TABLE_MAX_N, "fitted table too short");

// +-0 and 0 < x <= z by the bit pattern (negative nonzero and NaN excluded)
__device__ __forceinline__ bool below_cutoff_f32(float v, unsigned zbits) {
  const unsigned b = (unsigned)__float_as_int(v);
  const unsigned mag = b & 0x7fffffffu;
  return ((b >> 31) == 0 || mag == 0) && mag <= zbits;
}

template <int NMAX>
struct F32Tile {
  static constexpr int W = NMAX + 1;
  static constexpr int TILE = W <= 9 ? 1024 : 512;
  static constexpr int BLOCK = 256;
  // xs[TILE] floats, rows[TILE*W] floats, tab[64] floats, lst[TILE] u16
  static constexpr size_t kSmem = sizeof(float) * (TILE + TILE * W + 64) + sizeof(unsigned short) * TILE;
};

template <int NMAX>
__global__ void __launch_bounds__(256) f32_split_kernel(const float *__restrict__ x, int64_t count,
                                                        float *__restrict__ out) {
  using P = F32Tile<NMAX>;
  constexpr int NTOP = f32_top_order(NMAX);
  constexpr int W = P::W, TILE = P::TILE, BLOCK = P::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *rows = reinterpret_cast<float *>(smem_raw);  // 16-byte aligned, TILE*W
  float *xs = rows + TILE * W;
  float *tab = xs + TILE;
  unsigned short *lst = reinterpret_cast<unsigned short *>(tab + 64);
  __shared__ int cnt[1];
  if (threadIdx.x < 64) tab[threadIdx.x] = kExp2Frac32ff[threadIdx.x];
  const unsigned zbits = (unsigned)__float_as_int(BoysF32<NTOP>::kCutoff);
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t ntiles = (count + TILE - 1) / TILE;
  constexpr int PER = TILE / BLOCK;
  // the next tile's arguments are loaded into registers while the current
  // tile is evaluated, so the load latency hides behind the arithmetic
  float pre[PER];
  auto prefetch = [&](int64_t tile) {
    const int64_t b = tile * TILE;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int64_t i = b + k * BLOCK + threadIdx.x;
      pre[k] = (tile < ntiles && i < count) ? __ldcs(x + i) : 0.0f;
    }
  };
  prefetch(blockIdx.x);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t base = t * TILE;
    const int nel = (int)((count - base) < TILE ? (count - base) : TILE);
    if (threadIdx.x == 0) {
      bulk_wait_read();  // the previous tile's bulk copy has read the rows
      cnt[0] = 0;
    }
    __syncthreads();
    // every argument gets the cheap asymptote row in place (lane order, no
    // bank conflicts); the below-cut-off ones are listed for the closed form
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int j = k * BLOCK + threadIdx.x;
      const float v = pre[k];
      const bool lo = j < nel && below_cutoff_f32(v, zbits);
      xs[j] = v;
      float F[W];
      f32_asymptote<NMAX>(v, F);
#pragma unroll
      for (int m = 0; m < W; ++m) rows[j * W + m] = F[m];
      const unsigned mlo = __ballot_sync(0xffffffffu, lo);
      int plo = 0;
      if (lane == 0 && mlo) plo = atomicAdd(&cnt[0], __popc(mlo));
      plo = __shfl_sync(0xffffffffu, plo, 0);
      if (lo) lst[plo + __popc(mlo & lt)] = (unsigned short)j;
    }
    prefetch(t + gridDim.x);
    __syncthreads();
    // the closed form overwrites the rows of the listed arguments
    const int nlo = cnt[0];
    for (int q = threadIdx.x; q < nlo; q += BLOCK) {
      const int j = lst[q];
      float F[W];
      f32_formula<NTOP, NMAX>(xs[j], F, tab);
#pragma unroll
      for (int m = 0; m < W; ++m) rows[j * W + m] = F[m];
    }
    float *dst = out + base * W;
    const unsigned bytes = (unsigned)(nel * W * sizeof(float));
    if (nel == TILE && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      fence_proxy_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) bulk_store_s2g(dst, rows, bytes);  // a full tile: 16-byte multiple
    } else {
      __syncthreads();
      store_tile<float, BLOCK>(dst, rows, nel * W);
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
}

template <int NMAX>
int launch_f32(const float *x, int64_t count, float *out, cudaStream_t s) {
  using P = F32Tile<NMAX>;
  auto k = f32_split_kernel<NMAX>;
  static int grid_cap = 0;
  if (grid_cap == 0) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::kSmem) != cudaSuccess)
      return BOYS_ERR_CUDA;
    grid_cap = persistent_grid(k, P::BLOCK, P::kSmem, INT64_MAX);
  }
  const int64_t tiles = (count + P::TILE - 1) / P::TILE;
  const int grid = (int)(tiles < grid_cap ? tiles : grid_cap);
  k<<<grid, P::BLOCK, P::kSmem, s>>>(x, count, out);
  return cudaPeekAtLastError() == cudaSuccess ? BOYS_OK : BOYS_ERR_CUDA;
}

}  // namespace boys

#define BOYS_F32_CASE(k) \
  case k:                \
    return boys::launch_f32<k>(x, count, out, s);
