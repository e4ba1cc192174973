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

static_assert(f32_top_order(kMaxNF32) <= BOYS_F32_TABLE_MAX_N, "fitted table too short");

// +-0 and 0 < x <= z by the bit pattern (negative nonzero and NaN excluded)
__device__ __forceinline__ bool below_cutoff_f32(float v, unsigned zbits) {
  const unsigned b = (unsigned)__float_as_int(v);
  const unsigned mag = b & 0x7fffffffu;
  return ((b >> 31) == 0 || mag == 0) && mag <= zbits;
}

// MODE 0 writes rows F_0..F_NMAX; MODE 1 is the fused contraction
// out[i] = sum_m c[i, m] F_m(x_i) (one float per argument).
// BLOCK_ / TILE_ = 0: the default shape below.
template <int NMAX, int MODE = 0, int BLOCK_ = 0, int TILE_ = 0>
struct F32Tile {
  static constexpr int W = NMAX + 1;
  static constexpr int WO = MODE == 0 ? W : 1;  // floats written per argument
  // 8 arguments per thread; small blocks keep the closed-form list's last
  // round of a tile well filled (about 30% of a tile is listed, and a block
  // waits for its slowest warp), measured best on GB300 for each band.
  // Above n_max = 16 a row is up to 148 bytes: 2 arguments per thread in
  // 128-thread blocks (2^24 arguments: n_max = 36 at 1347 G values/s, against
  // 1079 with 64/256, 1271 with 64/128, 1237 with 128/128, 897 with 128/512)
  static constexpr int TILE = TILE_ ? TILE_ : (W <= 9 || MODE == 1 ? 1024 : W <= 17 ? 512 : 256);
  static constexpr int BLOCK = BLOCK_ ? BLOCK_ : (W <= 9 || MODE == 1 ? 128 : W <= 17 ? 64 : 128);
  // rows[TILE*WO] floats, xs[TILE] floats, tab[64] floats, lst[TILE] u16
  static constexpr size_t kSmem = sizeof(float) * (TILE + TILE * WO + 64) + sizeof(unsigned short) * TILE;
};

struct F32Coef {
  const float *c;  // contraction coefficients (MODE 1), element (i, m) at c[i*c_row + m*c_col]
  int64_t c_row, c_col;
};

// cu: the coefficients held in registers when they are the same for every
// argument (row stride 0), so the contraction costs no loads per argument
template <int W, int MODE>
__device__ __forceinline__ void f32_emit(float *__restrict__ rows, int j, int64_t i, const float (&F)[W],
                                         const F32Coef &cf, const float (&cu)[W]) {
  if constexpr (MODE == 0) {
#pragma unroll
    for (int m = 0; m < W; ++m) rows[j * W + m] = F[m];
  } else {
    float acc = 0.0f;
    if (cf.c_row == 0) {
#pragma unroll
      for (int m = 0; m < W; ++m) acc = fmaf(cu[m], F[m], acc);
    } else {
      const float *ci = cf.c + i * cf.c_row;
#pragma unroll
      for (int m = 0; m < W; ++m) acc = fmaf(__ldg(ci + m * cf.c_col), F[m], acc);
    }
    rows[j] = acc;
  }
}

// Minimum resident blocks each kernel is compiled for (launch bounds), as
// measured on GB300 (each setting in its own process):
//  * the contraction (MODE 1) is bound by instruction issue: 8 blocks of 128
//    threads (64 registers) keep enough warps to fill the schedulers (faster
//    than 72 registers and 7 blocks, and than 116 registers and 4 blocks);
//  * rows: a minimum of 1 lets the compiler take about 100 registers (shared
//    memory bounds the resident blocks either way).  Over every order at 2^25
//    arguments that is faster at n_max = 8, 9 and 15 (207 vs 215, 252 vs 258,
//    415 vs 428 us) and slower elsewhere (2-8% at n_max = 0..7, 9% at 16), so
//    only those orders ask for it.
template <int NMAX, int MODE>
constexpr int f32_min_blocks() {
  return MODE == 1 ? 8 : ((NMAX == 8 || NMAX == 9 || NMAX == 15) ? 1 : 0);
}

template <int NMAX, int MODE, int BLOCK_ = 0, int TILE_ = 0>
__global__ void __launch_bounds__(F32Tile<NMAX, MODE, BLOCK_, TILE_>::BLOCK, (f32_min_blocks<NMAX, MODE>()))
    f32_split_kernel(const float *__restrict__ x, int64_t count, float *__restrict__ out, const F32Coef cf) {
  using P = F32Tile<NMAX, MODE, BLOCK_, TILE_>;
  static_assert(P::BLOCK >= 64 && P::TILE % P::BLOCK == 0 && P::TILE <= 65536, "shape");  // 64: the table load
  constexpr int NTOP = f32_top_order(NMAX);
  constexpr int W = P::W, WO = P::WO, TILE = P::TILE, BLOCK = P::BLOCK;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *rows = reinterpret_cast<float *>(smem_raw);  // 16-byte aligned, TILE*WO
  float *xs = rows + TILE * WO;
  float *tab = xs + TILE;
  unsigned short *lst = reinterpret_cast<unsigned short *>(tab + 64);
  __shared__ int cnt[1];
  if (threadIdx.x < 64) tab[threadIdx.x] = kExp2Frac32ff[threadIdx.x];
  const unsigned zbits = (unsigned)__float_as_int(BoysF32<NTOP>::kCutoff);
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t ntiles = (count + TILE - 1) / TILE;
  constexpr int PER = TILE / BLOCK;
  float cu[W];
#pragma unroll
  for (int m = 0; m < W; ++m) cu[m] = (MODE == 1 && cf.c_row == 0) ? __ldg(cf.c + m * cf.c_col) : 0.0f;
  // Uniform contraction of the asymptote row: with F_m = F_0 prod_{k<=m} (k - 1/2) y
  // (y = 1/x), sum_m c_m F_m = F_0 P(y), P(y) = sum_m hu_m y^m and
  // hu_m = c_m prod_{k<=m} (k - 1/2): a Horner polynomial instead of the row
  // and its dot product.
  float hu[W];
  {
    float g = 1.0f;
#pragma unroll
    for (int m = 0; m < W; ++m) {
      if (m > 0) g *= float(m) - 0.5f;
      hu[m] = cu[m] * g;
    }
  }
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
      const bool valid = j < nel;
      const bool lo = valid && below_cutoff_f32(v, zbits);
      xs[j] = v;
      if (MODE == 1 && cf.c_row == 0) {
        const float y = boys_frcp_rn(v);
        float acc = hu[W - 1];
#pragma unroll
        for (int m = W - 2; m >= 0; --m) acc = fmaf(acc, y, hu[m]);
        if (valid) rows[j] = acc * (0.886226925452758f * boys_rsqrtf(v));
      } else {
        float F[W];
        f32_asymptote<NMAX>(v, F);
        if (MODE == 0 || valid) f32_emit<W, MODE>(rows, j, base + j, F, cf, cu);
      }
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
      f32_emit<W, MODE>(rows, j, base + j, F, cf, cu);
    }
    float *dst = out + base * WO;
    const unsigned bytes = (unsigned)(nel * WO * sizeof(float));
    if (nel == TILE && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      fence_proxy_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) bulk_store_s2g(dst, rows, bytes);  // a full tile: 16-byte multiple
    } else {
      __syncthreads();
      store_tile<float, BLOCK>(dst, rows, nel * WO);
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
}

template <int NMAX, int MODE = 0, int BLOCK_ = 0, int TILE_ = 0>
int launch_f32(const float *x, int64_t count, float *out, cudaStream_t s, F32Coef cf = F32Coef{nullptr, 0, 0}) {
  using P = F32Tile<NMAX, MODE, BLOCK_, TILE_>;
  auto k = f32_split_kernel<NMAX, MODE, BLOCK_, TILE_>;
  static std::atomic<int> cache[kMaxCachedDevices];
  const int grid_cap = device_setup(k, P::BLOCK, P::kSmem, P::kSmem, true, cache);
  if (grid_cap == 0) return BOYS_ERR_CUDA;
  const int64_t tiles = (count + P::TILE - 1) / P::TILE;
  const int grid = (int)(tiles < grid_cap ? tiles : grid_cap);
  k<<<grid, P::BLOCK, P::kSmem, s>>>(x, count, out, cf);
  return cudaPeekAtLastError() == cudaSuccess ? BOYS_OK : BOYS_ERR_CUDA;
}

}  // namespace boys

#define BOYS_F32_CASE(k) \
  case k:                \
    return boys::launch_f32<k>(x, count, out, s);

#define BOYS_F32_CONTRACT_CASE(k) \
  case k:                         \
    return boys::launch_f32<k, 1>(x, count, out, s, boys::F32Coef{c, c_row, c_col});
