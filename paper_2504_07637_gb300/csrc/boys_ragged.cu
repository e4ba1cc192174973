// Ragged batches: many requests of uneven length, each with its own n_max, in
// one graph-capturable call.
//
//   memset   zero the work counter and the error counter in the workspace
//   plan     one block validates every request, orders the requests by n_max
//            (a counting sort, highest order first, invalid requests last)
//            and prefix-sums their tile counts in that order into the
//            workspace (tiles never straddle two requests, so each tile has a
//            single n_max and runs its own fully unrolled kernel body)
//   eval     persistent blocks (resident blocks x SMs) take the next tile with a
//            global atomic, find its request by binary search in the tile
//            prefix (copied to shared memory), and run the FP64 tile body of
//            the plain path for that request's n_max.  Dynamic tile stealing
//            balances requests whose cost differs by n_max and length.
//
// The order by n_max keeps the SMs on one or two of the 17 kernel bodies at a
// time: taken in request order, every SM ran random orders, and instruction
// fetch stalled a warp about 20 cycles per issued instruction (ncu).
//
// No host synchronisation and no allocation: the call can be captured in a
// CUDA graph and replayed.  Arguments that only the device can read (the
// request arrays) are validated in the plan kernel; an invalid request is
// counted in the workspace error counter and its output range, when it lies
// inside [0, out_size), is filled with NaN.
#include <mutex>

#include "boys_f64.cuh"

namespace {

constexpr int kRaggedMaxN = 16;
constexpr int kPlanThreads = 1024;
constexpr int kSmemPrefixMax = 16384;  // requests whose tile prefix fits in shared memory

struct RaggedArgs {
  const double *x;
  int64_t x_size;
  const int64_t *offsets;
  const int32_t *n_max;
  const int64_t *out_offsets;
  int32_t num_requests;
  double *out;
  int64_t out_size;
  int *counters;       // [1] invalid requests; [2..3] next tile (64-bit)
  int64_t *tile_pref;  // [num_requests + 1], over the requests in perm order
  int32_t *perm;       // [num_requests]: the requests in the order their tiles run
};

// Workspace layout: 256 bytes of counters, the int64 tile prefix, then the
// int32 request order.
__host__ __device__ inline int64_t *prefix_of(void *ws) {
  return reinterpret_cast<int64_t *>(static_cast<char *>(ws) + 256);
}
__host__ __device__ inline int32_t *perm_of(void *ws, int32_t num_requests) {
  return reinterpret_cast<int32_t *>(prefix_of(ws) + num_requests + 1);
}
constexpr size_t ragged_ws_bytes(int32_t num_requests) {
  return 256 + sizeof(int64_t) * ((size_t)num_requests + 1) + sizeof(int32_t) * (size_t)num_requests;
}

// Buckets of the request order: n_max = kRaggedMaxN first, down to 0, then
// the invalid requests (whose tiles only fill NaN).
constexpr int kRaggedBuckets = kRaggedMaxN + 2;

// Tile count of request r for a given tile size, or the NaN-fill work of an
// invalid request; *bad = 1 for an invalid request.
template <int TILE>
__device__ __forceinline__ int64_t request_tiles(const RaggedArgs &a, int r, int *bad) {
  const int64_t lo = a.offsets[r], hi = a.offsets[r + 1];
  const int n = a.n_max[r];
  const int64_t olo = a.out_offsets[r], ohi = a.out_offsets[r + 1];
  const bool ok = lo >= 0 && hi >= lo && hi <= a.x_size && n >= 0 && n <= kRaggedMaxN && olo >= 0 &&
                  ohi <= a.out_size && ohi - olo == (hi - lo) * (int64_t)(n + 1);
  *bad = ok ? 0 : 1;
  if (ok) return (hi - lo + TILE - 1) / TILE;
  // invalid: fill its output range with NaN if that range is sane
  if (olo >= 0 && ohi >= olo && ohi <= a.out_size) return (ohi - olo + (int64_t)TILE * 8 - 1) / ((int64_t)TILE * 8);
  return 0;
}

template <int TILE>
__device__ __forceinline__ int request_bucket(const RaggedArgs &a, int r) {
  int bad = 0;
  request_tiles<TILE>(a, r, &bad);
  return bad ? kRaggedBuckets - 1 : kRaggedMaxN - a.n_max[r];
}

template <int TILE>
__global__ void __launch_bounds__(kPlanThreads) ragged_plan_kernel(const RaggedArgs a) {
  __shared__ int64_t carry;
  __shared__ int64_t warp_sums[kPlanThreads / 32];
  __shared__ int bad_total;
  __shared__ int hist[kRaggedBuckets], base[kRaggedBuckets];
  if (threadIdx.x == 0) {
    carry = 0;
    bad_total = 0;
    a.tile_pref[0] = 0;
  }
  if (threadIdx.x < kRaggedBuckets) hist[threadIdx.x] = 0;
  __syncthreads();
  // counting sort of the requests by bucket (the order within a bucket is
  // arbitrary: each request writes only its own rows, so the results do not
  // depend on it)
  for (int r = threadIdx.x; r < a.num_requests; r += kPlanThreads) atomicAdd(&hist[request_bucket<TILE>(a, r)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = 0; b < kRaggedBuckets; ++b) {
      base[b] = acc;
      acc += hist[b];
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < a.num_requests; r += kPlanThreads)
    a.perm[atomicAdd(&base[request_bucket<TILE>(a, r)], 1)] = r;
  __syncthreads();  // the block's writes of perm are visible to the block from here on
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 < a.num_requests; i0 += kPlanThreads) {
    const int i = i0 + threadIdx.x;
    int bad = 0;
    int64_t v = i < a.num_requests ? request_tiles<TILE>(a, a.perm[i], &bad) : 0;
    if (bad) atomicAdd(&bad_total, 1);
    // inclusive block scan: warp shuffles, then the warp totals
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t o = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += o;
    }
    if (lane == 31) warp_sums[warp] = v;
    __syncthreads();
    if (warp == 0) {
      int64_t w = warp_sums[lane];
      for (int d = 1; d < 32; d <<= 1) {
        const int64_t o = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += o;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    const int64_t incl = v + (warp ? warp_sums[warp - 1] : 0) + carry;
    if (i < a.num_requests) a.tile_pref[i + 1] = incl;
    __syncthreads();
    if (threadIdx.x == kPlanThreads - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) a.counters[1] = bad_total;
}

template <int BLOCK, int TILE>
struct RaggedSmem {
  boys::F64TileSmem<TILE> tile;
  int64_t cur;
};

template <int NMAX, int BLOCK, int TILE>
__device__ __forceinline__ void ragged_tile(const RaggedArgs &a, int r, int64_t k, boys::F64TileSmem<TILE> &sm) {
  const int64_t lo = a.offsets[r] + k * TILE;
  const int64_t hi = a.offsets[r + 1];
  const int nel = (int)((hi - lo) < TILE ? (hi - lo) : TILE);
  double *rows = a.out + a.out_offsets[r] + (k * TILE) * (NMAX + 1);
  boys::f64_tile<NMAX, BLOCK, TILE, boys::StoreRows<NMAX + 1>, false, false>(a.x + lo, nel,
                                                                             boys::StoreRows<NMAX + 1>{rows}, sm);
}

template <int BLOCK, int TILE>
__global__ void __launch_bounds__(BLOCK) ragged_eval_kernel(const RaggedArgs a) {
  __shared__ RaggedSmem<BLOCK, TILE> sm;
  extern __shared__ int64_t pref_s[];  // tile prefix when it fits, else unused
  boys::f64_load_table<BLOCK>(sm.tile);
  const int R = a.num_requests;
  const bool in_smem = R < kSmemPrefixMax;
  if (in_smem)
    for (int i = threadIdx.x; i <= R; i += BLOCK) pref_s[i] = a.tile_pref[i];
  __syncthreads();
  const int64_t *pref = in_smem ? pref_s : a.tile_pref;
  const int64_t total = pref[R];
  for (;;) {
    if (threadIdx.x == 0) sm.cur = atomicAdd(reinterpret_cast<unsigned long long *>(a.counters + 2), 1ULL);
    __syncthreads();
    const int64_t t = sm.cur;
    __syncthreads();
    if (t >= total) break;
    // position i with pref[i] <= t < pref[i+1], request perm[i]
    int lo = 0, hi = R;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pref[mid] <= t) lo = mid;
      else hi = mid;
    }
    const int r = a.perm[lo];
    const int64_t k = t - pref[lo];
    int bad = 0;
    request_tiles<TILE>(a, r, &bad);
    if (bad) {
      // NaN over this slice of the invalid request's output range
      const int64_t olo = a.out_offsets[r] + k * (int64_t)TILE * 8;
      const int64_t ohi = a.out_offsets[r + 1];
      const int64_t end = (ohi - olo) < (int64_t)TILE * 8 ? ohi : olo + (int64_t)TILE * 8;
      for (int64_t i = olo + threadIdx.x; i < end; i += BLOCK) a.out[i] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    switch (a.n_max[r]) {
#define BOYS_RAGGED_CASE(n) \
  case n:                   \
    ragged_tile<n, BLOCK, TILE>(a, r, k, sm.tile); \
    break;
      BOYS_RAGGED_CASE(0) BOYS_RAGGED_CASE(1) BOYS_RAGGED_CASE(2) BOYS_RAGGED_CASE(3) BOYS_RAGGED_CASE(4)
      BOYS_RAGGED_CASE(5) BOYS_RAGGED_CASE(6) BOYS_RAGGED_CASE(7) BOYS_RAGGED_CASE(8) BOYS_RAGGED_CASE(9)
      BOYS_RAGGED_CASE(10) BOYS_RAGGED_CASE(11) BOYS_RAGGED_CASE(12) BOYS_RAGGED_CASE(13) BOYS_RAGGED_CASE(14)
      BOYS_RAGGED_CASE(15) BOYS_RAGGED_CASE(16)
#undef BOYS_RAGGED_CASE
      default:
        break;
    }
  }
}

// Launch configurations the autotuner chooses from: (block, tile).
template <int BLOCK, int TILE>
int launch_ragged(const RaggedArgs &a, cudaStream_t s) {
  if (cudaMemsetAsync(a.counters, 0, 256, s) != cudaSuccess) return BOYS_ERR_CUDA;
  ragged_plan_kernel<TILE><<<1, kPlanThreads, 0, s>>>(a);
  if (cudaPeekAtLastError() != cudaSuccess) return BOYS_ERR_CUDA;
  const size_t dyn = a.num_requests < kSmemPrefixMax ? sizeof(int64_t) * (size_t)(a.num_requests + 1) : 0;
  auto k = ragged_eval_kernel<BLOCK, TILE>;
  // the shared-memory opt-in once per device; the grid depends on this call's prefix size
  static std::atomic<int> configured[boys::kMaxCachedDevices];
  if (boys::device_setup(k, BLOCK, 0, sizeof(int64_t) * kSmemPrefixMax, false, configured) == 0) return BOYS_ERR_CUDA;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BLOCK, dyn);
  if (per_sm < 1) per_sm = 1;
  k<<<sms * per_sm, BLOCK, dyn, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? BOYS_OK : BOYS_ERR_CUDA;
}

struct Variant {
  int block, tile;
  int (*launch)(const RaggedArgs &, cudaStream_t);
};
const Variant kVariants[] = {
    {256, 2048, launch_ragged<256, 2048>},
    {128, 1024, launch_ragged<128, 1024>},
    {256, 1024, launch_ragged<256, 1024>},
    {512, 4096, launch_ragged<512, 4096>},
    {128, 2048, launch_ragged<128, 2048>},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

}  // namespace

extern "C" {

int boys_ragged_num_variants(void) { return kNumVariants; }

boys_status boys_ragged_variant_info(int variant, int *block, int *tile) {
  if (variant < 0 || variant >= kNumVariants || !block || !tile) return BOYS_ERR_ARG;
  *block = kVariants[variant].block;
  *tile = kVariants[variant].tile;
  return BOYS_OK;
}

int boys_ragged_max_n(void) { return kRaggedMaxN; }

size_t boys_ragged_workspace_bytes(int32_t num_requests) {
  if (num_requests < 0) return 0;
  return ragged_ws_bytes(num_requests);
}

boys_status boys_eval_ragged_f64(const double *x, int64_t x_size, const int64_t *offsets, const int32_t *n_max,
                                 const int64_t *out_offsets, int32_t num_requests, double *out, int64_t out_size,
                                 void *workspace, size_t ws_bytes, int variant, void *stream) {
  if (num_requests < 0 || x_size < 0 || out_size < 0) return BOYS_ERR_COUNT;
  if (num_requests == 0) return BOYS_OK;
  if (!offsets || !n_max || !out_offsets || !workspace || (x_size > 0 && !x) || (out_size > 0 && !out))
    return BOYS_ERR_NULL;
  if (ws_bytes < boys_ragged_workspace_bytes(num_requests)) return BOYS_ERR_WORKSPACE;
  if (variant < -1 || variant >= kNumVariants) return BOYS_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) % 256) ||
      ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(offsets) |
        reinterpret_cast<uintptr_t>(out_offsets)) %
       8) ||
      (reinterpret_cast<uintptr_t>(n_max) % 4))
    return BOYS_ERR_ALIGN;
  RaggedArgs a{x, x_size, offsets, n_max, out_offsets, num_requests, out, out_size,
               static_cast<int *>(workspace), prefix_of(workspace), perm_of(workspace, num_requests)};
  return (boys_status)kVariants[variant < 0 ? 0 : variant].launch(a, static_cast<cudaStream_t>(stream));
}

boys_status boys_ragged_errors(const void *workspace, int64_t *n_bad_requests, void *stream) {
  if (!workspace || !n_bad_requests) return BOYS_ERR_NULL;
  int bad = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&bad, static_cast<const int *>(workspace) + 1, sizeof(int), cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return BOYS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return BOYS_ERR_CUDA;
  *n_bad_requests = bad;
  return BOYS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Ragged evaluation without a caller-provided workspace.
//
// Some callers cannot hand the library device scratch memory: for example a
// host application whose device memory is all owned by its own pool and that
// forbids libraries from calling cudaMalloc (an allocation can synchronise
// the device and fragments the pool), or code running where no device
// allocator is available to it.  For them the counters, the tile prefix and the
// request order live in one fixed array in the library's device image.  The array exists once
// per GPU that loads the library and stays allocated until the process
// exits; every call shares it, so calls whose work overlaps on the GPU race
// on it and must be ordered by the caller (for example, issued on one
// stream).

namespace {

constexpr int32_t kNoAllocMaxRequests = BOYS_RAGGED_NOALLOC_MAX_REQUESTS;
constexpr size_t kNoAllocScratchBytes = ragged_ws_bytes(kNoAllocMaxRequests);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
void *g_noalloc_addr[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device.  The name
// g_noalloc_scratch is only a host-side stand-in in host code, so the real
// address is looked up once per device, with that device current.
int noalloc_scratch(void **addr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return BOYS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return BOYS_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *addr = g_noalloc_addr[dev];
  return BOYS_OK;
}

}  // namespace

extern "C" boys_status boys_eval_ragged_f64_noalloc(const double *x, int64_t x_size, const int64_t *offsets,
                                                    const int32_t *n_max, const int64_t *out_offsets,
                                                    int32_t num_requests, double *out, int64_t out_size, int variant,
                                                    void *stream) {
  if (num_requests > kNoAllocMaxRequests) return BOYS_ERR_WORKSPACE;
  if (num_requests <= 0) {
    return boys_eval_ragged_f64(x, x_size, offsets, n_max, out_offsets, num_requests, out, out_size, nullptr, 0,
                                variant, stream);
  }
  void *scratch = nullptr;
  const int rc = noalloc_scratch(&scratch);
  if (rc) return (boys_status)rc;
  // the counters that must start at zero are cleared by the launch itself
  // (a memset of the first 256 bytes), and the plan kernel rewrites the
  // tile prefix, so nothing of the previous call's contents is used
  return boys_eval_ragged_f64(x, x_size, offsets, n_max, out_offsets, num_requests, out, out_size, scratch,
                              kNoAllocScratchBytes, variant, stream);
}
