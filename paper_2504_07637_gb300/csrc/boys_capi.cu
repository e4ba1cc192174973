// C ABI entry points: argument checks, then dispatch to the templated launchers.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "boys_coeffs_f64.inc"
#include "boys_common.cuh"
#include "boys_f32_row.cuh"

int boys_f64_dispatch_p0(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_f64_dispatch_p1(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_f64_dispatch_p2(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_f64_dispatch_p3(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_f64_dispatch_p4(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_f32_dispatch_p0(int n_max, const float *x, int64_t count, float *out, cudaStream_t s);
int boys_grad_dispatch_p0(int n_max, const double *x, int64_t count, const double *g, int64_t g_row, int64_t g_col,
                          double *grad, cudaStream_t s);
int boys_grad_dispatch_p1(int n_max, const double *x, int64_t count, const double *g, int64_t g_row, int64_t g_col,
                          double *grad, cudaStream_t s);
int boys_contract_dispatch_p0(int n_max, const double *x, int64_t count, const double *c, int64_t c_row,
                              int64_t c_col, double *out, cudaStream_t s);
int boys_contract_dispatch_p1(int n_max, const double *x, int64_t count, const double *c, int64_t c_row,
                              int64_t c_col, double *out, cudaStream_t s);
int boys_contract_f32_dispatch(int n_max, const float *x, int64_t count, const float *c, int64_t c_row, int64_t c_col,
                               float *out, cudaStream_t s);
int boys_two_point_dispatch_p0(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_two_point_dispatch_p1(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_two_point_dispatch_p2(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_two_point_dispatch_p3(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_two_point_dispatch_p4(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_grad_saved_launch(const double *F, int64_t ld_F, const double *g, int64_t g_row, int64_t g_col,
                           int64_t count, int n_max, double *grad, cudaStream_t s);
int boys_f32_dispatch_p1(int n_max, const float *x, int64_t count, float *out, cudaStream_t s);
int boys_f32_dispatch_p2(int n_max, const float *x, int64_t count, float *out, cudaStream_t s);
int boys_f32_dispatch_p3(int n_max, const float *x, int64_t count, float *out, cudaStream_t s);

namespace {

using boys::f32_top_order;
using boys::kMaxNF32;
using boys::kMaxNF32Contract;
using boys::kMaxNF64;

// The kernels are built for sm_103a only; reject other devices up front
// instead of failing inside a launch.
int device_ok() {
  // the answer per device never changes: 0 unknown, 1 sm_103, 2 other
  static unsigned char known[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BOYS_ERR_CUDA;
  if (dev >= 0 && dev < 64 && known[dev]) return known[dev] == 1 ? BOYS_OK : BOYS_ERR_DEVICE;
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return BOYS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return BOYS_ERR_CUDA;
  const bool ok = major == 10 && minor == 3;
  if (dev >= 0 && dev < 64) known[dev] = ok ? 1 : 2;
  return ok ? BOYS_OK : BOYS_ERR_DEVICE;
}

// A pointer the GPU cannot dereference (plain pageable host memory) would
// fault the kernel; refuse it on the host instead.
int device_accessible(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return BOYS_ERR_ARG;
  }
  if (a.type == cudaMemoryTypeUnregistered) return BOYS_ERR_ARG;
  // pinned host memory is read in place over the C2C link; that needs the
  // device mapping to be the identity (true under unified addressing)
  if (a.type == cudaMemoryTypeHost && a.devicePointer != p) return BOYS_ERR_ARG;
  return BOYS_OK;
}

int check_rows(const void *x, int64_t count, int n_max, int max_n, const void *out, size_t elem) {
  if (count < 0) return BOYS_ERR_COUNT;
  if (n_max < 0 || n_max > max_n) return BOYS_ERR_NMAX;
  if (count > INT64_MAX / (n_max + 1)) return BOYS_ERR_COUNT;
  if (count == 0) return BOYS_OK;
  if (!x || !out) return BOYS_ERR_NULL;
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(out)) % elem) return BOYS_ERR_ALIGN;
  int rc = device_ok();
  if (rc) return rc;
  if ((rc = device_accessible(x))) return rc;
  return device_accessible(out);
}

// A second stream (and its fork/join events) per device for the host-buffer
// pipeline, created on first use and kept for the life of the process.
struct HelperStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kMaxDevices = 64;
HelperStream g_helper[kMaxDevices];
std::mutex g_helper_mu;

int helper_for_current_device(HelperStream **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BOYS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_helper_mu);
  HelperStream &h = g_helper[dev];
  if (!h.s) {
    if (cudaStreamCreateWithFlags(&h.s, cudaStreamNonBlocking) != cudaSuccess) return BOYS_ERR_CUDA;
    if (cudaEventCreateWithFlags(&h.fork, cudaEventDisableTiming) != cudaSuccess) return BOYS_ERR_CUDA;
    if (cudaEventCreateWithFlags(&h.join, cudaEventDisableTiming) != cudaSuccess) return BOYS_ERR_CUDA;
  }
  *out = &h;
  return BOYS_OK;
}

int dispatch_f64(int n_max, const double *x, int64_t count, double *out, cudaStream_t s) {
  int rc;
  // the order ranges of boys_f64_p0.cu .. boys_f64_p4.cu
  if (n_max <= 12) rc = boys_f64_dispatch_p0(n_max, x, count, out, s);
  else if (n_max <= 20) rc = boys_f64_dispatch_p1(n_max, x, count, out, s);
  else if (n_max <= 26) rc = boys_f64_dispatch_p2(n_max, x, count, out, s);
  else if (n_max <= 31) rc = boys_f64_dispatch_p3(n_max, x, count, out, s);
  else rc = boys_f64_dispatch_p4(n_max, x, count, out, s);
  return rc < 0 ? BOYS_ERR_NMAX : rc;
}

int dispatch_f32(int n_max, const float *x, int64_t count, float *out, cudaStream_t s) {
  // the order ranges of boys_f32_p0.cu .. boys_f32_p3.cu
  const int rc = n_max <= 8    ? boys_f32_dispatch_p0(n_max, x, count, out, s)
                 : n_max <= 16 ? boys_f32_dispatch_p1(n_max, x, count, out, s)
                 : n_max <= 26 ? boys_f32_dispatch_p2(n_max, x, count, out, s)
                               : boys_f32_dispatch_p3(n_max, x, count, out, s);
  return rc < 0 ? BOYS_ERR_NMAX : rc;
}

constexpr int64_t kHostChunkGranule = 2048;  // the kernels' tile

// Host arrays streamed through a device workspace in double-buffered chunks:
// chunk i is copied in, evaluated and copied out on stream i % 2 (the
// caller's stream or the helper stream), so one chunk's copies (copy engines)
// overlap the other chunk's kernel, and same-stream order protects each buffer.
template <typename T, typename Dispatch>
int host_pipeline(const T *x_host, int64_t count, int n_max, int max_n, T *out_host, void *workspace,
                  size_t ws_bytes, cudaStream_t caller, Dispatch dispatch) {
  if (count < 0) return BOYS_ERR_COUNT;
  if (n_max < 0 || n_max > max_n) return BOYS_ERR_NMAX;
  if (count > INT64_MAX / (n_max + 1)) return BOYS_ERR_COUNT;
  if (count == 0) return BOYS_OK;
  if (!x_host || !out_host || !workspace) return BOYS_ERR_NULL;
  if ((reinterpret_cast<uintptr_t>(x_host) | reinterpret_cast<uintptr_t>(out_host)) % sizeof(T) ||
      reinterpret_cast<uintptr_t>(workspace) % 256)
    return BOYS_ERR_ALIGN;
  const size_t per_arg = sizeof(T) * (size_t)(n_max + 2);
  const int64_t chunk = (int64_t)(ws_bytes / (2 * per_arg)) / kHostChunkGranule * kHostChunkGranule;
  if (chunk < kHostChunkGranule) return BOYS_ERR_WORKSPACE;
  int rc = device_ok();
  if (rc) return rc;
  {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, workspace) != cudaSuccess) {
      cudaGetLastError();
      return BOYS_ERR_ARG;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return BOYS_ERR_ARG;
  }
  HelperStream *h = nullptr;
  if ((rc = helper_for_current_device(&h))) return rc;
  cudaStream_t s[2] = {caller, h->s};
  // the helper stream starts after everything already queued on the caller's stream
  if (cudaEventRecord(h->fork, s[0]) != cudaSuccess || cudaStreamWaitEvent(s[1], h->fork, 0) != cudaSuccess)
    return BOYS_ERR_CUDA;
  const int W = n_max + 1;
  char *ws = static_cast<char *>(workspace);
  T *xbuf[2], *obuf[2];
  for (int b = 0; b < 2; ++b) {
    xbuf[b] = reinterpret_cast<T *>(ws + (size_t)b * chunk * per_arg);
    obuf[b] = xbuf[b] + chunk;
  }
  int64_t i = 0;
  for (int64_t off = 0; off < count; off += chunk, ++i) {
    const int b = (int)(i & 1);
    const int64_t n = (count - off) < chunk ? (count - off) : chunk;
    if (cudaMemcpyAsync(xbuf[b], x_host + off, (size_t)n * sizeof(T), cudaMemcpyDefault, s[b]) != cudaSuccess)
      return BOYS_ERR_CUDA;
    if ((rc = dispatch(n_max, xbuf[b], n, obuf[b], s[b]))) return rc;
    if (cudaMemcpyAsync(out_host + off * W, obuf[b], (size_t)n * W * sizeof(T), cudaMemcpyDefault, s[b]) !=
        cudaSuccess)
      return BOYS_ERR_CUDA;
  }
  // the caller's stream completes only after the helper stream's chunks
  if (cudaEventRecord(h->join, s[1]) != cudaSuccess || cudaStreamWaitEvent(s[0], h->join, 0) != cudaSuccess)
    return BOYS_ERR_CUDA;
  return BOYS_OK;
}

}  // namespace

extern "C" {

const char *boys_status_string(int status) {
  switch (status) {
    case BOYS_OK: return "ok";
    case BOYS_ERR_NULL: return "null pointer";
    case BOYS_ERR_COUNT: return "invalid count";
    case BOYS_ERR_NMAX: return "n_max out of range";
    case BOYS_ERR_ALIGN: return "misaligned pointer";
    case BOYS_ERR_WORKSPACE: return "workspace too small";
    case BOYS_ERR_CUDA: return "CUDA error";
    case BOYS_ERR_ARG: return "invalid argument";
    case BOYS_ERR_DEVICE: return "device is not sm_103 (GB300)";
    default: return "unknown status";
  }
}

int boys_max_n(int precision_bits) {
  if (precision_bits == 53) return kMaxNF64;
  if (precision_bits == 24) return kMaxNF32;
  return -1;
}

double boys_cutoff(int n, int precision_bits) {
  if (precision_bits == 53 && n >= 0 && n <= BOYS_F64_TABLE_MAX_N) return kBoysF64CutoffHost[n];
  if (precision_bits == 24 && n >= 0 && n <= BOYS_F32_TABLE_MAX_N) return kBoysF32CutoffHost[n];
  return NAN;
}

int boys_top_order_f32(int n_max) {
  if (n_max < 0 || n_max > kMaxNF32) return -1;
  return f32_top_order(n_max);
}

boys_status boys_eval_f32(const float *x, int64_t count, int n_max, float *out, void *stream) {
  int rc = check_rows(x, count, n_max, kMaxNF32, out, sizeof(float));
  if (rc || count == 0) return (boys_status)rc;
  return (boys_status)dispatch_f32(n_max, x, count, out, static_cast<cudaStream_t>(stream));
}

int boys_top_order_f64(int n_max) {
  if (n_max < 0 || n_max > kMaxNF64) return -1;
  return boys::f64_top_order(n_max);
}

boys_status boys_eval_f64(const double *x, int64_t count, int n_max, double *out, void *stream) {
  int rc = check_rows(x, count, n_max, kMaxNF64, out, sizeof(double));
  if (rc || count == 0) return (boys_status)rc;
  return (boys_status)dispatch_f64(n_max, x, count, out, static_cast<cudaStream_t>(stream));
}

boys_status boys_eval_backward_f64(const double *x, const double *F, int64_t ld_F, const double *g, int64_t g_row_stride,
                                   int64_t g_col_stride, int64_t count, int n_max, double *grad_x, void *stream) {
  if (count < 0) return BOYS_ERR_COUNT;
  if (n_max < 0 || n_max > kMaxNF64 - 1) return BOYS_ERR_NMAX;
  if (g_row_stride < 0 || g_col_stride < 0) return BOYS_ERR_ARG;
  if (F && ld_F < n_max + 2) return BOYS_ERR_ARG;
  if (count == 0) return BOYS_OK;
  if (!g || !grad_x || (!F && !x)) return BOYS_ERR_NULL;
  if (F && count > INT64_MAX / ld_F) return BOYS_ERR_COUNT;
  if (g_row_stride && count > INT64_MAX / g_row_stride) return BOYS_ERR_COUNT;
  const uintptr_t bits = reinterpret_cast<uintptr_t>(g) | reinterpret_cast<uintptr_t>(grad_x) |
                         reinterpret_cast<uintptr_t>(F) | reinterpret_cast<uintptr_t>(x);
  if (bits % sizeof(double)) return BOYS_ERR_ALIGN;
  int rc = device_ok();
  if (rc) return (boys_status)rc;
  if ((rc = device_accessible(g)) || (rc = device_accessible(grad_x))) return (boys_status)rc;
  if ((rc = device_accessible(F ? (const void *)F : (const void *)x))) return (boys_status)rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (F) {
    rc = boys_grad_saved_launch(F, ld_F, g, g_row_stride, g_col_stride, count, n_max, grad_x, s);
  } else {
    rc = n_max <= 17 ? boys_grad_dispatch_p0(n_max, x, count, g, g_row_stride, g_col_stride, grad_x, s)
                     : boys_grad_dispatch_p1(n_max, x, count, g, g_row_stride, g_col_stride, grad_x, s);
    if (rc < 0) rc = BOYS_ERR_NMAX;
  }
  return (boys_status)rc;
}

boys_status boys_eval_f64_two_point(const double *x, int64_t count, int n_max, double *out, void *stream) {
  if (n_max < 2 && n_max >= 0) return boys_eval_f64(x, count, n_max, out, stream);  // nothing to split
  int rc = check_rows(x, count, n_max, kMaxNF64, out, sizeof(double));
  if (rc || count == 0) return (boys_status)rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the order ranges of boys_two_point_p0.cu .. boys_two_point_p4.cu
  if (n_max <= 14) rc = boys_two_point_dispatch_p0(n_max, x, count, out, s);
  else if (n_max <= 21) rc = boys_two_point_dispatch_p1(n_max, x, count, out, s);
  else if (n_max <= 27) rc = boys_two_point_dispatch_p2(n_max, x, count, out, s);
  else if (n_max <= 32) rc = boys_two_point_dispatch_p3(n_max, x, count, out, s);
  else rc = boys_two_point_dispatch_p4(n_max, x, count, out, s);
  return (boys_status)(rc < 0 ? BOYS_ERR_NMAX : rc);
}

boys_status boys_eval_contract_f64(const double *x, int64_t count, int n_max, const double *c, int64_t c_row,
                                   int64_t c_col, double *out, void *stream) {
  if (count < 0) return BOYS_ERR_COUNT;
  if (n_max < 0 || n_max > kMaxNF64) return BOYS_ERR_NMAX;
  if (c_row < 0 || c_col < 0) return BOYS_ERR_ARG;
  if (count == 0) return BOYS_OK;
  if (!x || !c || !out) return BOYS_ERR_NULL;
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(out)) %
      sizeof(double))
    return BOYS_ERR_ALIGN;
  int rc = device_ok();
  if (rc) return (boys_status)rc;
  if ((rc = device_accessible(x)) || (rc = device_accessible(c)) || (rc = device_accessible(out)))
    return (boys_status)rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = n_max <= 18 ? boys_contract_dispatch_p0(n_max, x, count, c, c_row, c_col, out, s)
                   : boys_contract_dispatch_p1(n_max, x, count, c, c_row, c_col, out, s);
  return (boys_status)(rc < 0 ? BOYS_ERR_NMAX : rc);
}

boys_status boys_eval_contract_f32(const float *x, int64_t count, int n_max, const float *c, int64_t c_row,
                                   int64_t c_col, float *out, void *stream) {
  if (count < 0) return BOYS_ERR_COUNT;
  if (n_max < 0 || n_max > kMaxNF32Contract) return BOYS_ERR_NMAX;
  if (c_row < 0 || c_col < 0) return BOYS_ERR_ARG;
  if (count == 0) return BOYS_OK;
  if (!x || !c || !out) return BOYS_ERR_NULL;
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(out)) %
      sizeof(float))
    return BOYS_ERR_ALIGN;
  int rc = device_ok();
  if (rc) return (boys_status)rc;
  if ((rc = device_accessible(x)) || (rc = device_accessible(c)) || (rc = device_accessible(out)))
    return (boys_status)rc;
  rc = boys_contract_f32_dispatch(n_max, x, count, c, c_row, c_col, out, static_cast<cudaStream_t>(stream));
  return (boys_status)(rc < 0 ? BOYS_ERR_NMAX : rc);
}

size_t boys_eval_f64_host_workspace(int n_max, int64_t chunk) {
  if (n_max < 0 || n_max > kMaxNF64 || chunk <= 0) return 0;
  chunk = (chunk + kHostChunkGranule - 1) / kHostChunkGranule * kHostChunkGranule;
  return (size_t)2 * (size_t)chunk * sizeof(double) * (size_t)(n_max + 2);
}

size_t boys_eval_f32_host_workspace(int n_max, int64_t chunk) {
  if (n_max < 0 || n_max > kMaxNF32 || chunk <= 0) return 0;
  chunk = (chunk + kHostChunkGranule - 1) / kHostChunkGranule * kHostChunkGranule;
  return (size_t)2 * (size_t)chunk * sizeof(float) * (size_t)(n_max + 2);
}

boys_status boys_eval_f64_host(const double *x_host, int64_t count, int n_max, double *out_host, void *workspace,
                               size_t ws_bytes, void *stream) {
  return (boys_status)host_pipeline<double>(x_host, count, n_max, kMaxNF64, out_host, workspace, ws_bytes,
                                            static_cast<cudaStream_t>(stream), dispatch_f64);
}

boys_status boys_eval_f32_host(const float *x_host, int64_t count, int n_max, float *out_host, void *workspace,
                               size_t ws_bytes, void *stream) {
  return (boys_status)host_pipeline<float>(x_host, count, n_max, kMaxNF32, out_host, workspace, ws_bytes,
                                           static_cast<cudaStream_t>(stream), dispatch_f32);
}

}  // extern "C"
