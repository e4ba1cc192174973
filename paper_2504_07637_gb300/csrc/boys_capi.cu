// C ABI entry points: argument checks, then dispatch to the templated launchers.
#include <math.h>
#include <stdint.h>

#include "boys_coeffs_f64.inc"
#include "boys_common.cuh"

int boys_f64_dispatch_p0(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_f64_dispatch_p1(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);
int boys_f64_dispatch_p2(int n_max, const double *x, int64_t count, double *out, cudaStream_t s);

namespace {

using boys::kMaxNF64;

// The kernels are built for sm_103a only; reject other devices up front
// instead of failing inside a launch.
int device_ok() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BOYS_ERR_CUDA;
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return BOYS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return BOYS_ERR_CUDA;
  return (major == 10 && minor == 3) ? BOYS_OK : BOYS_ERR_DEVICE;
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
  return -1;
}

double boys_cutoff(int n, int precision_bits) {
  if (precision_bits == 53 && n >= 0 && n <= BOYS_F64_TABLE_MAX_N) return kBoysF64CutoffHost[n];
  return NAN;
}

int boys_top_order_f64(int n_max) {
  if (n_max < 0 || n_max > kMaxNF64) return -1;
  return boys::f64_top_order(n_max);
}

boys_status boys_eval_f64(const double *x, int64_t count, int n_max, double *out, void *stream) {
  int rc = check_rows(x, count, n_max, kMaxNF64, out, sizeof(double));
  if (rc || count == 0) return (boys_status)rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_max <= 12) rc = boys_f64_dispatch_p0(n_max, x, count, out, s);
  else if (n_max <= 24) rc = boys_f64_dispatch_p1(n_max, x, count, out, s);
  else rc = boys_f64_dispatch_p2(n_max, x, count, out, s);
  return (boys_status)(rc < 0 ? BOYS_ERR_NMAX : rc);
}

}  // extern "C"
