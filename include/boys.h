/*
 * boys.h -- C ABI of the GB300 Boys-function library (libboys.so).
 *
 * The library evaluates the Boys functions (Sec. 1, Eq. "fn")
 *
 *     F_m(x) = int_0^1 t^{2m} exp(-x t^2) dt ,   m = 0..n_max,
 *
 * for large arrays of arguments with the paper's global approximation
 * (Sec. 2):  F_n = c_n / (x + Q~_n(x)^{n+1/2} e^{-x})^{n+1/2}  (Eq. "fq"),
 * Q~_n = q0 + q1 x + q2 x^2 u(x)/v(x) in root-product form (Eqs. "pqz", "pz",
 * "qz"), the switch to the asymptote c_n x^{-(n+1/2)} above the cut-off z_nb
 * (Eq. "limf1" and the cut-off equation of Sec. 2), and the downward
 * recursion of Eq. "r" that reuses e^{-x}.  The coefficients are the
 * library's own constrained minimax fits (Eq. "e" with the constraints of
 * Eqs. "q0", "q1", "qa", "qb").
 *
 * Conventions shared by every entry point:
 *  - Layout: out is row-major [count, n_max+1]; out[i*(n_max+1) + m] = F_m(x[i]).
 *  - Pointers named x, out, F, g, grad_x, offsets, ... are DEVICE pointers
 *    (cudaMalloc, managed or pinned-and-mapped memory), naturally aligned for
 *    their element type, and the output must not overlap an input.  The caller
 *    owns every buffer; the library never allocates, frees or synchronises in
 *    the evaluation calls (except where a function says otherwise).
 *  - stream: a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Work is enqueued asynchronously.
 *  - Domain (the paper's error measure is over x >= 0): x < 0 or NaN gives NaN
 *    in every column, x = +inf gives 0, x = 0 (or -0) gives 1/(2m+1).
 *  - Errors: every call returns a boys_status; host-checkable argument errors
 *    are reported before anything is launched; count == 0 is a no-op that
 *    returns BOYS_OK.  A launch failure is reported as BOYS_ERR_CUDA (the CUDA
 *    error is left for cudaGetLastError).
 */
#ifndef BOYS_GB300_H
#define BOYS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BOYS_OK = 0,
    BOYS_ERR_NULL = 1,      /* a required pointer is NULL */
    BOYS_ERR_COUNT = 2,     /* count < 0, or count*(n_max+1) overflows int64 */
    BOYS_ERR_NMAX = 3,      /* n_max outside [0, boys_max_n(precision)] */
    BOYS_ERR_ALIGN = 4,     /* a pointer is not aligned to its element size */
    BOYS_ERR_WORKSPACE = 5, /* caller workspace too small */
    BOYS_ERR_CUDA = 6,      /* a CUDA call failed */
    BOYS_ERR_ARG = 7,       /* other invalid argument (e.g. host memory, bad stride) */
    BOYS_ERR_DEVICE = 8     /* the current device is not sm_103 (GB300) */
} boys_status;

/* Human-readable name of a status code (static string). */
const char *boys_status_string(int status);

/* Largest n_max supported for 53-bit (double) or 24-bit (float) work. */
int boys_max_n(int precision_bits);

/* The cut-off z_{n,b} of Sec. 2 the library uses for order n and b = 53 or 24
 * bits, i.e. the root of R(n+1/2, z) = 2^-b; NaN for unsupported (n, b). */
double boys_cutoff(int n, int precision_bits);

/* The order n_top whose approximation the double path evaluates for a given
 * n_max (Sec. 3 suggests computing F_{n+1} and recursing down for a few more
 * bits); -1 if n_max is unsupported. */
int boys_top_order_f64(int n_max);

/* FP64 forward (Sec. 2, Eqs. "fq", "pqz", "r"; cut-off switch of Sec. 2).
 *   x:     device, [count] doubles
 *   out:   device, [count, n_max+1] doubles, row-major
 * Max relative error against the exact F_m: 2e-14 for every m. */
boys_status boys_eval_f64(const double *x, int64_t count, int n_max, double *out, void *stream);

/* The order n_top whose approximation the float path evaluates for n_max
 * (n_max itself up to 8, n_max + 1 above); -1 if unsupported. */
int boys_top_order_f32(int n_max);

/* FP32 forward: the same method in single precision, with float coefficients
 * from fits one order above the paper's single-precision column and the
 * error-amplifying steps (q0 + q1 x, Q^{n+1/2}, e^{-x}, D, D^{-(n+1/2)}) in
 * float-float arithmetic (Sec. 3 suggests extra precision for full 24-bit
 * results).
 *   x:   device, [count] floats
 *   out: device, [count, n_max+1] floats, row-major
 * Max relative error against the exact F_m at the float argument: 2e-6 for
 * every m where F_m >= FLT_MIN; below FLT_MIN (subnormal results) the error
 * is within 2e-6 relative plus one subnormal unit. */
boys_status boys_eval_f32(const float *x, int64_t count, int n_max, float *out, void *stream);

/* Device workspace, in bytes, that boys_eval_f64_host needs to stream chunks
 * of `chunk` arguments (rounded up to 2048) with double buffering; 0 for
 * invalid arguments. */
size_t boys_eval_f64_host_workspace(int n_max, int64_t chunk);

/* FP64 forward from and to HOST memory (the same results as boys_eval_f64).
 *   x_host:    host (or device), [count] doubles
 *   out_host:  host (or device), [count, n_max+1] doubles, row-major
 *   workspace: device memory, 256-byte aligned, ws_bytes long; the arguments
 *              are processed in chunks of ws_bytes / (16 (n_max+2)) (at least
 *              2048, else BOYS_ERR_WORKSPACE), each copied in, evaluated and
 *              copied out; the copies of one chunk run on the copy engines
 *              while the neighbouring chunk is evaluated.
 * Page-locked (pinned) host memory is needed for the copies to overlap; with
 * pageable memory the driver copies synchronously.  The library keeps one
 * helper stream and two events per device (created on the first call) to
 * overlap the chunks; work on `stream` that follows the call waits for all of
 * it.  Asynchronous: synchronise `stream` before reading out_host. */
boys_status boys_eval_f64_host(const double *x_host, int64_t count, int n_max, double *out_host, void *workspace,
                               size_t ws_bytes, void *stream);

/* Workspace size and host-buffer entry point of the float path; the same
 * contract as the double versions above, with float arrays. */
size_t boys_eval_f32_host_workspace(int n_max, int64_t chunk);
boys_status boys_eval_f32_host(const float *x_host, int64_t count, int n_max, float *out_host, void *workspace,
                               size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BOYS_GB300_H */
