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
 * results).  From n_max = 17 on (n_top >= 18), where the amplification
 * s^2 (T/D) stays large far out in x, the rational part of Q~ and its
 * coefficients are float-float too, the recursion's constants 1/(2m - 1) are
 * float pairs and the asymptote's product chain is compensated.
 * n_max <= boys_max_n(24) = 36.
 *   x:   device, [count] floats
 *   out: device, [count, n_max+1] floats, row-major
 * Max relative error against the exact F_m at the float argument: 2e-6 for
 * every m where F_m >= FLT_MIN; below FLT_MIN (subnormal results) the error
 * is within 2e-6 relative plus one subnormal unit. */
boys_status boys_eval_f32(const float *x, int64_t count, int n_max, float *out, void *stream);

/* FP64 adjoint: grad_x[i] = -sum_{m=0}^{n_max} g[i, m] F_{m+1}(x_i), the
 * gradient of sum_{i,m} g[i, m] F_m(x_i) with respect to x_i, because
 * differentiating Eq. "fn" under the integral gives dF_m/dx = -F_{m+1}.
 *   x:       device, [count] doubles (read only when F is NULL)
 *   F:       device, saved forward rows of at least n_max+2 columns
 *            (F_0..F_{n_max+1}), row-major with leading dimension ld_F >=
 *            n_max+2; column m+1 is read.  NULL: F_1..F_{n_max+1} are
 *            recomputed from x with the forward kernel of order n_max+1.
 *   g:       device; element (i, m) at g[i*g_row_stride + m*g_col_stride];
 *            strides are in elements, >= 0 (0 broadcasts, e.g. one weight
 *            vector shared by all rows)
 *   grad_x:  device, [count] doubles (overwritten)
 * n_max <= boys_max_n(53) - 1.  Relative error, normalised by
 * sum_m |g[i,m]| F_{m+1}(x_i): 1e-12.  Without F and with one weight vector
 * for all arguments (g_row_stride == 0, n_max <= 16), arguments above the
 * cut-off take the gradient of the asymptote as a polynomial in 1/x (Horner);
 * it differs from the saved-rows result by rounding only. */
boys_status boys_eval_backward_f64(const double *x, const double *F, int64_t ld_F, const double *g, int64_t g_row_stride,
                                   int64_t g_col_stride, int64_t count, int n_max, double *grad_x, void *stream);

/* FP64 forward with the two-point evaluation of Sec. 3 (Trick B): besides the
 * closed form at n_top (for m > n_bar), the closed form is also evaluated at
 * the top order of n_bar = n_max / 2 (for m <= n_bar), sharing e^{-x}; each
 * part has its own, shorter downward recursion.  The low orders come out
 * more accurate (e.g. F_0 at n_max = 36: about 5e-15 instead of 1.3e-14),
 * at the cost of a second closed form below the cut-off.  Arguments, layout
 * and bound (2e-14 for every m) as boys_eval_f64; n_max < 2 is the plain path. */
boys_status boys_eval_f64_two_point(const double *x, int64_t count, int n_max, double *out, void *stream);

/* Fused consumer: out[i] = sum_{m=0}^{n_max} c[i*c_row + m*c_col] F_m(x_i).
 * Integral codes use the Boys values at once, as inputs of a contraction or a
 * recurrence (Sec. 1: they are the special functions of one- and two-electron
 * integrals over Gaussians); evaluating that contraction inside the kernel
 * keeps the rows in registers, so only x, c and out touch memory.
 *   x:   device, [count] arguments
 *   c:   device coefficients; strides in elements, >= 0 (0 broadcasts one
 *        coefficient vector over all arguments)
 *   out: device, [count]
 * Same method and per-F_m accuracy as boys_eval_f64 / boys_eval_f32; the
 * contraction itself rounds in the working precision.  With one coefficient
 * vector for all arguments (c_row == 0; FP64 up to n_max = 16), arguments
 * above the cut-off take the contraction of the asymptote as a polynomial
 * in 1/x (Horner), without forming the row: the result differs from
 * contracting the rows by rounding only (a few ulp of sum_m |c_m| F_m). */
boys_status boys_eval_contract_f64(const double *x, int64_t count, int n_max, const double *c, int64_t c_row,
                                   int64_t c_col, double *out, void *stream);
/* The float contraction takes n_max <= 16 (else BOYS_ERR_NMAX): its sums and
 * Horner polynomials are plain FP32. */
boys_status boys_eval_contract_f32(const float *x, int64_t count, int n_max, const float *c, int64_t c_row,
                                   int64_t c_col, float *out, void *stream);

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

/* ---- ragged batches ----------------------------------------------------
 * R requests in one call, request r owning arguments x[offsets[r] ..
 * offsets[r+1]) and output rows out[out_offsets[r] .. out_offsets[r+1]) with
 * its own n_max[r] (0 <= n_max[r] <= boys_ragged_max_n()); the rows are laid
 * out as in boys_eval_f64, so out_offsets[r+1] - out_offsets[r] must equal
 * (offsets[r+1] - offsets[r]) * (n_max[r] + 1).  Same method and accuracy as
 * boys_eval_f64 (bitwise the same values for the same n_max).
 *   x:           device, x_size doubles
 *   offsets:     device, [R+1] int64 (argument offsets, non-decreasing)
 *   n_max:       device, [R] int32
 *   out_offsets: device, [R+1] int64 (element offsets into out)
 *   out:         device, out_size doubles
 *   workspace:   device, 256-byte aligned, >= boys_ragged_workspace_bytes(R)
 *   variant:     launch configuration (block size, tile) from
 *                boys_ragged_variant_info, or -1 for the default; the Python
 *                autotuner picks one by timing them
 * The request arrays live on the device, so they are validated there: a
 * request with a bad n_max, bad offsets or a range outside x_size/out_size
 * produces no values; it is counted (boys_ragged_errors) and, when its
 * output range lies inside [0, out_size), that range is filled with NaN.
 * The call enqueues one memset and two kernels (a one-block plan, which
 * also orders the requests by n_max so that the GPU works on one order at a
 * time, and the persistent evaluation), allocates nothing and never
 * synchronises, so it can be captured in a CUDA graph and replayed. */
size_t boys_ragged_workspace_bytes(int32_t num_requests);
int boys_ragged_max_n(void);
int boys_ragged_num_variants(void);
boys_status boys_ragged_variant_info(int variant, int *block, int *tile);
boys_status boys_eval_ragged_f64(const double *x, int64_t x_size, const int64_t *offsets, const int32_t *n_max,
                                 const int64_t *out_offsets, int32_t num_requests, double *out, int64_t out_size,
                                 void *workspace, size_t ws_bytes, int variant, void *stream);

/* Ragged evaluation for callers that cannot provide device scratch memory.
 *
 * The paper has no counterpart; this is a convenience of the library.
 * Callers that cannot allocate device memory -- e.g. a host whose device
 * memory is all held by its own pool and that forbids libraries from calling
 * cudaMalloc, or code with no device allocator at hand -- cannot pass the
 * workspace boys_eval_ragged_f64 needs.  This entry point takes the same
 * arguments minus the workspace and uses a fixed scratch array compiled into
 * the library instead; it calls no allocation routine.
 *   - At most BOYS_RAGGED_NOALLOC_MAX_REQUESTS requests (the array holds the
 *     counters, the tile prefix and the request order for that many: about
 *     768 KiB); more
 *     returns BOYS_ERR_WORKSPACE before anything is launched.
 *   - The array exists once per GPU that loads the library and stays
 *     allocated until the process exits.
 *   - The first call on a device looks up the array's device address (a
 *     one-time set-up per device, done with that device current); make that
 *     first call before any stream capture.
 *   - Every call shares the array, which keeps the last call's contents; the
 *     call clears what must start at zero itself.  Calls whose work overlaps
 *     on the GPU race on the array: order them (e.g. one stream).
 *   - The count of invalid requests that boys_ragged_errors reads from a
 *     workspace is not available here (the array's address stays inside the
 *     library): an invalid request shows only as its output range filled
 *     with NaN, where that range lies inside [0, out_size).
 * Results are those of boys_eval_ragged_f64, bit for bit. */
#define BOYS_RAGGED_NOALLOC_MAX_REQUESTS 65536
boys_status boys_eval_ragged_f64_noalloc(const double *x, int64_t x_size, const int64_t *offsets, const int32_t *n_max,
                                         const int64_t *out_offsets, int32_t num_requests, double *out,
                                         int64_t out_size, int variant, void *stream);

/* Number of invalid requests seen by the last boys_eval_ragged_f64 that used
 * this workspace.  Synchronises `stream` (the call that filled the
 * workspace must have been enqueued on it or before it). */
boys_status boys_ragged_errors(const void *workspace, int64_t *n_bad_requests, void *stream);

/* Workspace size and host-buffer entry point of the float path; the same
 * contract as the double versions above, with float arrays. */
size_t boys_eval_f32_host_workspace(int n_max, int64_t chunk);
boys_status boys_eval_f32_host(const float *x_host, int64_t count, int n_max, float *out_host, void *workspace,
                               size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BOYS_GB300_H */
