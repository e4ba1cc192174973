/*
 * boys_oracle.c -- plain, slow, long-double CPU evaluator of the Boys functions.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes is the plain definition (Sec. 1, Eq. "fn"):
 *
 *     F_n(x) = int_0^1 t^{2n} exp(-x t^2) dt ,   x >= 0,
 *
 * not the paper's approximation.  Three independent evaluations are provided:
 *
 *   (1) x = 0:       F_n(0) = 1/(2n+1)  (the integral of t^{2n}).
 *   (2) 0 < x <= X_S: the all-positive series obtained by integrating the
 *       definition by parts repeatedly,
 *           F_n(x) = e^{-x} sum_{k>=0} (2x)^k / prod_{j=0..k} (2n+2j+1),
 *       for the highest order, then the downward recursion of Eq. "r"
 *       (Sec. 2), which the paper states is stable.  Integrating Eq. "fn" by
 *       parts gives  F_{m-1} = (2x F_m + e^{-x}) / (2m-1);  the printed
 *       Eq. "r" has 2m+1 in the denominator, which contradicts F_m(0) =
 *       1/(2m+1) and is read as a typesetting slip.
 *   (3) x > X_S:     F_0 = (1/2) sqrt(pi/x) erf(sqrt(x)) and the same recursion
 *       run upward, F_{m+1} = ((2m+1) F_m - e^{-x}) / (2x), stable for x > m.
 *   (4) cross-check: Gauss-Legendre quadrature of the definition itself.
 *
 * Domain: the paper's error measure (Eq. "e") is over x >= 0.  Outside it
 * (x < 0 or NaN) every column is NaN; x = +inf gives 0 (the limit of Eq.
 * "limf1").
 *
 * The cut-off z_nb of Sec. 2 solves  z^{n+1/2} F_n(z) / c_n = 1 - 2^{-b}.
 * Because  x^{n+1/2} F_n(x) / c_n  is the regularized lower incomplete gamma
 * function P(n+1/2, x), the equation is  R(n+1/2, z) = 2^{-b}  with
 * R = 1 - P, and R for half-integer order is the positive sum
 *     R(n+1/2, x) = erfc(sqrt x) + e^{-x} sum_{k=0}^{n-1} x^{k+1/2} / Gamma(k+3/2),
 * which this file evaluates without cancellation and solves by bisection.
 *
 * Precision: long double (64-bit significand on x86-64, IEEE binary128 on
 * AArch64), far below the 2e-14 / 2e-6 tolerances the library is checked at.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>

typedef long double ld;

#define ORACLE_OK 0
#define ORACLE_EINVAL 1

static const ld LD_PI = 3.141592653589793238462643383279502884197L;

/* Largest argument handled by the series; above it the erf/upward branch. */
static ld series_limit(int n_top)
{
    ld a = (ld)(2 * n_top + 40);
    return a > 120.0L ? a : 120.0L;
}

/* Branch (2): F_n(x) by the all-positive series, 0 < x. */
static ld series_fn(int n, ld x)
{
    const ld two_x = 2.0L * x;
    ld term = 1.0L / (ld)(2 * n + 1);
    ld sum = term;
    const ld tiny = LDBL_EPSILON * 0x1p-8L;
    for (long k = 1; k < 10000000L; ++k) {
        const ld denom = (ld)(2L * n + 2L * k + 1L);
        term *= two_x / denom;
        sum += term;
        /* past the peak (ratio <= 1/2), the tail is below one term */
        if (two_x <= 0.5L * denom && term <= sum * tiny)
            break;
    }
    return expl(-x) * sum;
}

/* Fill row[0..n_max] with F_0..F_{n_max} at one argument. */
static void eval_row(ld x, int n_max, ld *row)
{
    if (isnan(x) || x < 0.0L) {
        for (int m = 0; m <= n_max; ++m)
            row[m] = NAN;
        return;
    }
    if (isinf(x)) {
        for (int m = 0; m <= n_max; ++m)
            row[m] = 0.0L;
        return;
    }
    if (x == 0.0L) {
        for (int m = 0; m <= n_max; ++m)
            row[m] = 1.0L / (ld)(2 * m + 1);
        return;
    }
    const ld e = expl(-x);
    if (x <= series_limit(n_max)) {
        row[n_max] = series_fn(n_max, x);
        for (int m = n_max; m >= 1; --m)
            row[m - 1] = (2.0L * x * row[m] + e) / (ld)(2 * m - 1);
    } else {
        row[0] = 0.5L * sqrtl(LD_PI / x) * erfl(sqrtl(x));
        for (int m = 0; m < n_max; ++m)
            row[m + 1] = ((ld)(2 * m + 1) * row[m] - e) / (2.0L * x);
    }
}

int boys_oracle_precision_bits(void) { return LDBL_MANT_DIG; }

/* out[i*(n_max+1) + m] = F_m(x[i]), long double in and out. */
int boys_oracle_eval_ld(const ld *x, int64_t count, int n_max, ld *out)
{
    if (count < 0 || n_max < 0 || (count > 0 && (!x || !out)))
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < count; ++i)
        eval_row(x[i], n_max, out + i * (int64_t)(n_max + 1));
    return ORACLE_OK;
}

/* Same, double in and out (each value rounded once from long double). */
int boys_oracle_eval(const double *x, int64_t count, int n_max, double *out)
{
    if (count < 0 || n_max < 0 || (count > 0 && (!x || !out)))
        return ORACLE_EINVAL;
    ld row[1024];
    if (n_max >= 1024)
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < count; ++i) {
        eval_row((ld)x[i], n_max, row);
        for (int m = 0; m <= n_max; ++m)
            out[i * (int64_t)(n_max + 1) + m] = (double)row[m];
    }
    return ORACLE_OK;
}

/* Branch (2) alone for one order n (tests compare the branches). */
int boys_oracle_series_ld(const ld *x, int64_t count, int n, ld *out)
{
    if (count < 0 || n < 0 || (count > 0 && (!x || !out)))
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < count; ++i)
        out[i] = x[i] == 0.0L ? 1.0L / (ld)(2 * n + 1) : series_fn(n, x[i]);
    return ORACLE_OK;
}

/* Branch (3) alone: rows F_0..F_{n_max} from erf and upward recursion. */
int boys_oracle_erf_upward_ld(const ld *x, int64_t count, int n_max, ld *out)
{
    if (count < 0 || n_max < 0 || (count > 0 && (!x || !out)))
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < count; ++i) {
        ld *row = out + i * (int64_t)(n_max + 1);
        const ld xi = x[i];
        const ld e = expl(-xi);
        row[0] = 0.5L * sqrtl(LD_PI / xi) * erfl(sqrtl(xi));
        for (int m = 0; m < n_max; ++m)
            row[m + 1] = ((ld)(2 * m + 1) * row[m] - e) / (2.0L * xi);
    }
    return ORACLE_OK;
}

/* Gauss-Legendre nodes/weights on [-1, 1] by Newton on P_K. */
#define GL_K 24
static void gl_rule(ld *node, ld *weight)
{
    for (int i = 0; i < GL_K; ++i) {
        ld t = cosl(LD_PI * ((ld)i + 0.75L) / ((ld)GL_K + 0.5L));
        ld dp = 0.0L;
        for (int it = 0; it < 100; ++it) {
            ld p0 = 1.0L, p1 = t;
            for (int k = 2; k <= GL_K; ++k) {
                ld p2 = ((ld)(2 * k - 1) * t * p1 - (ld)(k - 1) * p0) / (ld)k;
                p0 = p1;
                p1 = p2;
            }
            dp = (ld)GL_K * (t * p1 - p0) / (t * t - 1.0L);
            ld dt = p1 / dp;
            t -= dt;
            if (fabsl(dt) <= LDBL_EPSILON * 0.5L)
                break;
        }
        {
            /* recompute the derivative at the converged node */
            ld p0 = 1.0L, p1 = t;
            for (int k = 2; k <= GL_K; ++k) {
                ld p2 = ((ld)(2 * k - 1) * t * p1 - (ld)(k - 1) * p0) / (ld)k;
                p0 = p1;
                p1 = p2;
            }
            dp = (ld)GL_K * (t * p1 - p0) / (t * t - 1.0L);
        }
        node[i] = t;
        weight[i] = 2.0L / ((1.0L - t * t) * dp * dp);
    }
}

/* Branch (4): quadrature of the definition for one order n.
 * x <= 1: integrate t^{2n} e^{-x t^2} over [0,1] directly.
 * x > 1 : substitute u = t sqrt(x):  F_n = x^{-(n+1/2)} int_0^{sqrt x} u^{2n} e^{-u^2} du,
 *         truncated where the integrand is below 1e-60 of its peak. */
int boys_oracle_quad_ld(const ld *x, int64_t count, int n, ld *out)
{
    if (count < 0 || n < 0 || (count > 0 && (!x || !out)))
        return ORACLE_EINVAL;
    ld node[GL_K], weight[GL_K];
    gl_rule(node, weight);
    for (int64_t i = 0; i < count; ++i) {
        const ld xi = x[i];
        ld acc = 0.0L;
        if (xi <= 1.0L) {
            const int panels = 8;
            for (int p = 0; p < panels; ++p) {
                const ld a = (ld)p / panels, b = (ld)(p + 1) / panels;
                const ld half = 0.5L * (b - a), mid = 0.5L * (a + b);
                for (int k = 0; k < GL_K; ++k) {
                    const ld t = mid + half * node[k];
                    acc += half * weight[k] * powl(t, 2 * n) * expl(-xi * t * t);
                }
            }
            out[i] = acc;
        } else {
            const ld sx = sqrtl(xi);
            ld upper = sqrtl((ld)n + 0.5L) + 12.0L;
            if (upper > sx)
                upper = sx;
            const ld width = 0.25L;
            const int panels = (int)ceill(upper / width);
            for (int p = 0; p < panels; ++p) {
                const ld a = p * width;
                ld b = (p + 1) * width;
                if (b > upper)
                    b = upper;
                const ld half = 0.5L * (b - a), mid = 0.5L * (a + b);
                for (int k = 0; k < GL_K; ++k) {
                    const ld u = mid + half * node[k];
                    acc += half * weight[k] * powl(u, 2 * n) * expl(-u * u);
                }
            }
            out[i] = acc * powl(xi, -((ld)n + 0.5L));
        }
    }
    return ORACLE_OK;
}

/* Gradient of  sum_m g[i, m] F_m(x_i)  with respect to x_i, using
 * dF_m/dx = -F_{m+1}  (differentiate Eq. "fn" under the integral):
 *     grad[i] = - sum_{m=0}^{n_max} g[i*g_row + m*g_col] F_{m+1}(x_i). */
int boys_oracle_grad(const double *x, const double *g, int64_t g_row, int64_t g_col, int64_t count,
                     int n_max, double *grad)
{
    if (count < 0 || n_max < 0 || n_max >= 1023 || (count > 0 && (!x || !g || !grad)))
        return ORACLE_EINVAL;
    ld row[1024];
    for (int64_t i = 0; i < count; ++i) {
        eval_row((ld)x[i], n_max + 1, row);
        ld acc = 0.0L;
        for (int m = 0; m <= n_max; ++m)
            acc += (ld)g[i * g_row + (int64_t)m * g_col] * row[m + 1];
        grad[i] = (double)(-acc);
    }
    return ORACLE_OK;
}

/* Long-double variant of the gradient (normalisation term included):
 * grad[i] = -sum g F_{m+1};  scale[i] = sum |g| F_{m+1}. */
int boys_oracle_grad_ld(const ld *x, const ld *g, int64_t g_row, int64_t g_col, int64_t count,
                        int n_max, ld *grad, ld *scale)
{
    if (count < 0 || n_max < 0 || n_max >= 1023 || (count > 0 && (!x || !g || !grad)))
        return ORACLE_EINVAL;
    ld row[1024];
    for (int64_t i = 0; i < count; ++i) {
        eval_row(x[i], n_max + 1, row);
        ld acc = 0.0L, mag = 0.0L;
        for (int m = 0; m <= n_max; ++m) {
            const ld gm = g[i * g_row + (int64_t)m * g_col];
            acc += gm * row[m + 1];
            mag += fabsl(gm) * row[m + 1];
        }
        grad[i] = -acc;
        if (scale)
            scale[i] = mag;
    }
    return ORACLE_OK;
}

/* R(n+1/2, x) = Gamma(n+1/2, x) / Gamma(n+1/2), x >= 0, as the positive sum
 * erfc(sqrt x) + e^{-x} sum_{k=0}^{n-1} x^{k+1/2} / Gamma(k+3/2). */
static ld upper_ratio(int n, ld x)
{
    if (n < 0 || !(x >= 0.0L))
        return NAN;
    const ld sx = sqrtl(x);
    ld acc = erfcl(sx);
    ld term = expl(-x) * sx / (0.5L * sqrtl(LD_PI)); /* x^{1/2} e^{-x} / Gamma(3/2) */
    for (int k = 0; k < n; ++k) {
        acc += term;
        term *= x / ((ld)k + 1.5L);
    }
    return acc;
}

int boys_oracle_upper_ratio_ld(int n, const ld *x, int64_t count, ld *out)
{
    if (count < 0 || n < 0 || (count > 0 && (!x || !out)))
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < count; ++i)
        out[i] = upper_ratio(n, x[i]);
    return ORACLE_OK;
}

/* Cut-off z_nb: the root of R(n+1/2, z) = 2^{-b}, by bisection (R decreases in z). */
double boys_oracle_cutoff(int n, int bits)
{
    if (n < 0 || bits <= 0 || bits > 200)
        return NAN;
    const ld target = ldexpl(1.0L, -bits);
    ld lo = 0.0L, hi = 1.0L;
    while (upper_ratio(n, hi) > target)
        hi *= 2.0L;
    for (int it = 0; it < 400; ++it) {
        const ld mid = 0.5L * (lo + hi);
        if (mid <= lo || mid >= hi)
            break;
        if (upper_ratio(n, mid) > target)
            lo = mid;
        else
            hi = mid;
    }
    return (double)(0.5L * (lo + hi));
}

/* c_n = (2n)! sqrt(pi) / (n! 2^{2n+1}) = Gamma(n+1/2)/2 (Sec. 2), by the
 * product form c_0 = sqrt(pi)/2, c_{m+1} = (m+1/2) c_m. */
int boys_oracle_c_ld(int n_max, ld *out)
{
    if (n_max < 0 || !out)
        return ORACLE_EINVAL;
    ld c = 0.5L * sqrtl(LD_PI);
    for (int m = 0; m <= n_max; ++m) {
        out[m] = c;
        c *= (ld)m + 0.5L;
    }
    return ORACLE_OK;
}
