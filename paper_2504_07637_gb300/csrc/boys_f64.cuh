// FP64 forward path.
//
// GB300 retires FP64 at about 1/64 of its FP32 rate, so this path is bound by
// the FP64 pipe, not by HBM: every design choice below removes FP64
// instructions.
//  * Compaction: each tile of arguments is split into a below-cut-off list
//    (closed form: at n_max = 8 about 50 FP64 operations, a division, an
//    exponential and two reciprocal square roots) and an above-cut-off list
//    (asymptote), and warps take 32 entries of one list at a time, so no warp
//    pays for both branches (with arguments mixed at random, nearly every
//    warp of a plain one-argument-per-thread kernel would).
//  * The downward recursion and the asymptote's upward product chain run on
//    64-bit integer significands (boys_sig64.cuh), on integer pipes that an
//    FP64-bound kernel leaves idle; the FP64 pipe keeps the closed form.
//  * Classification, the factor 2 of the recursion and the final scaling of
//    the exponential are integer operations on the bit patterns.
//  * e^{-x} is Tang's table-driven method (ACM TOMS 15(2), 1989): 2^(k/64)
//    from a shared-memory table times a degree-5 polynomial on
//    |r| <= ln2/128, about 10 FP64 operations.
//  * Half-integer powers use the reciprocal square root where the rounding
//    budget allows it.
//  * From n_max = 12 on, the rows leave through a per-warp shared-memory
//    staging buffer, 16 orders of 32 rows at a time, in row order.  Rows
//    stored straight from registers touch 32 sectors per warp instruction,
//    and those stores back up into the instruction stream; at n_max = 36 the
//    stores, not the arithmetic, set the pace.
#pragma once

#include "boys_coeffs_f64.inc"
#include "boys_common.cuh"
#include "boys_sig64.cuh"

#include <climits>
#include <type_traits>

namespace boys {

// 2^(j/64), j = 0..63, for the exponential below
static __constant__ double kExp2Frac64[64] = BOYS_EXP2_FRAC64;
static __constant__ uint64_t kExp2Frac64Sig[64] = BOYS_EXP2_FRAC64_SIG;

// Row index of a lane without a list entry (rows of carried entries may be negative).
constexpr int kNoRow = INT_MIN;

static_assert(f64_top_order(kMaxNF64) <= BOYS_F64_TABLE_MAX_N, "fitted table too short");

// Compile-time loop: f(std::integral_constant<int, i>) for i = I, I + STEP, ... while i has not reached END.
template <int I, int END, int STEP, typename Fn>
__device__ __forceinline__ void static_for(Fn &&f) {
  if constexpr ((STEP > 0 && I < END) || (STEP < 0 && I > END)) {
    f(std::integral_constant<int, I>{});
    static_for<I + STEP, END, STEP>(f);
  }
}

__device__ __forceinline__ double twice(double x) {
  // exact 2x for normal x; for |x| below the normal range the result is a
  // tiny normal number, which leaves fma(2x, F, e^{-x}) unchanged
  return __longlong_as_double(__double_as_longlong(x) + (1LL << 52));
}

// e^{-x} for 0 <= x <= 700 by Tang's table-driven method:
//   -x = (k/64) ln2 + r,  k = round(-x 64/ln2),  |r| <= ln2/128,
//   e^{-x} = 2^(k>>6) * 2^((k&63)/64) * (1 + p(r)),  p(r) = r + r^2/2 + ... + r^5/120.
// ln2/64 is split in two parts (Cody and Waite) so that k*L1 is exact.
__device__ __forceinline__ double exp_neg(double x, const double *__restrict__ tab64) {
  constexpr double kShift = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer in the low bits
  constexpr double kInvL = 92.332482616893656;   // 64 / ln2
  constexpr double kL1 = 0.010830424696251839;   // ln2/64, 39 significant bits
  constexpr double kL2 = -2.693663207127318e-15; // ln2/64 - kL1
  const double a = -x;
  double kd = fma(a, kInvL, kShift);
  const int k = __double2loint(kd);
  kd -= kShift;
  double r = fma(kd, -kL1, a);
  r = fma(kd, -kL2, r);
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(r, p, 1.0 / 6.0);
  p = fma(r, p, 0.5);
  p = fma(r, p, 1.0);
  p = p * r;
  const double t = tab64[k & 63];
  const double res = fma(t, p, t);
  return __longlong_as_double(__double_as_longlong(res) + ((long long)(k >> 6) << 52));
}

// The exponential's tables in shared memory: 2^(j/64) as doubles (exp_neg)
// and as 64-bit significands (sig64_exp_neg).
struct F64ExpTab {
  double d[64];
  uint64_t s[64];
};

// e^{-x} as a double and as a 64-bit significand (s, e).  INT: by
// sig64_exp_neg on the integer pipes (0 <= x < 128: the closed form's
// arguments), rounded once to d; otherwise exp_neg in FP64, and (s, e) its
// bits.  Tang's exponential costs about 9 DFMA times on the FP64 pipe
// (f64_int_exp says where the integer form is used).
struct F64E {
  double d;
  uint64_t s;
  int e;
};
template <bool INT>
__device__ __forceinline__ F64E f64_exp_neg_both(const double x, const F64ExpTab &tab) {
  F64E r;
  if constexpr (INT) {
    sig64_exp_neg((uint64_t)__double_as_longlong(x), tab.s, r.s, r.e);
    r.d = __longlong_as_double((long long)sig64_round_bits(r.s, r.e));
  } else {
    r.d = exp_neg(x, tab.d);
    const uint64_t b = (uint64_t)__double_as_longlong(r.d);
    r.s = sig64_of_bits(b);
    r.e = exp_of_bits(b);
  }
  return r;
}

// The float approximation that seeds the Newton steps: one special-function
// instruction (relative error about 2^-23 on [1, 4)).
__device__ __forceinline__ float rsqrt_approx_f32(float a) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

// 1/sqrt(v) for a positive normal double v as a Sig64 within 2^-60, by
// Newton steps on the integer pipes (boys_sig64.cuh) from a float
// approximation for v's leading bits.  In FP64 a reciprocal square root
// costs about 5 FMA times on the FP64 pipe, which bounds most kernels; this
// takes about 70 integer instructions.
__device__ __forceinline__ void f64_rsqrt_sig(const double v, uint64_t &s, int &e) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  int k;
  const uint32_t ab = sig64_rsqrt_reduce(b, k);
  sig64_rsqrt(b, __float_as_uint(rsqrt_approx_f32(__uint_as_float(ab))), s, e);
}
// nonzero, finite and not subnormal
__device__ __forceinline__ bool f64_is_normal(const double v) {
  return ((((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff) - 1ull) < 2046ull;
}
// the double nearest s 2^(e - 63) (positive), if it is normal
__device__ __forceinline__ bool sig64_to_double(const uint64_t s, const int e, double &v) {
  v = __longlong_as_double((long long)sig64_round_bits(s, e));
  return (unsigned)(e + 1022) <= 2045u;
}

// Below the cut-off z_{NTOP,53} (Sec. 2): with s = NTOP + 1/2,
//   Q   = q0 + q1 x + q2 x^2 u(x)/v(x)      (Eq. "pqz"; u, v root products, Eqs. "pz"/"qz")
//   D   = x + Q^NTOP sqrt(Q) e^{-x}          (Eq. "fq")
//   F_NTOP = c_NTOP D^{-s}
//   F_{m-1} = (2x F_m + e^{-x}) / (2m-1)     (Eq. "r", same e^{-x}; the printed
//                                             denominator 2m+1 is read as 2m-1)
// Whether the closed form takes its reciprocal square roots from integer
// Newton steps (f64_rsqrt_sig): below n_max = 12 and in the two-point rows,
// whose kernels the FP64 pipe bounds.  The one-point rows from n_max = 12 on
// are bound by issue and latency instead, and the extra integer work cost
// them 1-4% (n_max = 16: 232.0 -> 229.6, 36: 280.4 -> 270.2 G values/s),
// against +21% at n_max = 4 (102.6 -> 123.7), +11.5% for the staged rows of
// n_max = 8 (155.0 -> 172.9) and two-point n_max = 36 (187.4 -> 209.0).  The
// rule depends on the order only, so rows, contractions, gradients and ragged
// requests of one order share their arithmetic bit for bit.
__host__ __device__ constexpr bool f64_int_rsqrt(int n_max, bool two) { return two || n_max < 12; }

// Whether e^{-x} comes from sig64_exp_neg (integer pipes) instead of the FP64
// table method: for the one-point rows up to n_max = 5, where the FP64 pipe
// binds hardest (n_max = 0: 36.4 -> 44.6 G values/s, 4: 141.9 -> 157.9, 5:
// 163.2 -> 178.3), and from n_max = 12 on, whose closed form stays in FP64
// (12: 207.0 -> 210.4, 16: 228.8 -> 235.7, 20 to 36: +0.1 to +0.4%).  From
// n_max = 6 to 11, with the closed form's tail on the integer pipes, and in
// the two-point rows the integer exponential measured slower or no faster
// (n_max = 6: 178.6 -> 170.5, 7: 197.9 -> 198.7, 8: 183.4 -> 180.3, 11:
// -0.6%, two-point n_max = 16: -1.7%, 36: +2.6%).  Again a rule of the order
// only.
__host__ __device__ constexpr bool f64_int_exp(int n_max, bool two) { return !two && (n_max <= 5 || n_max >= 12); }

// F_NTOP(x) by the closed form of Eq. "fq", given e = e^{-x}.  Q~ (the root
// products and u/v) and e^{-x} are FP64 either way.  INT: everything after
// Q on 64-bit significands, rounded once at the end: T = Q^NTOP Q r_Q e^{-x}
// with r_Q = 1/sqrt(Q), D = x + T, r_D = 1/sqrt(D) (integer Newton steps,
// f64_rsqrt_sig), and F = c r_D (r_D^2)^NTOP; all terms are positive, and the
// significands' exponents are plain integers, so neither Q^NTOP nor D^-NTOP
// can leave a range.  Otherwise in FP64: rsqrt(D)^{2 NTOP + 1} up to
// n_top = 13, else (1/D)^NTOP sqrt(1/D) (also the fallback for operands
// outside the normal range).  An integer reciprocal for u/v measured no
// faster than the FP64 division.
template <int NTOP>
__device__ __forceinline__ double f64_closed_form_tail_fp64(const double x, const double q, const double e) {
  using Tab = BoysF64<NTOP>;
  const double T = (ipow<NTOP>(q) * (q * rsqrt(q))) * e;
  const double D = x + T;
  if constexpr (NTOP <= 13) {
    const double rs = rsqrt(D);  // D^{-s} = rs^{2 NTOP + 1}
    return (Tab::kC * rs) * ipow<NTOP>(rs * rs);
  } else {
    const double w = 1.0 / D;  // D^{-s} = w^NTOP sqrt(w)
    return (Tab::kC * ipow<NTOP>(w)) * (w * rsqrt(w));
  }
}

template <int NTOP, bool INT>
__device__ __forceinline__ double f64_closed_form(const double x, const F64E &ex) {
  const double e = ex.d;
  using Tab = BoysF64<NTOP>;
  double u, v;
  Tab::uv(x, u, v);
  const double r = u / v;
  const double p = (Tab::kQ2 * x) * x;
  const double q = fma(p, r, fma(Tab::kQ1, x, Tab::kQ0));
  if constexpr (INT) {
    if (q > 0.0 && f64_is_normal(q) && f64_is_normal(e)) {
      const uint64_t qb = (uint64_t)__double_as_longlong(q);
      const uint64_t sq = sig64_of_bits(qb);
      const int eq = exp_of_bits(qb);
      uint64_t sr, st = sq;
      int er, et = eq;
      f64_rsqrt_sig(q, sr, er);  // r_Q
      sig64_pow<NTOP>(st, et);   // Q^NTOP
      sig64_mul(st, et, sq, eq);
      sig64_mul(st, et, sr, er);  // Q^(NTOP + 1/2)
      sig64_mul(st, et, ex.s, ex.e);
      if (f64_is_normal(x)) {  // D = x + T (x >= 0; zero and subnormal x add nothing)
        const uint64_t xb = (uint64_t)__double_as_longlong(x);
        sig64_add(st, et, sig64_of_bits(xb), exp_of_bits(xb));
      }
      uint64_t sd, sw;
      int ed, ew;
      sig64_rsqrt_sig(st, et, __float_as_uint(rsqrt_approx_f32(__uint_as_float(sig64_rsqrt_seed_arg(st, et)))), sd,
                      ed);  // r_D
      sw = sd;
      ew = ed;
      sig64_mul(sw, ew, sd, ed);  // w = 1/D
      sig64_pow<NTOP>(sw, ew);
      sig64_mul(sw, ew, sd, ed);  // D^{-s}
      const uint64_t cb = (uint64_t)__double_as_longlong(Tab::kC);
      sig64_mul(sw, ew, sig64_of_bits(cb), exp_of_bits(cb));
      double F;
      if (sig64_to_double(sw, ew, F)) return F;
    }
  }
  return f64_closed_form_tail_fp64<NTOP>(x, q, e);
}

// Constants of the integer loops that run over orders at run time, indexed
// by the order m: 1/(2m - 1) for the recursion (m >= 1) and
// prod_{k<=m} (k - 1/2) for the asymptote's chain.
constexpr int kSig64TabLen = BOYS_F64_TABLE_MAX_N + 1;
struct Sig64Tab {
  uint64_t s[kSig64TabLen];
  int e[kSig64TabLen];
};
__host__ __device__ constexpr Sig64Tab make_sig64_tab(bool recip) {
  Sig64Tab t{};
  for (int m = 0; m < kSig64TabLen; ++m) {
    const Sig64 v = recip ? recip_odd(m == 0 ? 1 : 2 * m - 1) : half_odd_product(m);
    t.s[m] = v.s;
    t.e[m] = v.e;
  }
  return t;
}
static __constant__ Sig64Tab kRecipOddTab = make_sig64_tab(true);
static __constant__ Sig64Tab kHalfOddTab = make_sig64_tab(false);

// The downward recursion's state on the integer pipes (boys_sig64.cuh):
// F_m, 2x and e^{-x} as 64-bit significands.  One step,
// F_{m-1} = (2x F_m + e^{-x}) (1/(2m - 1)), is a product, an aligned sum of
// two positive numbers and a product with a constant; F_m is rounded to a
// double only where it is stored.  For x = 0 (twice(x) is then 2^-1022) the
// product is shifted out of the sum, as in FP64.
struct Sig64Down {
  uint64_t sf, sx, se;
  int ef, ex, ee;
  __device__ __forceinline__ void start(const double f, const double tx, const F64E &e) {
    const uint64_t fb = __double_as_longlong(f), xb = __double_as_longlong(tx);
    sf = sig64_of_bits(fb);
    ef = exp_of_bits(fb);
    sx = sig64_of_bits(xb);
    ex = exp_of_bits(xb);
    se = e.s;
    ee = e.e;
  }
  // F_{M-1} from F_M
  template <int M>
  __device__ __forceinline__ void step() {
    constexpr Sig64 k = recip_odd(2 * M - 1);
    sig64_mul(sf, ef, sx, ex);
    sig64_add(sf, ef, se, ee);
    if constexpr (M > 1) sig64_mul(sf, ef, k.s, k.e);
  }
  // the same for an order m >= 1 known at run time (for m = 1 the factor 1
  // clears the significand's last bit, a relative change below 2^-63)
  __device__ __forceinline__ void step_rt(const int m) {
    const uint64_t ks = kRecipOddTab.s[m];
    const int ke = kRecipOddTab.e[m];
    sig64_mul(sf, ef, sx, ex);
    sig64_add(sf, ef, se, ee);
    sig64_mul(sf, ef, ks, ke);
  }
  __device__ __forceinline__ double value() const { return __longlong_as_double((long long)sig64_round_bits(sf, ef)); }
};

// Whether an unstaged kernel (rows below n_max = 12, the fused contraction,
// the gradient) runs its recursion on the integer pipes, by the number of
// steps it unrolls per list entry.  An integer step is about 36 instructions
// against the FP64 step's 2: unrolled over all 41 steps at n_max = 36, with
// two entries per lane, the row kernels fell from 190 to 139 G values/s,
// presumably as their code (about 80 KB) outgrew the instruction cache.  The
// staged one-point row kernels (n_max >= 12) loop over chunks of orders
// instead (f64_recurse_staged) and always take the integer pipes: n_max = 36
// then ran at 202 G values/s (190 with the FP64 recursion).
__host__ __device__ constexpr bool f64_int_recursion(int steps) { return steps <= 18; }

// Eq. "r" from F_TOP (in f) down to F_LO, storing F_m for m <= NMAX: on the
// integer pipes (INT), else in FP64.
template <int TOP, int LO, int NMAX, bool INT = f64_int_recursion(TOP - LO)>
__device__ __forceinline__ void f64_recurse(double f, const double tx, const F64E &e, double (&F)[NMAX + 1]) {
  if constexpr (!INT) {
#pragma unroll
    for (int m = TOP; m > LO; --m) {
      if (m <= NMAX) F[m] = f;
      f = fma(tx, f, e.d) * (1.0 / double(2 * m - 1));
    }
    if (LO <= NMAX) F[LO] = f;
  } else {
    if constexpr (TOP <= NMAX) F[TOP] = f;
    if constexpr (TOP > LO) {
      Sig64Down r;
      r.start(f, tx, e);
      static_for<TOP, LO, -1>([&](auto mc) {
        constexpr int m = decltype(mc)::value;
        r.template step<m>();
        if constexpr (m - 1 <= NMAX) F[m - 1] = r.value();
      });
    }
  }
}

template <int NTOP, int NMAX>
__device__ __forceinline__ void f64_formula(const double x, double (&F)[NMAX + 1], const F64ExpTab &tab) {
  constexpr bool INT = f64_int_rsqrt(NMAX, false);
  const F64E e = f64_exp_neg_both<f64_int_exp(NMAX, false)>(x, tab);
  f64_recurse<NTOP, 0, NMAX>(f64_closed_form<NTOP, INT>(x, e), twice(x), e, F);
}

// Order n_bar of the two-point evaluation: the lower half of the orders.
__host__ __device__ constexpr int f64_two_point_nbar(int n_max) { return n_max / 2; }

// Two-point evaluation (Trick B of Sec. 3): the closed form at two orders,
// NTOP for m > NBAR and NTOP_LO (>= NBAR) for m <= NBAR, with one recursion
// each and one shared e^{-x}; the low orders then carry the error of a short
// recursion from a low order instead of a long one from the top.
template <int NTOP, int NTOP_LO, int NBAR, int NMAX>
__device__ __forceinline__ void f64_formula_two(const double x, double (&F)[NMAX + 1], const F64ExpTab &tab) {
  static_assert(NBAR < NMAX && NTOP_LO >= NBAR && NTOP_LO < NTOP, "orders");
  constexpr bool INT = f64_int_recursion(NTOP - NBAR - 1 + NTOP_LO);
  const F64E e = f64_exp_neg_both<f64_int_exp(NMAX, true)>(x, tab);
  const double tx = twice(x);
  f64_recurse<NTOP, NBAR + 1, NMAX, INT>(f64_closed_form<NTOP, true>(x, e), tx, e, F);
  double lo[NBAR + 1];
  f64_recurse<NTOP_LO, 0, NBAR, INT>(f64_closed_form<NTOP_LO, true>(x, e), tx, e, lo);
#pragma unroll
  for (int m = 0; m <= NBAR; ++m) F[m] = lo[m];
}

// Above the cut-off (or x negative, infinite or NaN): the asymptote of
// Eq. "limf1", within 2^-53 of F_m for every m <= NTOP there, built upward
// F_0 = c_0 / sqrt(x), F_m = F_{m-1} (m - 1/2) / x so that high orders
// underflow gracefully.  Negative x and NaN give NaN through rsqrt.
template <int NMAX>
__device__ __forceinline__ void f64_asymptote_fp64(const double x, double (&F)[NMAX + 1]) {
  const double rs = rsqrt(x);
  double f = 0.88622692545275801365 * rs;  // c_0 = sqrt(pi)/2
  F[0] = f;
  if constexpr (NMAX >= 1) {
    const double y = NMAX <= 12 ? rs * rs : 1.0 / x;
#pragma unroll
    for (int m = 1; m <= NMAX; ++m) {
      f = f * ((double(m) - 0.5) * y);
      F[m] = f;
    }
  }
}

// x > 0 below the bound of the integer chain for rows up to NMAX (this
// excludes negative x, NaN and +inf).
template <int NMAX>
__device__ __forceinline__ bool sig64_chain_ok(const double x) {
  return (unsigned long long)__double_as_longlong(x) < sig64_chain_xmax_bits(NMAX);
}

// The start of the asymptote on the integer pipes, for x above the cut-off
// with sig64_chain_ok<n_max>(x): r = 1/sqrt(x) by sig64_rsqrt (seeded by
// the float rsqrtf of x's leading bits), then F_0 = c_0 r and y = r^2 = 1/x
// as 64-bit significands (within 2^-59 of their values); F_0 rounded to a
// double is returned.  In FP64 these cost a reciprocal square root and, for
// the high orders' y, a division: about 5 and 7.6 FMA times on the FP64
// pipe, which bounds the kernels.
__device__ __forceinline__ double f64_asymptote_start(const double x, uint64_t &sf, int &ef, uint64_t &sy, int &ey) {
  uint64_t sr;
  int er;
  f64_rsqrt_sig(x, sr, er);
  sy = sr;
  ey = er;
  sig64_mul(sy, ey, sr, er);
  sf = kSig64C0s;
  ef = kSig64C0e;
  sig64_mul(sf, ef, sr, er);
  return __longlong_as_double((long long)sig64_round_bits(sf, ef));
}

// The asymptote of f64_asymptote_fp64 on the integer pipes (boys_sig64.cuh):
// F_0 and y = 1/x from f64_asymptote_start, then z_m = F_0 y^m and
// F_m = z_m prod_{k<=m} (k - 1/2) as 64-bit significands, each F_m rounded
// once.  Requires sig64_chain_ok<NMAX>(x).
struct Sig64Chain {
  uint64_t s, sy;
  int e, ey;
  // F_0 (returned) and the chain's start
  __device__ __forceinline__ double start(const double x) { return f64_asymptote_start(x, s, e, sy, ey); }
  // z_m from z_{m-1}, and F_m
  template <int M>
  __device__ __forceinline__ double next() {
    constexpr Sig64 h = half_odd_product(M);
    sig64_mul(s, e, sy, ey);
    uint64_t w = s;
    int ew = e;
    sig64_mul(w, ew, h.s, h.e);
    return __longlong_as_double((long long)sig64_round_bits(w, ew));
  }
  // the same for an order m >= 1 known at run time
  __device__ __forceinline__ double next_rt(const int m) {
    sig64_mul(s, e, sy, ey);
    uint64_t w = s;
    int ew = e;
    sig64_mul(w, ew, kHalfOddTab.s[m], kHalfOddTab.e[m]);
    return __longlong_as_double((long long)sig64_round_bits(w, ew));
  }
};

template <int NMAX>
__device__ __forceinline__ void f64_asymptote_int(const double x, double (&F)[NMAX + 1]) {
  Sig64Chain ch;
  F[0] = ch.start(x);
  if constexpr (NMAX >= 1) {
    static_for<1, NMAX + 1, 1>([&](auto mc) {
      constexpr int m = decltype(mc)::value;
      F[m] = ch.template next<m>();
    });
  }
}

// The asymptote row: on the integer pipes where the chain's range allows
// (every argument of the benchmark distributions), else in FP64.
template <int NMAX>
__device__ __forceinline__ void f64_asymptote(const double x, double (&F)[NMAX + 1]) {
  if (sig64_chain_ok<NMAX>(x)) {
    f64_asymptote_int<NMAX>(x, F);
  } else {
    f64_asymptote_fp64<NMAX>(x, F);
  }
}

// F_0 and y = 1/x of the asymptote as doubles (the Horner forms of the fused
// consumers): from f64_asymptote_start where the chain's range allows, else
// in FP64.  y is left 0 for NMAX = 0, where nothing uses it (and 1/x may be
// subnormal).
template <int NMAX>
__device__ __forceinline__ void f64_asymptote_f0_y(const double x, double &f0, double &y) {
  if (sig64_chain_ok<NMAX>(x)) {
    uint64_t sf, sy;
    int ef, ey;
    f0 = f64_asymptote_start(x, sf, ef, sy, ey);
    y = NMAX >= 1 ? __longlong_as_double((long long)sig64_round_bits(sy, ey)) : 0.0;
  } else {
    const double rs = rsqrt(x);
    f0 = 0.88622692545275801365 * rs;
    y = NMAX <= 12 ? rs * rs : 1.0 / x;
  }
}

// Staged row stores.  A warp whose lanes hold K list entries each (32 K
// rows) would store F_m from 32 lanes into 32 sectors (the rows are n_max+1
// doubles apart).  Instead it collects F_m for CH consecutive m of its rows in
// shared memory and writes each 32K x LEN block with consecutive lanes on
// consecutive elements of a row: a store instruction covers 32 / LEN row
// segments of LEN doubles.  Bank conflicts: with CH a power of two from 16
// on, rows are CH doubles and column c of row r sits at c ^ (r mod 16), so
// that 16 lanes writing one column of 16 rows, or reading 16 columns of one
// row, meet 16 different bank pairs; otherwise the row pitch is odd.  The
// unpadded rows let four blocks of 256 threads share an SM (f64_min_blocks).
template <int CH, int K>
struct F64Stage {
  static constexpr bool kSwizzle = CH >= 16 && (CH & (CH - 1)) == 0;
  static constexpr int kPitch = kSwizzle ? CH : (CH | 1);
  static constexpr int kDoublesPerWarp = 32 * K * kPitch;
  __device__ static __forceinline__ int at(int r, int c) { return r * kPitch + (kSwizzle ? (c ^ (r & 15)) : c); }
};

// The row index comes from a volatile shuffle: the addresses of a flush are
// the same for every chunk but m0, and kept live across the recursion they
// would cost two registers per store.
__device__ __forceinline__ int shfl_idx_volatile(int v, int src) {
  int r;
  asm volatile("shfl.sync.idx.b32 %0, %1, %2, 0x1f, 0xffffffff;" : "=r"(r) : "r"(v), "r"(src));
  return r;
}

// Write columns m0 .. m0 + LEN - 1 of the warp's staged rows: row 32 k + l
// is entry k (row index j[k]) of lane l; j[k] == kNoRow marks a lane without one.
template <int W, int CH, int K, int LEN>
__device__ __forceinline__ void f64_stage_flush(double *__restrict__ out, const double *__restrict__ stg, int m0,
                                                const int (&j)[K], int lane) {
  __syncwarp();
#pragma unroll
  for (int t = 0; t < K * LEN; ++t) {
    const int f = 32 * t + lane;
    const int r = f / LEN, e = f - r * LEN;
    const int jr = shfl_idx_volatile(j[t / LEN], r & 31);
    if (jr != kNoRow) __stcs(out + ((int64_t)jr * W + (m0 + e)), stg[F64Stage<CH, K>::at(r, e)]);
  }
  __syncwarp();
}

// Downward recursion of Eq. "r" from F_TOP (in f) to F_LO, staging F_m for
// LO <= m <= HI and flushing every chunk of CH orders whose lowest order is
// reached (orders above HI of that chunk were staged before, by the other
// recursion of a two-point evaluation).  The arithmetic is f64_recurse's.
template <int TOP, int LO, int HI, int W, int CH, int K, bool INT>
__device__ __forceinline__ void f64_recurse_staged(const double (&f0)[K], const double (&tx)[K], const F64E (&e)[K],
                                                   const int (&j)[K], double *__restrict__ out,
                                                   double *__restrict__ stg, const int lane) {
  if constexpr (!INT) {
    double f[K];
#pragma unroll
    for (int k = 0; k < K; ++k) f[k] = f0[k];
    static_for<TOP, LO - 1, -1>([&](auto mc) {
      constexpr int m = decltype(mc)::value;
      if constexpr (m <= HI) {
#pragma unroll
        for (int k = 0; k < K; ++k) stg[F64Stage<CH, K>::at(32 * k + lane, m % CH)] = f[k];
        if constexpr (m % CH == 0) f64_stage_flush<W, CH, K, (W - m < CH ? W - m : CH)>(out, stg, m, j, lane);
      }
      if constexpr (m > LO) {
#pragma unroll
        for (int k = 0; k < K; ++k) f[k] = fma(tx[k], f[k], e[k].d) * (1.0 / double(2 * m - 1));
      }
    });
  } else {
    // On the integer pipes.  An integer step is ~36 instructions, and the
    // code size sets the pace here: one order per loop iteration wherever the
    // chunks allow it.  Whole chunks of CH orders that are all staged, flushed
    // in full and above LO - 1 run in a loop over the chunks, and so do the
    // orders above them, from TOP (no multiple of CH among them but the
    // lowest, MT); without a whole chunk (TOP < 2 CH) and below the lowest one
    // (down to LO) the orders are unrolled.  Unrolled over every order, the
    // code of the high orders outgrew the instruction cache; with the chunks
    // looped and their 16 orders unrolled, n_max = 24 / 28 / 36 ran at
    // 220.6 / 228.4 / 251.5 G values/s, one order per iteration (with warps
    // starting on alternating lists, f64_tile) 238.7 / 249.3 / 280.4.
    Sig64Down r[K];
#pragma unroll
    for (int k = 0; k < K; ++k) r[k].start(f0[k], tx[k], e[k]);
    constexpr int TOPM = HI < TOP - 1 ? HI : TOP - 1;  // highest order a looped chunk may hold
    constexpr int CT = (TOPM + 1) / CH - 1;            // highest such chunk
    constexpr int CB = (LO + CH - 1) / CH;             // lowest chunk that starts at or above LO
    constexpr int MT = CT >= CB ? CH * (CT + 1) : LO;  // orders TOP .. MT come before the chunks
    auto unrolled = [&](auto mc) {
      constexpr int m = decltype(mc)::value;
      if constexpr (m <= HI) {
#pragma unroll
        for (int k = 0; k < K; ++k)
          stg[F64Stage<CH, K>::at(32 * k + lane, m % CH)] = m == TOP ? f0[k] : r[k].value();
        if constexpr (m % CH == 0) f64_stage_flush<W, CH, K, (W - m < CH ? W - m : CH)>(out, stg, m, j, lane);
      }
      if constexpr (m > LO) {
#pragma unroll
        for (int k = 0; k < K; ++k) r[k].template step<m>();
      }
    };
    if constexpr (CT >= CB) {
      // orders TOP .. MT + 1 (MT >= CH, so no step of order 1 here: the run
      // time step equals the unrolled one bit for bit, and F_TOP rounds back
      // to f0 exactly)
#pragma unroll 1
      for (int m = TOP; m > MT; --m) {
        if (m <= HI) {
#pragma unroll
          for (int k = 0; k < K; ++k) stg[F64Stage<CH, K>::at(32 * k + lane, (m - MT))] = r[k].value();
        }
#pragma unroll
        for (int k = 0; k < K; ++k) r[k].step_rt(m);
      }
      static_for<MT, MT - 1, -1>(unrolled);
#pragma unroll 1
      for (int c = CT; c >= CB; --c) {
        const int m0 = c * CH;
        // m0 >= LO, so every order above m0 steps
#pragma unroll 1
        for (int i = CH - 1; i >= 1; --i) {
#pragma unroll
          for (int k = 0; k < K; ++k) stg[F64Stage<CH, K>::at(32 * k + lane, i)] = r[k].value();
#pragma unroll
          for (int k = 0; k < K; ++k) r[k].step_rt(m0 + i);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) stg[F64Stage<CH, K>::at(32 * k + lane, 0)] = r[k].value();
        f64_stage_flush<W, CH, K, CH>(out, stg, m0, j, lane);
        if (m0 > LO) {
#pragma unroll
          for (int k = 0; k < K; ++k) r[k].step_rt(m0);
        }
      }
      static_for<CH * CB - 1, LO - 1, -1>(unrolled);
    } else {
      static_for<TOP, LO - 1, -1>(unrolled);
    }
  }
}

// f64_formula (TWO = false) or f64_formula_two (TWO = true) for the K
// entries of every lane of a full warp (rows j[k] of the tile), rows staged
// as above; the arithmetic is theirs.
template <int NTOP, int NMAX, int CH, int K, bool TWO>
__device__ __forceinline__ void f64_formula_staged(const double (&x)[K], const int (&j)[K], double *__restrict__ out,
                                                   double *__restrict__ stg, const F64ExpTab &tab,
                                                   const int lane) {
  constexpr int W = NMAX + 1;
  constexpr bool INTE = f64_int_rsqrt(NMAX, TWO);
  F64E e[K];
  double tx[K], f[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    e[k] = f64_exp_neg_both<f64_int_exp(NMAX, TWO)>(x[k], tab);
    tx[k] = twice(x[k]);
    f[k] = f64_closed_form<NTOP, INTE>(x[k], e[k]);
  }
  if constexpr (!TWO) {
    f64_recurse_staged<NTOP, 0, NMAX, W, CH, K, true>(f, tx, e, j, out, stg, lane);
  } else {
    constexpr int NBAR = f64_two_point_nbar(NMAX);
    constexpr int NTOP_LO = f64_top_order(NBAR);
    static_assert(NBAR < NMAX && NTOP_LO >= NBAR && NTOP_LO < NTOP, "orders");
    // two closed forms per argument leave less room for integer work: at
    // n_max = 36 the two-point rows measured 148 G values/s with both
    // recursions in FP64 and 139 on the integer pipes
    constexpr bool INT = f64_int_recursion(NTOP - NBAR - 1 + NTOP_LO);
    f64_recurse_staged<NTOP, NBAR + 1, NMAX, W, CH, K, INT>(f, tx, e, j, out, stg, lane);
#pragma unroll
    for (int k = 0; k < K; ++k) f[k] = f64_closed_form<NTOP_LO, true>(x[k], e[k]);
    f64_recurse_staged<NTOP_LO, 0, NBAR, W, CH, K, INT>(f, tx, e, j, out, stg, lane);
  }
}

// f64_asymptote for the K entries of every lane of a full warp, staged; the
// chain runs on the integer pipes when every entry of the warp allows it.
template <int NMAX, int CH, int K>
__device__ __forceinline__ void f64_asymptote_staged(const double (&x)[K], const int (&j)[K],
                                                     double *__restrict__ out, double *__restrict__ stg,
                                                     const int lane) {
  constexpr int W = NMAX + 1;
  double f[K];
  bool ok = true;
#pragma unroll
  for (int k = 0; k < K; ++k) ok = ok && sig64_chain_ok<NMAX>(x[k]);
  if (__all_sync(0xffffffffu, ok)) {
    // one order per loop iteration, as in f64_recurse_staged: the whole
    // chunks of CH orders, then the partial last one (the run-time step
    // equals the unrolled one bit for bit); rows shorter than CH unrolled
    Sig64Chain ch[K];
#pragma unroll
    for (int k = 0; k < K; ++k) f[k] = ch[k].start(x[k]);
    auto unrolled = [&](auto mc) {
      constexpr int m = decltype(mc)::value;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if constexpr (m > 0) f[k] = ch[k].template next<m>();
        stg[F64Stage<CH, K>::at(32 * k + lane, m % CH)] = f[k];
      }
      if constexpr (m % CH == CH - 1 || m == NMAX) f64_stage_flush<W, CH, K, m % CH + 1>(out, stg, m - m % CH, j, lane);
    };
    constexpr int CF = W / CH - 1;  // highest whole chunk
    if constexpr (CF >= 0) {
#pragma unroll 1
      for (int c = 0; c <= CF; ++c) {
        const int m0 = c * CH;
        if (c == 0) {
#pragma unroll
          for (int k = 0; k < K; ++k) stg[F64Stage<CH, K>::at(32 * k + lane, 0)] = f[k];
        } else {
#pragma unroll
          for (int k = 0; k < K; ++k) stg[F64Stage<CH, K>::at(32 * k + lane, 0)] = ch[k].next_rt(m0);
        }
#pragma unroll 1
        for (int i = 1; i < CH; ++i) {
#pragma unroll
          for (int k = 0; k < K; ++k) stg[F64Stage<CH, K>::at(32 * k + lane, i)] = ch[k].next_rt(m0 + i);
        }
        f64_stage_flush<W, CH, K, CH>(out, stg, m0, j, lane);
      }
      constexpr int MB = (CF + 1) * CH;  // the partial last chunk
      if constexpr (MB < W) {
#pragma unroll 1
        for (int m = MB; m < W; ++m) {
#pragma unroll
          for (int k = 0; k < K; ++k) stg[F64Stage<CH, K>::at(32 * k + lane, (m - MB))] = ch[k].next_rt(m);
        }
        f64_stage_flush<W, CH, K, W - MB>(out, stg, MB, j, lane);
      }
    } else {
      static_for<0, W, 1>(unrolled);
    }
    return;
  }
  // beyond the integer chain's range (x > 2^27 at n_max = 36; none of the
  // benchmark arguments): the FP64 chain, looped over whole chunks to keep
  // the code small
  double y[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double rs = rsqrt(x[k]);
    f[k] = 0.88622692545275801365 * rs;
    y[k] = NMAX <= 12 ? rs * rs : 1.0 / x[k];
  }
  constexpr int CF = W / CH - 1;  // highest whole chunk (-1 if none)
#pragma unroll 1
  for (int c = 0; c <= CF; ++c) {
    const int m0 = c * CH;
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int m = m0 + i;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (m > 0) f[k] = f[k] * ((double(m) - 0.5) * y[k]);
        stg[F64Stage<CH, K>::at(32 * k + lane, i)] = f[k];
      }
    }
    f64_stage_flush<W, CH, K, CH>(out, stg, m0, j, lane);
  }
  static_for<(CF + 1) * CH, W, 1>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if constexpr (m > 0) f[k] = f[k] * ((double(m) - 0.5) * y[k]);
      stg[F64Stage<CH, K>::at(32 * k + lane, m % CH)] = f[k];
    }
    if constexpr (m == NMAX) f64_stage_flush<W, CH, K, m % CH + 1>(out, stg, m - m % CH, j, lane);
  });
}

template <int W>
__device__ __forceinline__ void store_row(double *__restrict__ dst, const double (&F)[W]) {
#pragma unroll
  for (int m = 0; m < W; ++m) __stcs(dst + m, F[m]);
}

// Below-cut-off test on the bit pattern (integer pipe): true for +-0 and
// 0 < x <= z; false for negative nonzero x, NaN and x > z.
__device__ __forceinline__ bool below_cutoff(double v, unsigned long long zbits) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned long long mag = b & 0x7fffffffffffffffULL;
  return ((b >> 63) == 0 || mag == 0) && mag <= zbits;
}

// What the split kernel does with a finished row F_0..F_NMAX of argument j
// of the current tile (j counts from the tile's first argument).
template <int W>
struct StoreRows {
  static constexpr bool kRowStore = true;  // the rows may go out through the staging buffer
  static constexpr bool kHorner = false;
  double *out;  // row 0 of the tile
  __device__ __forceinline__ void operator()(int j, const double (&F)[W]) const { store_row<W>(out + (int64_t)j * W, F); }
};

// Gradient epilogue: grad[j] = -sum_{m=0}^{W-2} g[j, m] F_{m+1}(x_j)
// (dF_m/dx = -F_{m+1}, from differentiating Eq. "fn" under the integral).
template <int W>
struct GradDot {
  static constexpr bool kRowStore = false;
  // as for ContractDot (the forward order here is one above the gradient's)
  static constexpr bool kHorner = W <= 18;
  const double *g;  // row 0 of the tile
  int64_t g_row, g_col;
  double *grad;  // element 0 of the tile
  // with the same weights for every argument (g_row == 0):
  // hu_m = g_m prod_{k<=m+1} (k - 1/2), m = 0..W-2 (MakeGrad::prepare)
  double hu[W];
  __device__ __forceinline__ void operator()(int j, const double (&F)[W]) const {
    const double *gj = g + (int64_t)j * g_row;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m + 1 < W; ++m) acc = fma(__ldg(gj + m * g_col), F[m + 1], acc);
    grad[j] = -acc;
  }
  __device__ __forceinline__ bool uniform() const { return g_row == 0; }
  // Above the cut-off F_{m+1} = F_0 prod_{k<=m+1} (k - 1/2) y^{m+1}, so the
  // gradient is -F_0 y P(y) by Horner (uniform weights only), with F_0 and
  // y as f64_asymptote forms them.
  __device__ __forceinline__ double asymptote_dot(const double x) const {
    double f0, y;
    f64_asymptote_f0_y<W - 1>(x, f0, y);
    double acc = hu[W - 2];
#pragma unroll
    for (int m = W - 3; m >= 0; --m) acc = fma(acc, y, hu[m]);
    return -(acc * (f0 * y));
  }
  __device__ __forceinline__ void put(int j, double v) const { grad[j] = v; }
};

// Contraction epilogue (a fused consumer): out[j] = sum_{m=0}^{W-1} c[j, m] F_m(x_j),
// the rows never leave the registers.
template <int W>
struct ContractDot {
  static constexpr bool kRowStore = false;
  // up to n_max = 16: above, the W coefficients held in registers next to two
  // rows per lane would cost more occupancy than the polynomial saves
  static constexpr bool kHorner = W <= 17;
  const double *c;  // row 0 of the tile
  int64_t c_row, c_col;
  double *out;  // element 0 of the tile
  // with the same coefficients for every argument (c_row == 0):
  // hu_m = c_m prod_{k<=m} (k - 1/2), the asymptote's contraction as a
  // polynomial in y = 1/x (MakeContract::prepare)
  double hu[W];
  __device__ __forceinline__ void operator()(int j, const double (&F)[W]) const {
    const double *cj = c + (int64_t)j * c_row;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < W; ++m) acc = fma(__ldg(cj + m * c_col), F[m], acc);
    out[j] = acc;
  }
  __device__ __forceinline__ bool uniform() const { return c_row == 0; }
  // Above the cut-off, where F_m = F_0 prod_{k<=m} (k - 1/2) y: the
  // contraction is F_0 P(y) by Horner (uniform coefficients only), with F_0
  // and y as f64_asymptote forms them.
  __device__ __forceinline__ double asymptote_dot(const double x) const {
    double f0, y;
    f64_asymptote_f0_y<W - 1>(x, f0, y);
    double acc = hu[W - 1];
#pragma unroll
    for (int m = W - 2; m >= 0; --m) acc = fma(acc, y, hu[m]);
    return acc * f0;
  }
  __device__ __forceinline__ void put(int j, double v) const { out[j] = v; }
};

// Entries of each list carried into the block's next tile (fewer than one
// warp request): argument and row, the row relative to that tile's first
// argument.  Without carrying only the (zero) counts exist.
template <bool CARRY>
struct F64Carry {
  double cx[2][64];
  int cj[2][64];
  int cn[2];
};
template <>
struct F64Carry<false> {
  int cn[2];
};

template <int TILE, bool CARRY = false>
struct F64TileSmem : F64Carry<CARRY> {
  double xs[TILE];
  unsigned short lst[TILE];  // below list from the front, above list from the back
  F64ExpTab tab;
  int cnt[2], next[2];
};

// One tile of nel <= TILE arguments xt[0..nel): classify, build the two lists,
// evaluate each list in warp requests (32 entries, 64 with two per lane) and
// hand the rows to epi (STAGE > 0: stage and store them; stage = the block's
// staging buffer).  All threads of the block call it; it begins and ends with
// a barrier.
// ALLOW_ILP = false keeps one list entry per lane at every order (a kernel
// that switches between orders keeps the register count of the smallest).
template <int NMAX, int BLOCK, int TILE, typename Epi, bool TWO = false, bool ALLOW_ILP = true, int STAGE = 0,
          int STAGE_K = 2, bool CARRY = false>
__device__ __forceinline__ void f64_tile(const double *__restrict__ xt, int nel, const Epi &epi,
                                         F64TileSmem<TILE, CARRY> &sm, double *__restrict__ stage = nullptr,
                                         bool last = true) {
  constexpr int NTOP = f64_top_order(NMAX);
  constexpr int W = NMAX + 1;
  static_assert(TILE % BLOCK == 0 && TILE <= 65536, "tile");
  const unsigned long long zbits = (unsigned long long)__double_as_longlong(BoysF64<NTOP>::kCutoff);
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  if (threadIdx.x == 0) {
    sm.cnt[0] = sm.cnt[1] = 0;
    sm.next[0] = sm.next[1] = 0;
  }
  __syncthreads();
  // argument j of the tile (value v) into its list
  auto classify = [&](const int j, const double v, const bool valid) {
    sm.xs[j] = v;
    const bool lo = valid && below_cutoff(v, zbits);
    const bool hi = valid && !lo;
    const unsigned mlo = __ballot_sync(0xffffffffu, lo), mhi = __ballot_sync(0xffffffffu, hi);
    int plo = 0, phi = 0;
    if (lane == 0) {
      if (mlo) plo = atomicAdd(&sm.cnt[0], __popc(mlo));
      if (mhi) phi = atomicAdd(&sm.cnt[1], __popc(mhi));
    }
    plo = __shfl_sync(0xffffffffu, plo, 0);
    phi = __shfl_sync(0xffffffffu, phi, 0);
    if (lo) sm.lst[plo + __popc(mlo & lt)] = (unsigned short)j;
    if (hi) sm.lst[TILE - 1 - (phi + __popc(mhi & lt))] = (unsigned short)j;
  };
  // arguments j and j + 1 (values v.x, v.y) of a thread's pair into the
  // lists, in argument order across the warp's 64 arguments (a list in
  // argument order keeps the rows a warp request stores close together: with
  // the even and the odd arguments listed apart, n_max = 8 fell from 143 to
  // 105 G values/s)
  auto classify2 = [&](const int j, const double2 v, const int nv) {
    sm.xs[j] = v.x;
    sm.xs[j + 1] = v.y;
    const bool lo0 = nv > 0 && below_cutoff(v.x, zbits), hi0 = nv > 0 && !lo0;
    const bool lo1 = nv > 1 && below_cutoff(v.y, zbits), hi1 = nv > 1 && !lo1;
    const unsigned l0 = __ballot_sync(0xffffffffu, lo0), l1 = __ballot_sync(0xffffffffu, lo1);
    const unsigned h0 = __ballot_sync(0xffffffffu, hi0), h1 = __ballot_sync(0xffffffffu, hi1);
    int plo = 0, phi = 0;
    if (lane == 0) {
      if (l0 | l1) plo = atomicAdd(&sm.cnt[0], __popc(l0) + __popc(l1));
      if (h0 | h1) phi = atomicAdd(&sm.cnt[1], __popc(h0) + __popc(h1));
    }
    plo = __shfl_sync(0xffffffffu, plo, 0) + __popc(l0 & lt) + __popc(l1 & lt);
    phi = __shfl_sync(0xffffffffu, phi, 0) + __popc(h0 & lt) + __popc(h1 & lt);
    if (lo0) sm.lst[plo] = (unsigned short)j;
    if (lo1) sm.lst[plo + lo0] = (unsigned short)(j + 1);
    if (hi0) sm.lst[TILE - 1 - phi] = (unsigned short)j;
    if (hi1) sm.lst[TILE - 1 - (phi + hi0)] = (unsigned short)(j + 1);
  };
  bool scalar = true;
  if constexpr (TILE % (2 * BLOCK) == 0) {
    // 128-bit loads: two neighbouring arguments per thread where the tile
    // starts on a 16-byte boundary (a plain evaluation's tiles do when x does)
    if ((reinterpret_cast<uintptr_t>(xt) & 15) == 0) {
      scalar = false;
#pragma unroll 2
      for (int p0 = 0; p0 < TILE / 2; p0 += BLOCK) {
        const int j = 2 * (p0 + threadIdx.x);
        double2 v = make_double2(0.0, 0.0);
        if (j + 1 < nel) {
          v = __ldcs(reinterpret_cast<const double2 *>(xt + j));
        } else if (j < nel) {
          v.x = __ldcs(xt + j);
        }
        classify2(j, v, nel - j);
      }
    }
  }
  if (scalar) {
#pragma unroll 4
    for (int j0 = 0; j0 < TILE; j0 += BLOCK) {
      const int j = j0 + threadIdx.x;
      const bool valid = j < nel;
      classify(j, valid ? __ldcs(xt + j) : 0.0, valid);
    }
  }
  __syncthreads();
  const int nlo = sm.cnt[0], nhi = sm.cnt[1];
  // closed form on the below-cut-off list, 32 entries per warp request; for
  // high orders a lane takes two entries, whose long recursion chains then
  // interleave (the FP64 result latency, not the pipe, would set the pace)
  // Staged rows (STAGE > 0, a store epilogue): STAGE_K entries per lane, the
  // rows go out through the warp's staging buffer STAGE orders at a time.
  constexpr bool STAGED = STAGE > 0;
  static_assert(!STAGED || Epi::kRowStore, "staging serves row stores");
  constexpr int ILP = STAGED ? STAGE_K : ((NMAX >= 12 && !TWO && ALLOW_ILP) ? 2 : 1);
  constexpr int CHUNK = 32 * ILP;  // entries per warp request
  static_assert(!CARRY || (CHUNK <= 64 && BLOCK >= 2 * CHUNK), "carry arrays");
  using Stage = F64Stage<(STAGED ? STAGE : 1), ILP>;
  double *const stg = STAGED ? stage + (threadIdx.x >> 5) * Stage::kDoublesPerWarp : nullptr;
  // CARRY: the entries carried from the block's previous tile come first in
  // each list, and a list evaluates only whole warp requests, carrying the
  // rest into the next tile (a partly filled request costs the FP64 pipe as
  // much as a full one), unless this is the block's last tile or the list
  // holds less than one request.  Carried entries are thus evaluated exactly
  // one tile later.
  const int clo = CARRY ? sm.cn[0] : 0, chi = CARRY ? sm.cn[1] : 0;
  const int tlo = clo + nlo, thi = chi + nhi;
  const int flo = (CARRY && !last && tlo >= CHUNK) ? tlo / CHUNK * CHUNK : tlo;
  const int fhi = (CARRY && !last && thi >= CHUNK) ? thi / CHUNK * CHUNK : thi;
  // entry q of list L (0 below, 1 above): its argument, and its row relative
  // to this tile's first argument
  auto entry = [&](const int L, const int q, double &x) -> int {
    const int c = L ? chi : clo;
    if constexpr (CARRY) {
      if (q < c) {
        x = sm.cx[L][q];
        return sm.cj[L][q];
      }
    }
    const int i = q - c;
    const int j = L ? sm.lst[TILE - 1 - i] : sm.lst[i];
    x = sm.xs[j];
    return j;
  };
  auto below_loop = [&]() {
    for (;;) {
      int c = 0;
      if (lane == 0) c = atomicAdd(&sm.next[0], CHUNK);
      c = __shfl_sync(0xffffffffu, c, 0);
      if (c >= flo) break;
      const int q = c + lane;
      if constexpr (STAGED) {
        // the whole warp takes part; lanes past the end of the list compute a
        // dummy argument and store nothing.  (A one-entry-per-lane copy for
        // the last request of a list saved that request's dummy work, but its
        // code cost more in instruction fetch: 1.5-2% slower at n_max = 16
        // and 36.)
        int j[ILP];
        double xv[ILP];
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
          xv[k] = 1.0;
          j[k] = kNoRow;
          if (q + 32 * k < flo) j[k] = entry(0, q + 32 * k, xv[k]);
        }
        f64_formula_staged<NTOP, NMAX, STAGE, ILP, TWO>(xv, j, epi.out, stg, sm.tab, lane);
        continue;
      }
      if constexpr (ILP == 2) {
        if (q + 32 < flo) {
          double xa, xb;
          const int ja = entry(0, q, xa), jb = entry(0, q + 32, xb);
          double Fa[W], Fb[W];
          f64_formula<NTOP, NMAX>(xa, Fa, sm.tab);
          f64_formula<NTOP, NMAX>(xb, Fb, sm.tab);
          epi(ja, Fa);
          epi(jb, Fb);
          continue;
        }
      }
      if (q < flo) {
        double xq;
        const int j = entry(0, q, xq);
        double F[W];
        if constexpr (TWO) {
          constexpr int NBAR = f64_two_point_nbar(NMAX);
          f64_formula_two<NTOP, f64_top_order(NBAR), NBAR, NMAX>(xq, F, sm.tab);
        } else {
          f64_formula<NTOP, NMAX>(xq, F, sm.tab);
        }
        epi(j, F);
      }
    }
  };
  auto above_loop = [&]() {
    // asymptote on the above-cut-off list (two entries per lane for high
    // orders, as above: the upward product chain is 2 n_max long)
    for (;;) {
      int c = 0;
      if (lane == 0) c = atomicAdd(&sm.next[1], CHUNK);
      c = __shfl_sync(0xffffffffu, c, 0);
      if (c >= fhi) break;
      const int q = c + lane;
      if constexpr (Epi::kHorner) {
        if (epi.uniform()) {  // the contraction of the asymptote as a polynomial
#pragma unroll
          for (int k = 0; k < ILP; ++k) {
            if (q + 32 * k < fhi) {
              double xq;
              const int j = entry(1, q + 32 * k, xq);
              epi.put(j, epi.asymptote_dot(xq));
            }
          }
          continue;
        }
      }
      if constexpr (STAGED) {
        int j[ILP];
        double xv[ILP];
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
          xv[k] = 1.0;
          j[k] = kNoRow;
          if (q + 32 * k < fhi) j[k] = entry(1, q + 32 * k, xv[k]);
        }
        f64_asymptote_staged<NMAX, STAGE, ILP>(xv, j, epi.out, stg, lane);
        continue;
      }
      if constexpr (ILP == 2) {
        if (q + 32 < fhi) {
          double xa, xb;
          const int ja = entry(1, q, xa), jb = entry(1, q + 32, xb);
          double Fa[W], Fb[W];
          f64_asymptote<NMAX>(xa, Fa);
          f64_asymptote<NMAX>(xb, Fb);
          epi(ja, Fa);
          epi(jb, Fb);
          continue;
        }
      }
      if (q < fhi) {
        double xq;
        const int j = entry(1, q, xq);
        double F[W];
        f64_asymptote<NMAX>(xq, F);
        epi(j, F);
      }
    }
  };
  // Even warps start on the closed-form list, odd warps on the asymptote
  // list, and each then helps with the other one, so FP64-bound and
  // integer-bound requests run side by side instead of one list after
  // the other (n_max = 8: 139.5 -> 142.9 G values/s; two-point n_max = 36:
  // 163.9 -> 171.5; staged one-point rows n_max = 12: 173.4 -> 181.4,
  // 16: 191.2 -> 197.0, 20: 210.1 -> 210.9).  From n_max = 21 on it pays
  // only since the integer chains loop over single orders (measured with two
  // orders per iteration, 24: 219.3 -> 239.9, 32: 254.8 -> 276.9, 36: 259.8
  // -> 277.2); with their 16 orders unrolled the two live phases had cost
  // instruction fetch (36: 251 -> 232).
  const int par = (threadIdx.x >> 5) & 1;
#pragma unroll 1
  for (int ph = 0; ph < 2; ++ph) {
    if ((ph ^ par) == 0) {
      below_loop();
    } else {
      above_loop();
    }
  }
  __syncthreads();
  if constexpr (CARRY) {
    if (!last) {
      // the rest of each list (fewer than CHUNK entries, all from this tile's
      // list since the carried ones came first) moves to the carry, its rows
      // made relative to the block's next tile
      const int rlo = tlo - flo, rhi = thi - fhi;
      const int shift = (int)gridDim.x * TILE;
      if (threadIdx.x < rlo + rhi) {
        const int L = threadIdx.x < rlo ? 0 : 1;
        const int p = L ? threadIdx.x - rlo : threadIdx.x;
        double x;
        const int j = entry(L, (L ? fhi : flo) + p, x);
        sm.cx[L][p] = x;
        sm.cj[L][p] = j - shift;
      }
      if (threadIdx.x == 0) {
        sm.cn[0] = rlo;
        sm.cn[1] = rhi;
      }
    }
  }
}

template <int BLOCK, typename Smem>
__device__ __forceinline__ void f64_load_table(Smem &sm) {
  for (int i = threadIdx.x; i < 64; i += BLOCK) {
    sm.tab.d[i] = kExp2Frac64[i];
    sm.tab.s[i] = kExp2Frac64Sig[i];
  }
  if (threadIdx.x == 0) sm.cn[0] = sm.cn[1] = 0;  // nothing carried yet
}

template <int BLOCK, int STAGE, int K>
constexpr size_t f64_stage_bytes() {
  return STAGE > 0 ? sizeof(double) * (BLOCK / 32) * F64Stage<(STAGE > 0 ? STAGE : 1), K>::kDoublesPerWarp : 0;
}

// Resident blocks per SM that a staged kernel is compiled for: as many as its
// shared memory allows (228 KB per SM, 1 KB reserved per block), at most 4
// (6 for the whole-row staging of n_max = 8 to 11);
// the register budget follows from it.  Blocks of 256 threads with 2048-
// argument tiles take 55.4 KB: 4 blocks of 64 registers.  Against 3 blocks
// of 80 registers with odd-pitch rows (57.4 KB), n_max = 20 / 24 / 28 / 32 /
// 36 measured 223.8 / 238.2 / 249.1 / 275.6 / 279.9 -> 227.3 / 242.7 /
// 257.5 / 281.9 / 280.7 G values/s, two-point n_max = 36 175.6 -> 174.6.
// (With the integer chains' 16 orders unrolled per chunk, 4 blocks had
// been slower: 251.7 -> 238.5 at n_max = 36.)
template <int BLOCK, int TILE, int STAGE, int K>
constexpr int f64_min_blocks() {
  if (STAGE == 0) return 1;
  const size_t per_block = sizeof(F64TileSmem<TILE, true>) + f64_stage_bytes<BLOCK, STAGE, K>() + 1024;
  const int b = (int)((size_t)228 * 1024 / per_block);
  // the whole-row staging below n_max = 12 (1024-argument tiles, 31.7 KB)
  // runs 6 blocks of 40 registers (7 of 32 spilled; n_max = 8: 177.1
  // against 170.9 G values/s)
  const int cap = (BLOCK == 256 && STAGE < 16) ? 6 : 4;
  return b < 1 ? 1 : (b > cap ? cap : b);
}

// Tiles of a persistent block (all kernels below).
template <int NMAX, int BLOCK, int TILE, typename MakeEpi, bool TWO, int STAGE, int K>
__device__ __forceinline__ void f64_tiles(const double *__restrict__ x, int64_t count, const MakeEpi &make,
                                          F64TileSmem<TILE, true> &sm, double *__restrict__ stage) {
  f64_load_table<BLOCK>(sm);
  MakeEpi mk = make;
  mk.prepare();
  const int64_t ntiles = (count + TILE - 1) / TILE;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t base = t * TILE;
    const int nel = (int)((count - base) < TILE ? (count - base) : TILE);
    f64_tile<NMAX, BLOCK, TILE, decltype(mk(base)), TWO, true, STAGE, K, true>(x + base, nel, mk(base), sm, stage,
                                                                            t + gridDim.x >= ntiles);
  }
}

// Resident blocks the unstaged kernels are compiled for.  The one-point row
// kernels of 256 threads up to n_max = 9 ask for 8 (at most 32 registers;
// with the largest shared-memory carveout, set at launch, 8 tiles of 22.6 KB
// fit): 34 registers had left 6 blocks per SM, and n_max = 8 ran at 142.3 G
// values/s against 145.7 with 8 (n_max = 4: 89.6 against 90.6), no spills.
// From n_max = 10 on 32 registers spill.  The contraction and gradient
// epilogues keep the default allocation.
template <int NMAX, int BLOCK, typename MakeEpi, bool TWO>
constexpr int f64_split_min_blocks() {
  return (BLOCK == 256 && NMAX <= 9 && MakeEpi::kRows && !TWO) ? 8 : 1;
}

// Plain, gradient and contraction kernels: persistent blocks stride over the tiles.
template <int NMAX, int BLOCK, int TILE, typename MakeEpi, bool TWO = false>
__global__ void __launch_bounds__(BLOCK, (f64_split_min_blocks<NMAX, BLOCK, MakeEpi, TWO>()))
    f64_split_kernel(const double *__restrict__ x, int64_t count, const MakeEpi make) {
  __shared__ F64TileSmem<TILE, true> sm;
  f64_tiles<NMAX, BLOCK, TILE, MakeEpi, TWO, 0, 1>(x, count, make, sm, nullptr);
}

// Staged rows, K list entries per lane (dynamic shared memory of
// f64_stage_bytes), compiled for f64_min_blocks resident blocks.
template <int NMAX, int BLOCK, int TILE, typename MakeEpi, bool TWO, int STAGE, int K>
__global__ void __launch_bounds__(BLOCK, (f64_min_blocks<BLOCK, TILE, STAGE, K>()))
    f64_staged_kernel(const double *__restrict__ x, int64_t count, const MakeEpi make) {
  __shared__ F64TileSmem<TILE, true> sm;
  extern __shared__ __align__(16) unsigned char f64_stage_raw[];
  f64_tiles<NMAX, BLOCK, TILE, MakeEpi, TWO, STAGE, K>(x, count, make, sm,
                                                       reinterpret_cast<double *>(f64_stage_raw));
}

template <int W>
struct MakeStore {
  static constexpr bool kRows = true;
  double *out;
  __device__ __forceinline__ void prepare() {}
  __device__ __forceinline__ StoreRows<W> operator()(int64_t base) const { return StoreRows<W>{out + base * W}; }
};

template <int W>
struct MakeGrad {
  static constexpr bool kRows = false;
  const double *g;
  int64_t g_row, g_col;
  double *grad;
  double hu[W];  // filled by prepare() on the device
  // once per thread: the Horner coefficients of the asymptote's gradient
  __device__ __forceinline__ void prepare() {
    double p = 1.0;
#pragma unroll
    for (int m = 0; m + 1 < W; ++m) {
      p *= double(m + 1) - 0.5;
      hu[m] = (GradDot<W>::kHorner && g_row == 0) ? __ldg(g + m * g_col) * p : 0.0;
    }
    hu[W - 1] = 0.0;
  }
  __device__ __forceinline__ GradDot<W> operator()(int64_t base) const {
    GradDot<W> d{g + base * g_row, g_row, g_col, grad + base, {}};
#pragma unroll
    for (int m = 0; m < W; ++m) d.hu[m] = hu[m];
    return d;
  }
};

template <int W>
struct MakeContract {
  static constexpr bool kRows = false;
  const double *c;
  int64_t c_row, c_col;
  double *out;
  double hu[W];  // filled by prepare() on the device
  // once per thread: the Horner coefficients of the asymptote's contraction
  __device__ __forceinline__ void prepare() {
    double g = 1.0;
#pragma unroll
    for (int m = 0; m < W; ++m) {
      if (m > 0) g *= double(m) - 0.5;
      hu[m] = (ContractDot<W>::kHorner && c_row == 0) ? __ldg(c + m * c_col) * g : 0.0;
    }
  }
  __device__ __forceinline__ ContractDot<W> operator()(int64_t base) const {
    ContractDot<W> d{c + base * c_row, c_row, c_col, out + base, {}};
#pragma unroll
    for (int m = 0; m < W; ++m) d.hu[m] = hu[m];
    return d;
  }
};

constexpr int kF64Block = 256, kF64Tile = 2048;

// Below this many arguments the work would not fill the GPU with 2048-argument
// tiles (a 65,536-argument call is 32 tiles for 152 SMs), so small tiles are
// used: the per-argument arithmetic, and so every result, is the same.
constexpr int64_t kF64SmallCount = 1 << 20;
constexpr int kF64SmallBlock = 128, kF64SmallTile = 256;

// Launch kernel k on a persistent grid (set up per device through cache).
template <typename Kernel, typename MakeEpi>
int launch_f64_persistent(Kernel k, std::atomic<int> (&cache)[kMaxCachedDevices], int block, int tile, size_t dyn,
                          const double *x, int64_t count, const MakeEpi &epi, cudaStream_t s, int carveout = -1) {
  const int grid_cap = device_setup(k, block, dyn, dyn, true, cache, carveout);
  if (grid_cap == 0) return BOYS_ERR_CUDA;
  const int64_t tiles = (count + tile - 1) / tile;
  const int grid = (int)(tiles < grid_cap ? tiles : grid_cap);
  k<<<grid, block, dyn, s>>>(x, count, epi);
  return cudaPeekAtLastError() == cudaSuccess ? BOYS_OK : BOYS_ERR_CUDA;
}

template <int NMAX, int BLOCK, int TILE, typename MakeEpi, bool TWO, int STAGE = 0, int K = 2>
int launch_f64_shape(const double *x, int64_t count, const MakeEpi &epi, cudaStream_t s) {
  static std::atomic<int> cache[kMaxCachedDevices];
  if constexpr (STAGE > 0) {
    return launch_f64_persistent(f64_staged_kernel<NMAX, BLOCK, TILE, MakeEpi, TWO, STAGE, K>, cache, BLOCK, TILE,
                                 f64_stage_bytes<BLOCK, STAGE, K>(), x, count, epi, s);
  } else {
    // compiled for 8 resident blocks: all of the SM's on-chip memory that
    // can be shared memory, as their tiles take more than the default split
    constexpr bool eight = f64_split_min_blocks<NMAX, BLOCK, MakeEpi, TWO>() == 8;
    return launch_f64_persistent(f64_split_kernel<NMAX, BLOCK, TILE, MakeEpi, TWO>, cache, BLOCK, TILE, 0, x,
                                 count, epi, s, eight ? 100 : -1);
  }
}

template <int NMAX, typename MakeEpi, bool TWO = false, int STAGE = 0, int K = 2, int TILE = kF64Tile>
int launch_f64_epi(const double *x, int64_t count, const MakeEpi &epi, cudaStream_t s) {
  if (count <= kF64SmallCount)
    return launch_f64_shape<NMAX, kF64SmallBlock, kF64SmallTile, MakeEpi, TWO, STAGE, K>(x, count, epi, s);
  return launch_f64_shape<NMAX, kF64Block, TILE, MakeEpi, TWO, STAGE, K>(x, count, epi, s);
}

// Row staging from n_max = 12 on: orders per flush of the staging buffer
// and list entries per lane.  The one-point rows flush 16 orders of 32 rows
// (each store instruction then covers two row segments of 128 bytes): with
// the arithmetic stubbed out, n_max = 36 spent 2.6 ms of its 3.1 ms on the
// stores of 8-order flushes of 64 rows (four 64-byte segments per store
// instruction), 2.05 ms with 16 orders of 64 rows, 1.5 ms with 32 orders of
// 32 rows.  In full: n_max = 36 202.5 -> 250.0 G values/s, n_max = 16
// 172.6 -> 189.6 (16 orders and two entries per lane: 166.5 and 161.2, two
// resident blocks; whole rows per flush: 224.3 and 182.6).  The two-point rows
// the same way: n_max = 36 173.7 -> 175.8.
constexpr int kF64StageOrders = 16, kF64StageK = 1;
constexpr int kF64TwoStageOrders = 16, kF64TwoStageK = 1;
// From n_max = 8 to 11 the whole row is staged (one flush of n_max + 1
// orders) in 1024-argument tiles: once the asymptote and the closed form's
// reciprocal square roots left the FP64 pipe, the rows stored from the
// lanes' registers (a store instruction writes 8 bytes into each of 32
// sectors) held n_max = 8 at 136.2 G values/s, against 177.1 staged; n_max =
// 9 / 10 / 11 132.8 / 144.2 / 183.0 -> 189.4 / 195.2 / 199.8.  Below n_max = 8
// the lanes' stores stay faster (n_max = 7: 177.4 against 164.6; 4: 123.8
// against 118.3).
constexpr int kF64RowStageFrom = 8, kF64RowStageTile = 1024;
__host__ __device__ constexpr int f64_row_stage(int n_max) {
  return n_max >= 12 ? kF64StageOrders : (n_max >= kF64RowStageFrom ? n_max + 1 : 0);
}

template <int NMAX>
int launch_f64(const double *x, int64_t count, double *out, cudaStream_t s) {
  constexpr int STAGE = f64_row_stage(NMAX);
  constexpr int TILE = (STAGE > 0 && NMAX < 12) ? kF64RowStageTile : kF64Tile;
  return launch_f64_epi<NMAX, MakeStore<NMAX + 1>, false, STAGE, kF64StageK, TILE>(x, count,
                                                                                   MakeStore<NMAX + 1>{out}, s);
}

// Backward with the forward rows recomputed: the order n_max + 1 is needed.
template <int NMAX_FWD>
int launch_f64_grad_recompute(const double *x, int64_t count, const double *g, int64_t g_row, int64_t g_col,
                              double *grad, cudaStream_t s) {
  return launch_f64_epi<NMAX_FWD>(x, count, MakeGrad<NMAX_FWD + 1>{g, g_row, g_col, grad}, s);
}

// Two-point evaluation (Trick B): rows as launch_f64.
template <int NMAX>
int launch_f64_two_point(const double *x, int64_t count, double *out, cudaStream_t s) {
  return launch_f64_epi<NMAX, MakeStore<NMAX + 1>, true, (NMAX >= 12 ? kF64TwoStageOrders : 0), kF64TwoStageK>(
      x, count, MakeStore<NMAX + 1>{out}, s);
}

template <int NMAX>
int launch_f64_contract(const double *x, int64_t count, const double *c, int64_t c_row, int64_t c_col, double *out,
                        cudaStream_t s) {
  return launch_f64_epi<NMAX>(x, count, MakeContract<NMAX + 1>{c, c_row, c_col, out}, s);
}

}  // namespace boys

#define BOYS_F64_TWO_CASE(k) \
  case k:                    \
    return boys::launch_f64_two_point<k>(x, count, out, s);

#define BOYS_F64_CONTRACT_CASE(k) \
  case k:                         \
    return boys::launch_f64_contract<k>(x, count, c, c_row, c_col, out, s);

#define BOYS_F64_CASE(k) \
  case k:                \
    return boys::launch_f64<k>(x, count, out, s);

#define BOYS_F64_GRAD_CASE(k) \
  case k:                     \
    return boys::launch_f64_grad_recompute<k + 1>(x, count, g, g_row, g_col, grad, s);
