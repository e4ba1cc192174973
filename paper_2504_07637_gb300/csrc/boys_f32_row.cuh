// FP32 path: the per-argument evaluation (host- and device-compilable so the
// same code can be exercised on the CPU).
//
// The closed form amplifies relative errors: dF/F = -s^2 (T/D) dQ/Q with
// s = n + 1/2, T = Q^s e^{-x}, D = x + T, which is s^2 = 72 at x -> 0 for
// n = 8.  Plain FP32 therefore loses ~6 bits (the paper's single-precision
// column of Table I).  Here every quantity on the amplified path -- q0 + q1 x,
// Q^s, e^{-x}, D and D^{-s} -- is carried as a float-float pair (~48 bits),
// while the rational part q2 x^2 u/v, whose contribution vanishes as x^2 where
// the amplification is largest, and the recursion stay in FP32.  The fits are
// one order N above the paper's single-precision column (~27-31 bits, cf. the
// "about 28-bit accurate approximations" of Sec. 3), so the fit error stays
// below FP32 rounding.
#pragma once

#include "boys_ff.cuh"

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define BOYS_F32_DEVFN __host__ __device__ __forceinline__
#else
#define BOYS_F32_DEVFN inline
#endif

BOYS_F32_DEVFN int boys_float_as_int(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_int(f);
#else
  int i;
  std::memcpy(&i, &f, 4);
  return i;
#endif
}
BOYS_F32_DEVFN float boys_int_as_float(int i) {
#ifdef __CUDA_ARCH__
  return __int_as_float(i);
#else
  float f;
  std::memcpy(&f, &i, 4);
  return f;
#endif
}
BOYS_F32_DEVFN float boys_rsqrtf(float a) {
#ifdef __CUDA_ARCH__
  return rsqrtf(a);
#else
  return 1.0f / std::sqrt(a);
#endif
}
// a / b with a couple of ulp error (one MUFU reciprocal and a multiply)
BOYS_F32_DEVFN float boys_fdiv_approx(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
// 1/b correctly rounded
BOYS_F32_DEVFN float boys_frcp_rn(float b) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(b);
#else
  return 1.0f / b;
#endif
}

#include "boys_coeffs_f32.inc"

namespace boys {

// e^{-x} as a float-float pair for 0 <= x <= 80, by Tang's table-driven
// method (ACM TOMS 15(2), 1989) in the float-float setting:
//   -x = (k/32) ln2 + r,  |r| <= ln2/64,  e^{-x} = 2^(k>>5) 2^((k&31)/32) (1 + p(r)),
// with ln2/32 split in three parts (Cody and Waite) so r is accurate to
// 2^-31 absolute, and p(r) = r + r^2/2 + r^3/6 + r^4/24 in FP32 (truncation
// 2^-35, rounding 2^-30 absolute).  tab holds 2^(j/32) as (hi, lo) pairs.
BOYS_F32_DEVFN ff ff_exp_neg(float x, const float *tab) {
  const float kShift = 12582912.0f;          // 1.5 * 2^23
  const float kInvL = 46.16624069213867f;   // 32 / ln2
  const float kL1 = 0.02165985107421875f;   // ln2/32 to 12 significant bits
  const float kL2 = 9.98377799987793e-07f;  // the next 12 bits
  const float kL3 = -5.952044412893542e-11f; // the remainder
  float kd = fmaf(-x, kInvL, kShift);
  const int k = boys_float_as_int(kd) - boys_float_as_int(kShift);
  kd = kd - kShift;
  float r = fmaf(kd, -kL1, -x);
  r = fmaf(kd, -kL2, r);
  r = fmaf(kd, -kL3, r);
  float p = fmaf(r, 1.0f / 24.0f, 1.0f / 6.0f);
  p = fmaf(r, p, 0.5f);
  p = fmaf(r, p, 1.0f);
  p = p * r;
  const int j = k & 31;
  const float th = tab[2 * j], tl = tab[2 * j + 1];
  ff e = fast_two_sum(th, fmaf(th, p, tl + tl * p));
  const float scale = boys_int_as_float((127 + (k >> 5)) << 23);
  e.hi *= scale;
  e.lo *= scale;
  return e;
}

// a^K for a float-float a, rounded to float: float-float up to the last
// squaring (or multiplication), which is done in FP32 on the pair
template <int K>
BOYS_F32_DEVFN float f32_power_tail(ff a) {
  if constexpr (K == 0) {
    return 1.0f;
  } else if constexpr (K == 1) {
    return a.hi;
  } else {
    const ff h = ff_ipow<K / 2>(a);
    // (h.hi + h.lo)^2 ~ h.hi^2 + 2 h.hi h.lo
    const float sq = fmaf(h.hi, h.hi, 2.0f * h.hi * h.lo);
    if constexpr (K % 2) {
      return sq * a.hi;
    } else {
      return sq;
    }
  }
}

// Below the cut-off z_{NTOP,24}: Eqs. "pqz", "fq" and "r" (denominator read
// as 2m-1), as in the double path.
// 1/d as a pair of floats, h + l, for the long recursions
template <int D>
struct F32RecipPair {
  static constexpr float h = 1.0f / float(D);
  static constexpr float l = float(1.0 / double(D) - double(h));
};

// Eq. "r" from F_M (in fm) down to F_0, storing F_m for m <= NMAX, with
// 1/(2m - 1) as a float pair: over a long recursion the rounding of the
// constants themselves, the same for every argument, would otherwise add up.
template <int M, int NMAX>
BOYS_F32_DEVFN void f32_recurse_pair(const float tx, const float e, float &fm, float (&F)[NMAX + 1]) {
  if constexpr (M <= NMAX) F[M] = fm;
  if constexpr (M >= 1) {
    const float sm = fmaf(tx, fm, e);
    fm = fmaf(sm, F32RecipPair<2 * M - 1>::h, sm * F32RecipPair<2 * M - 1>::l);
    f32_recurse_pair<M - 1, NMAX>(tx, e, fm, F);
  }
}

// From this order on the float path evaluates the rational part of Q~ in
// float-float: the closed form multiplies a relative error of Q by s^2 (T/D),
// and at high orders T/D stays near 1 far out in x, where q2 x^2 u/v is a
// large part of Q (at n = 37, float u/v and float coefficients cost the
// closed form 5e-6; in float-float it keeps about 1e-6).
constexpr int kF32FFRationalFrom = 18;

template <int NTOP, int NMAX>
BOYS_F32_DEVFN void f32_formula(const float x, float (&F)[NMAX + 1], const float *tab) {
  using Tab = BoysF32<NTOP>;
  ff q = ff_add(ff{Tab::kQ0hi, Tab::kQ0lo}, ff_mul_f(ff{Tab::kQ1hi, Tab::kQ1lo}, x));
  if constexpr (NTOP < kF32FFRationalFrom) {
    float u, v;
    Tab::uv(x, u, v);
    // the rational part enters Q with weight ~x^2, where the amplification has
    // fallen off: a couple of ulp in u/v cost nothing measurable
    const float t = ((Tab::kQ2 * x) * x) * boys_fdiv_approx(u, v);
    q = ff_add_f(q, t);
  } else {
    ff u, v;
    Tab::uv_ff(x, u, v);
    const ff r = ff_mul(u, ff_rcp(v, boys_fdiv_approx(1.0f, v.hi)));
    q = ff_add(q, ff_mul(ff_mul_f(ff_mul_f(ff{Tab::kQ2, Tab::kQ2lo}, x), x), r));
  }
  const ff e = ff_exp_neg(x, tab);
  const ff T = ff_mul(ff_mul(ff_ipow<NTOP>(q), ff_sqrt(q, boys_rsqrtf(q.hi))), e);
  const ff D = ff_add_f(T, x);
  const ff w = ff_rcp(D, boys_fdiv_approx(1.0f, D.hi));  // seed; the Newton step restores ~46 bits
  // D^{-s} = w^NTOP sqrt(w): w carries the error of D amplified by s, so it
  // stays float-float; the power is float-float up to its last squaring,
  // which (with sqrt(w) and c) rounds only a few times in FP32.  Above
  // n = 17, c_n and w^NTOP would leave the float range (c_35 > FLT_MAX, and
  // w^NTOP < FLT_MIN near the cut-off) although F_n does not, so there
  // F_n = (C w)^NTOP sqrt(C w) with C = c_n^(1/(n+1/2)), about 13 at n = 37.
  float f;
  if constexpr (NTOP <= 17) {
    f = f32_power_tail<NTOP>(w) * (Tab::kChi * (w.hi * boys_rsqrtf(w.hi)));
  } else {
    const ff cw = ff_mul(ff{Tab::kCshi, Tab::kCslo}, w);
    f = f32_power_tail<NTOP>(cw) * (cw.hi * boys_rsqrtf(cw.hi));
  }
  const float tx = x + x;
  float fm = f;
  if constexpr (NTOP < kF32FFRationalFrom) {
#pragma unroll
    for (int m = NTOP; m >= 1; --m) {
      if (m <= NMAX) F[m] = fm;
      fm = fmaf(tx, fm, e.hi) * (1.0f / float(2 * m - 1));
    }
    F[0] = fm;
  } else {
    f32_recurse_pair<NTOP, NMAX>(tx, e.hi, fm, F);
  }
}

// From this n_max on the asymptote's chain is compensated (below).
constexpr int kF32CompensatedChainFrom = 17;

// Above the cut-off (or x negative, infinite or NaN): the asymptote of
// Eq. "limf1" built upward from F_0 = c_0 / sqrt(x),
// F_m = F_{m-1} (m - 1/2) y with y = 1/x.
// In plain FP32 each order adds two roundings, and the rounding of y itself
// grows as m in y^m: about 2.5e-6 at m = 36.  From n_max = 17 on the chain
// is a compensated product (Graillat, IEEE Trans. Comput. 58(7), 2009): the
// exact rounding errors of a_m = (m - 1/2) y and of each product, found with
// fused multiply-adds, are carried in e and added back to every F_m, and the
// error of y is removed through rho = 1 - x y (1/x = y (1 + rho + ...), so
// y^m carries a factor 1 + m rho).  Every F_m is then within about one
// rounding of c_0 x^{-1/2} prod (k - 1/2) / x.
template <int NMAX>
BOYS_F32_DEVFN void f32_asymptote(const float x, float (&F)[NMAX + 1]) {
  const float rs = boys_rsqrtf(x);
  float f = 0.886226925452758f * rs;
  F[0] = f;
  const float y = boys_frcp_rn(x);
  if constexpr (NMAX < kF32CompensatedChainFrom) {
#pragma unroll
    for (int m = 1; m <= NMAX; ++m) {
      f = f * ((float(m) - 0.5f) * y);
      F[m] = f;
    }
  } else {
    // x = +inf gives y = 0 and the row 0; rho would be NaN there
    const float rho = x < 3.0e38f ? fmaf(-x, y, 1.0f) : 0.0f;
    float e = 0.0f;
#pragma unroll
    for (int m = 1; m <= NMAX; ++m) {
      const float h = float(m) - 0.5f;
      const float a = h * y;
      const float ea = fmaf(h, y, -a);  // exact: a + ea = h y
      const float p = f * a;
      const float ep = fmaf(f, a, -p);  // exact: p + ep = f a
      e = fmaf(e, a, fmaf(f, ea, ep));
      f = p;
      F[m] = fmaf(f, float(m) * rho, f + e);
    }
  }
}

}  // namespace boys
