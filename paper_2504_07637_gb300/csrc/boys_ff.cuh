// Float-float ("double-word") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  On GB300 one FP64 instruction costs as much pipe
// time as ~64 FP32 instructions, so the handful of error-amplifying steps of
// the FP32 path run in this representation instead of in double.
//
// Building blocks, each from its published source:
//   two_sum       Knuth, TAOCP vol. 2, 4.2.2 (error-free sum, any order)
//   fast_two_sum  Dekker, Numer. Math. 18 (1971) (error-free sum, |a| >= |b|)
//   two_prod      exact product via one fused multiply-add (IEEE 754-2008 fma)
//   mul / add     double-word products and sums as analysed by Joldes, Muller
//                 and Popescu, ACM TOMS 44(4), 2017 (relative error a few u^2,
//                 u = 2^-24); add assumes operands of equal sign, which holds
//                 for every sum the Boys path forms (all terms positive)
//   sqrt, rcp     one Newton/Karp-Markstein correction of an FP32 seed
#pragma once

#ifdef __CUDACC__
#define BOYS_FF_HD __host__ __device__ __forceinline__
#else
#define BOYS_FF_HD inline
#include <cmath>
using std::fmaf;
using std::sqrt;
#endif

namespace boys {

struct ff {
  float hi, lo;
};

BOYS_FF_HD ff ff_make(float hi, float lo) { return ff{hi, lo}; }

BOYS_FF_HD ff fast_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return ff{s, e};
}

BOYS_FF_HD ff two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  const float e = (a - (s - bp)) + (b - bp);
  return ff{s, e};
}

BOYS_FF_HD ff two_prod(float a, float b) {
  const float p = a * b;
  return ff{p, fmaf(a, b, -p)};
}

BOYS_FF_HD ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  float e = fmaf(a.hi, b.lo, p.lo);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p.hi, e);
}

BOYS_FF_HD ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

BOYS_FF_HD ff ff_sqr(ff a) {
  ff p = two_prod(a.hi, a.hi);
  return fast_two_sum(p.hi, fmaf(a.hi + a.hi, a.lo, p.lo));
}

// a + b for a, b of equal sign
BOYS_FF_HD ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

BOYS_FF_HD ff ff_add_f(ff a, float b) {
  ff s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, s.lo + a.lo);
}

// x - y for any signs (the root factors x - y of Eqs. "pz"/"qz"): Knuth's
// error-free sum of x and -y.hi, then y.lo
BOYS_FF_HD ff ff_sub_f(ff y, float x) {
  const ff s = two_sum(x, -y.hi);
  return fast_two_sum(s.hi, s.lo - y.lo);
}

// sqrt(a), a > 0: seed s = a.hi * rsqrt(a.hi), then one correction with the
// exact residual a - s^2 (Karp and Markstein, ACM TOMS 23(4), 1997)
BOYS_FF_HD ff ff_sqrt(ff a, float rs) {
  const float s = a.hi * rs;
  const float e = fmaf(-s, s, a.hi) + a.lo;
  return fast_two_sum(s, e * (0.5f * rs));
}

// 1/a, a > 0, from an FP32 seed r ~ 1/a.hi: one Newton step on the exact residual
BOYS_FF_HD ff ff_rcp(ff a, float r) {
  const float e = fmaf(-a.hi, r, 1.0f) - a.lo * r;
  return fast_two_sum(r, r * e);
}

template <int K>
BOYS_FF_HD ff ff_ipow(ff a) {
  if constexpr (K == 0) {
    return ff{1.0f, 0.0f};
  } else if constexpr (K == 1) {
    return a;
  } else {
    const ff h = ff_ipow<K / 2>(a);
    if constexpr (K % 2) {
      return ff_mul(ff_sqr(h), a);
    } else {
      return ff_sqr(h);
    }
  }
}

}  // namespace boys
