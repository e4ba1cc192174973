// 64-bit significand arithmetic on the integer pipes.
//
// Above the cut-off the Boys row is the asymptote of Eq. "limf1",
// F_m = F_0 prod_{k<=m} (k - 1/2) / x, a chain of 2 n_max double
// multiplications.  GB300 retires about 1.7 FP64 operations per clock per SM,
// but its integer pipes take 32-bit multiply-adds at a far higher rate, and
// in this kernel they are nearly idle.  So the chain runs on integers:
// values are s 2^(e - 63) with a 64-bit significand s in [2^63, 2^64), one
// product is three 32 x 32 -> 64-bit multiply-adds, and each F_m is rounded
// to a double once.  With 11 guard bits every F_m is within one rounding of
// the exact chain from F_0 and 1/x, against 2m roundings for the double
// chain.
//
// The downward recursion of Eq. "r", F_{m-1} = (2x F_m + e^{-x}) / (2m - 1),
// has only positive terms, so it runs the same way: a product, an aligned
// sum and a product with the constant 1/(2m - 1) per order.
//
// Everything here is plain integer arithmetic, valid on the host too.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define BOYS_HD __host__ __device__ __forceinline__
#define BOYS_HD_CONSTEXPR __host__ __device__ constexpr
#else
#define BOYS_HD inline
#define BOYS_HD_CONSTEXPR constexpr
#endif

namespace boys {

// A positive number s 2^(e - 63), s in [2^63, 2^64).
struct Sig64 {
  uint64_t s;
  int e;
};

// floor(a b / 2^64) minus at most 1: with a = a1 2^32 + a0 and b likewise,
// a b = a1 b1 2^64 + (a1 b0 + a0 b1) 2^32 + a0 b0, and the low half of the
// cross products' sum and all of a0 b0 (together below 2^65) are left out.
// For a, b >= 2^63 the result is at least 2^62, so its relative error is
// below 2^-62.
BOYS_HD uint64_t mulhi_trunc(uint64_t a, uint64_t b) {
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
  const uint64_t u = (uint64_t)a0 * b1;
  // a1 b0 + (u mod 2^32) <= (2^32 - 1)^2 + 2^32 - 1 < 2^64: no overflow
  const uint64_t v = (uint64_t)a1 * b0 + (uint32_t)u;
  return (uint64_t)a1 * b1 + (u >> 32) + (v >> 32);
}

// The significand and exponent of the magnitude of a normal double, from its
// bits (the sign is ignored).
BOYS_HD uint64_t sig64_of_bits(uint64_t bits) { return (bits << 11) | (1ull << 63); }
BOYS_HD int exp_of_bits(uint64_t bits) { return (int)((bits >> 52) & 0x7ff) - 1023; }

// The product of two Sig64 numbers: (s_a, e_a) (s_b, e_b) -> (s, e).
// mulhi_trunc gives t in [2^62, 2^64), the product being t 2^(e_a + e_b - 62);
// one left shift when t < 2^63 normalises it.
BOYS_HD void sig64_mul(uint64_t &s, int &e, uint64_t sb, int eb) {
  const uint64_t t = mulhi_trunc(s, sb);
  const int top = (int)(t >> 63);
  s = top ? t : t << 1;
  e += eb + top;
}

// The sum of two Sig64 numbers: (s_a, e_a) + (s_b, e_b) -> (s, e).  The
// smaller is shifted to the larger's exponent (truncated; by 63 at most, so a
// negligible one adds a unit of 2^-63 relative), and a carry out of the
// 64-bit sum is shifted back in.  Relative error below 2^-62.
BOYS_HD void sig64_add(uint64_t &s, int &e, uint64_t sb, int eb) {
  const int d = e - eb;
  const uint64_t big = d >= 0 ? s : sb;
  uint64_t small = d >= 0 ? sb : s;
  const int ad = d >= 0 ? d : -d;
  small >>= (ad < 63 ? ad : 63);
  e = d >= 0 ? e : eb;
  const uint64_t sum = big + small;
  const int carry = sum < big;
  s = carry ? (sum >> 1) | (1ull << 63) : sum;
  e += carry;
}

// The bits of the double nearest s 2^(e - 63) (ties away from zero), for a
// result in the normal range (-1022 <= e <= 1023).  Rounding up to 2^53
// carries into the exponent field, which is the right value.
BOYS_HD uint64_t sig64_round_bits(uint64_t s, int e) {
  const uint64_t m = (s >> 11) + ((s >> 10) & 1);
  return m + ((uint64_t)(e + 1022) << 52);
}

// r + c (d >= 0) or r - c (d < 0) for a correction c below r 2^-18, renormalised
// (a carry out of the 64 bits, or a fall below 2^63, moves the exponent by
// one).  Selects, not branches: the sign of d differs from lane to lane.
BOYS_HD void sig64_nudge(uint64_t &s, int &e, int64_t d, uint64_t c) {
  const uint64_t up = s + c, dn = s - c;
  const bool pos = d >= 0;
  const bool carry = pos && up < s;
  const bool borrow = !pos && dn < (1ull << 63);
  const uint64_t u = pos ? up : dn;
  s = carry ? (u >> 1) | (1ull << 63) : (borrow ? u << 1 : u);
  e += (int)carry - (int)borrow;
}

// 1/sqrt(x) for a positive normal double x, by Newton's method on 64-bit
// significands.  Write x = a 4^k with a in [1, 4).  sig64_rsqrt_reduce gives
// k and the bits of a float holding a's leading 24 bits, whose reciprocal
// square root (a float approximation, e.g. the device's rsqrtf) seeds r;
// sig64_rsqrt then takes two steps r <- r (1 + d/2), d = 1 - a r^2, each of
// which maps a relative error eps to about 3 eps^2 / 2 (2^-20 -> 2^-39 ->
// 2^-77).  d is formed in fixed point from t = a r^2, which the products leave
// within 2^-18 of 1: |d| 2^64 < 2^46 as a signed integer.  The products add
// relative errors below 2^-62 each, so the result is within 2^-60 of
// 1/sqrt(x) for a seed within 2^-20 of 1/sqrt(a).
BOYS_HD uint32_t sig64_rsqrt_reduce(uint64_t xbits, int &k) {
  const int ex = exp_of_bits(xbits);
  const int p = ex & 1;  // ex = 2k + p, also for negative ex (two's complement)
  k = (ex - p) / 2;
  return ((uint32_t)(127 + p) << 23) | (uint32_t)((xbits >> 29) & 0x7fffffu);
}

// The seed's argument for a Sig64 value s 2^(e - 63): a float holding the
// leading 24 bits of a = s 2^(p - 63) in [1, 4), p = e mod 2.
BOYS_HD uint32_t sig64_rsqrt_seed_arg(uint64_t s, int e) {
  return ((uint32_t)(127 + (e & 1)) << 23) | (uint32_t)((s >> 40) & 0x7fffffu);
}

// 1/sqrt of the positive number sa 2^(ea - 63), sa in [2^63, 2^64), from a
// seed within 2^-20 of 1/sqrt(a) (a as in sig64_rsqrt_seed_arg).
BOYS_HD void sig64_rsqrt_sig(uint64_t sa, int ea, uint32_t seed_bits, uint64_t &s, int &e) {
  const int p = ea & 1;  // ea = 2k + p, also for negative ea (two's complement)
  const int k = (ea - p) / 2;
  uint64_t sr = (uint64_t)((seed_bits & 0x7fffffu) | 0x800000u) << 40;
  int er = (int)((seed_bits >> 23) & 0xffu) - 127;
  for (int it = 0; it < 2; ++it) {
    uint64_t t = sr;
    int et = er;
    sig64_mul(t, et, sr, er);
    sig64_mul(t, et, sa, p);
    // d 2^64 from t 2^(et - 63), et being -1 (t < 1) or 0 (t >= 1)
    const int64_t d = et == 0 ? -(int64_t)((t - (1ull << 63)) << 1) : (int64_t)(0ull - t);
    sig64_nudge(sr, er, d, mulhi_trunc(sr, d < 0 ? (uint64_t)(-d) : (uint64_t)d) >> 1);  // r |d| / 2
  }
  s = sr;
  e = er - k;
}

// The same for a positive normal double x.
BOYS_HD void sig64_rsqrt(uint64_t xbits, uint32_t seed_bits, uint64_t &s, int &e) {
  sig64_rsqrt_sig(sig64_of_bits(xbits), exp_of_bits(xbits), seed_bits, s, e);
}

// x^n (n >= 0) by repeated squaring, each product a sig64_mul.
template <int N>
BOYS_HD void sig64_pow(uint64_t &s, int &e) {
  static_assert(N >= 0, "power");
  if constexpr (N == 0) {
    s = 1ull << 63;
    e = 0;
  } else if constexpr (N > 1) {
    uint64_t bs = s;
    int be = e;
    sig64_pow<N / 2>(bs, be);
    sig64_mul(bs, be, bs, be);
    if constexpr (N % 2 == 1) sig64_mul(bs, be, s, e);
    s = bs;
    e = be;
  }
}

// The high 64 bits of a 64 x 64-bit product, unsigned and signed (floor).
BOYS_HD uint64_t mulhi_u64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}
BOYS_HD int64_t mulhi_s64(int64_t a, int64_t b) {
#if defined(__CUDA_ARCH__)
  return __mul64hi(a, b);
#else
  return (int64_t)(((__int128)a * b) >> 64);
#endif
}

// e^{-x} for 0 <= x < 128 as a Sig64, by Tang's table-driven method in 64-bit
// fixed point:
//   X = x 2^57 (exact for x >= 2^-5, else within 2^-57; 0 below 2^-57),
//   k = round(x 64/ln2), r = x - k ln2/64 (|r| <= ln2/128 plus 2^-50):
//   R = X - k Lh - (k Ll) 2^-64, with ln2/64 2^57 = Lh + Ll 2^-64,
//   e^{-r} = sum_{i<=6} (-r)^i / i! by Horner on 2^62-scaled coefficients
//   (the first term left out is below 2^-65; each step truncates 2^-62),
//   e^{-x} = 2^q 2^(j/64) e^{-r} with -k = 64 q + j, 2^(j/64) from tab (the
//   64-bit significands round(2^(j/64) 2^63)).
// The error is below 2^-55 relative (R within 1.5 units of 2^-57).
constexpr uint64_t kExpInvL = 0xb8aa3b295c17f0bcull;  // round(64/ln2 2^57)
constexpr uint64_t kExpLh = 0x58b90bfbe8e7bull;       // floor(ln2/64 2^57)
constexpr uint64_t kExpLl = 0xcd5e4f1d9cc01f98ull;    // its remainder 2^64, rounded
// round((-1)^i / i! 2^62), i = 0..6
constexpr int64_t kExpA0 = 4611686018427387904ll, kExpA1 = -4611686018427387904ll, kExpA2 = 2305843009213693952ll,
                  kExpA3 = -768614336404564651ll, kExpA4 = 192153584101141163ll, kExpA5 = -38430716820228233ll,
                  kExpA6 = 6405119470038039ll;
BOYS_HD void sig64_exp_neg(uint64_t xbits, const uint64_t *tab, uint64_t &s, int &e) {
  const int ex = exp_of_bits(xbits);  // -1023 for 0 and subnormals
  const int sh = 6 - ex;
  const uint64_t X = sh < 64 ? sig64_of_bits(xbits) >> sh : 0ull;
  const int64_t k = (int64_t)((mulhi_u64(X, kExpInvL) + (1ull << 49)) >> 50);
  const int64_t R = (int64_t)(X - (uint64_t)k * kExpLh - mulhi_u64((uint64_t)k, kExpLl));
  const int64_t R7 = R * 128;  // r 2^64 (|R| < 2^50)
  int64_t acc = kExpA5 + mulhi_s64(R7, kExpA6);
  acc = kExpA4 + mulhi_s64(R7, acc);
  acc = kExpA3 + mulhi_s64(R7, acc);
  acc = kExpA2 + mulhi_s64(R7, acc);
  acc = kExpA1 + mulhi_s64(R7, acc);
  acc = kExpA0 + mulhi_s64(R7, acc);
  // acc = e^{-r} 2^62 in (2^61, 2^63)
  const bool hi = acc >= (int64_t)(1ull << 62);
  const uint64_t sq = hi ? (uint64_t)acc << 1 : (uint64_t)acc << 2;
  const int64_t nk = -k;
  s = tab[nk & 63];
  e = 0;
  sig64_mul(s, e, sq, hi ? 0 : -1);
  e += (int)(nk >> 6);
}

// c_0 = sqrt(pi)/2 (Eq. "limf1": F_0 = c_0 / sqrt(x) above the cut-off),
// rounded to 64 bits: 0.886226925452758013649... = 0xe2dfc48da77b553d 2^-64.
constexpr uint64_t kSig64C0s = 0xe2dfc48da77b553dull;
constexpr int kSig64C0e = -1;

// prod_{k=1}^{m} (k - 1/2) = (2m - 1)!! / 2^m as a Sig64, each factor
// applied exactly and the product rounded to 64 bits (relative error below
// m 2^-64).  (2k - 1) s needs at most 71 bits, held as hi 2^32 + lo.
BOYS_HD_CONSTEXPR Sig64 half_odd_product(int m) {
  uint64_t s = 1ull << 63;
  int e = 0;
  for (int k = 1; k <= m; ++k) {
    const uint64_t odd = (uint64_t)(2 * k - 1);
    const uint64_t plo = (s & 0xffffffffull) * odd;
    const uint64_t hi = (s >> 32) * odd + (plo >> 32);
    const uint64_t lo = plo & 0xffffffffull;
    int r = 0;  // the product is in [2^(63 + r), 2^(64 + r))
    while ((hi >> (32 + r)) != 0) ++r;
    uint64_t t = (hi << (32 - r)) | (lo >> r);
    if (r > 0) t += (lo >> (r - 1)) & 1;  // round to nearest
    if (t == 0) {                         // rounded up to 2^64
      t = 1ull << 63;
      ++r;
    }
    s = t;
    e += r - 1;  // (k - 1/2) = (2k - 1) / 2
  }
  return Sig64{s, e};
}

// 1/d for an odd d >= 1 as a Sig64, rounded to nearest: for d >= 3, with
// 2^(k-1) < d < 2^k, s = round(2^(63+k) / d) by long division (the leading
// quotient bit of 2^(63+k) is 0) and e = -k.
BOYS_HD_CONSTEXPR Sig64 recip_odd(int d) {
  if (d == 1) return Sig64{1ull << 63, 0};
  int k = 0;
  while ((1 << k) < d) ++k;
  uint64_t q = 0, r = 1;  // dividend: a one followed by 63 + k zeros
  for (int i = 0; i < 63 + k; ++i) {
    r <<= 1;
    const uint64_t bit = r >= (uint64_t)d ? 1 : 0;
    r -= bit * (uint64_t)d;
    q = (q << 1) | bit;
  }
  if (2 * r >= (uint64_t)d) ++q;
  return Sig64{q, -k};
}

// The bits of a bound x_max below which the integer chain gives every F_m,
// m <= n_max, in the normal range: for x < 2^floor(2038/(2n+1)),
// F_n(x) >= c_1 x^-(n+1/2) > 2^-1021 (n >= 1), and 1/x is normal.  +inf when
// the bound is beyond the double range (n_max = 0, where there is no chain).
BOYS_HD_CONSTEXPR uint64_t sig64_chain_xmax_bits(int n_max) {
  const int l = 2038 / (2 * n_max + 1);
  return l >= 1024 ? 0x7ff0000000000000ull : (uint64_t)(l + 1023) << 52;
}

}  // namespace boys
