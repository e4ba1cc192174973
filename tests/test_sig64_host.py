"""The integer significand arithmetic of the FP64 kernels' downward recursion
and asymptote (csrc/boys_sig64.cuh), compiled for the host and checked
against exact integer and rational arithmetic (the truncated 64 x 64 high
product, the rounding of a significand to a double, the constants
prod_{k<=m} (k - 1/2), 1/(2m - 1) and sqrt(pi)/2, the reciprocal square root
by Newton steps, the bound below which every F_m of the chain is a normal
double), and, composed as the kernels compose it, against the oracle."""
import math
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_2504_07637_gb300", "csrc", "boys_sig64.cuh")

HARNESS = r"""
#include "boys_sig64.cuh"
#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>
using namespace boys;
// the closed form after Q as the kernels form it on the integer pipes (n_top
// known at compile time): T = Q^n Q r_Q e^{-x}, D = x + T, r_D = D^{-1/2},
// F = c r_D (r_D^2)^n, from doubles q, e, x, c (the seeds: float 1/sqrt)
static uint32_t host_seed(uint32_t abits) {  // 1/sqrt(a) in float, a in [1, 4)
  float a, r;
  std::memcpy(&a, &abits, 4);
  r = 1.0f / std::sqrt(a);
  uint32_t rb;
  std::memcpy(&rb, &r, 4);
  return rb;
}
template <int N>
uint64_t tail(uint64_t qb, uint64_t ebits, uint64_t xb, uint64_t cb) {
  const uint64_t sq = sig64_of_bits(qb);
  const int eq = exp_of_bits(qb);
  uint64_t sr, st = sq;
  int er, et = eq, k;
  sig64_rsqrt(qb, host_seed(sig64_rsqrt_reduce(qb, k)), sr, er);
  sig64_pow<N>(st, et);
  sig64_mul(st, et, sq, eq);
  sig64_mul(st, et, sr, er);
  sig64_mul(st, et, sig64_of_bits(ebits), exp_of_bits(ebits));
  if (((xb >> 52) & 0x7ff) != 0) sig64_add(st, et, sig64_of_bits(xb), exp_of_bits(xb));
  uint64_t sd, sw;
  int ed, ew;
  sig64_rsqrt_sig(st, et, host_seed(sig64_rsqrt_seed_arg(st, et)), sd, ed);
  sw = sd;
  ew = ed;
  sig64_mul(sw, ew, sd, ed);
  sig64_pow<N>(sw, ew);
  sig64_mul(sw, ew, sd, ed);
  sig64_mul(sw, ew, sig64_of_bits(cb), exp_of_bits(cb));
  return sig64_round_bits(sw, ew);
}

template <int... N>
void pow_all(uint64_t s0, int e0, std::integer_sequence<int, N...>) {
  auto one = [&](auto n) {
    uint64_t s = s0;
    int e = e0;
    sig64_pow<decltype(n)::value>(s, e);
    std::printf("%llu %d ", (unsigned long long)s, e);
  };
  (one(std::integral_constant<int, N>{}), ...);
}
int main() {
  char op[8];
  unsigned long long a, b;
  int e;
  while (std::scanf("%7s", op) == 1) {
    if (op[0] == 'm') {  // m a b: mulhi_trunc
      std::scanf("%llu %llu", &a, &b);
      std::printf("%llu\n", (unsigned long long)mulhi_trunc(a, b));
    } else if (op[0] == 'r') {  // r s e: sig64_round_bits
      std::scanf("%llu %d", &a, &e);
      std::printf("%llu\n", (unsigned long long)sig64_round_bits(a, e));
    } else if (op[0] == 'h') {  // h m: half_odd_product
      std::scanf("%d", &e);
      const Sig64 h = half_odd_product(e);
      std::printf("%llu %d\n", (unsigned long long)h.s, h.e);
    } else if (op[0] == 'x') {  // x n: sig64_chain_xmax_bits
      std::scanf("%d", &e);
      std::printf("%llu\n", (unsigned long long)sig64_chain_xmax_bits(e));
    } else if (op[0] == 'd') {  // d top x_bits f_bits e_bits: F_top-1 .. F_0 by the integer recursion
      unsigned long long xb, fb, eb;
      std::scanf("%d %llu %llu %llu", &e, &xb, &fb, &eb);
      const unsigned long long tb = xb + (1ull << 52);  // 2x as the kernels form it
      uint64_t sf = sig64_of_bits(fb), sx = sig64_of_bits(tb), se = sig64_of_bits(eb);
      int ef = exp_of_bits(fb), ex = exp_of_bits(tb), ee = exp_of_bits(eb);
      for (int m = e; m >= 1; --m) {
        sig64_mul(sf, ef, sx, ex);
        sig64_add(sf, ef, se, ee);
        const Sig64 k = recip_odd(2 * m - 1);
        sig64_mul(sf, ef, k.s, k.e);
        std::printf("%llu ", (unsigned long long)sig64_round_bits(sf, ef));
      }
      std::printf("\n");
    } else if (op[0] == 'q') {  // q x_bits seed_bits: 1/sqrt(x) by sig64_rsqrt
      unsigned long long xb;
      unsigned sb;
      std::scanf("%llu %u", &xb, &sb);
      uint64_t s;
      int es;
      sig64_rsqrt(xb, sb, s, es);
      std::printf("%llu %d\n", (unsigned long long)s, es);
    } else if (op[0] == 'p') {  // p s e: s 2^(e - 63) to the powers 0 .. 40, as sig64_pow
      unsigned long long sb;
      std::scanf("%llu %d", &sb, &e);
      pow_all(sb, e, std::make_integer_sequence<int, 41>{});
      std::printf("\n");
    } else if (op[0] == 's') {  // s sig e seed_bits: 1/sqrt of s 2^(e - 63) by sig64_rsqrt_sig
      unsigned long long sb;
      unsigned seed;
      std::scanf("%llu %d %u", &sb, &e, &seed);
      uint64_t s;
      int es;
      sig64_rsqrt_sig(sb, e, seed, s, es);
      std::printf("%llu %d %u\n", (unsigned long long)s, es, sig64_rsqrt_seed_arg(sb, e));
    } else if (op[0] == 'E') {  // E x_bits: e^{-x} by sig64_exp_neg
      unsigned long long xb;
      std::scanf("%llu", &xb);
      static const uint64_t tab[64] = BOYS_EXP2_FRAC64_SIG;
      uint64_t s;
      int es;
      sig64_exp_neg(xb, tab, s, es);
      std::printf("%llu %d\n", (unsigned long long)s, es);
    } else if (op[0] == 'T') {  // T n q e x c: the closed form's integer tail
      unsigned long long qb, eb2, xb, cb;
      std::scanf("%d %llu %llu %llu %llu", &e, &qb, &eb2, &xb, &cb);
      unsigned long long r = 0;
      switch (e) {
        case 1: r = tail<1>(qb, eb2, xb, cb); break;
        case 5: r = tail<5>(qb, eb2, xb, cb); break;
        case 9: r = tail<9>(qb, eb2, xb, cb); break;
        case 13: r = tail<13>(qb, eb2, xb, cb); break;
        case 20: r = tail<20>(qb, eb2, xb, cb); break;
        case 40: r = tail<40>(qb, eb2, xb, cb); break;
      }
      std::printf("%llu\n", r);
    } else if (op[0] == 'k') {  // k x_bits: sig64_rsqrt_reduce
      unsigned long long xb;
      std::scanf("%llu", &xb);
      int k;
      const uint32_t ab = sig64_rsqrt_reduce(xb, k);
      std::printf("%u %d\n", ab, k);
    } else if (op[0] == 'a') {  // a n x_bits seed_bits: F_0 .. F_n as the kernels' integer asymptote
      unsigned long long xb;
      unsigned sb;
      std::scanf("%d %llu %u", &e, &xb, &sb);
      uint64_t sr, sy, s;
      int er, ey, es;
      sig64_rsqrt(xb, sb, sr, er);
      sy = sr;
      ey = er;
      sig64_mul(sy, ey, sr, er);  // y = r^2
      s = kSig64C0s;
      es = kSig64C0e;
      sig64_mul(s, es, sr, er);  // F_0 = c_0 r
      std::printf("%llu ", (unsigned long long)sig64_round_bits(s, es));
      for (int m = 1; m <= e; ++m) {
        sig64_mul(s, es, sy, ey);
        const Sig64 h = half_odd_product(m);
        uint64_t w = s;
        int ew = es;
        sig64_mul(w, ew, h.s, h.e);
        std::printf("%llu ", (unsigned long long)sig64_round_bits(w, ew));
      }
      std::printf("\n");
    } else if (op[0] == 'c') {  // c n f0_bits y_bits: F_1 .. F_n by the integer chain
      unsigned long long fb, yb;
      std::scanf("%d %llu %llu", &e, &fb, &yb);
      uint64_t s = sig64_of_bits(fb), sy = sig64_of_bits(yb);
      int es = exp_of_bits(fb), ey = exp_of_bits(yb);
      for (int m = 1; m <= e; ++m) {
        sig64_mul(s, es, sy, ey);
        const Sig64 h = half_odd_product(m);
        uint64_t w = s;
        int ew = es;
        sig64_mul(w, ew, h.s, h.e);
        std::printf("%llu ", (unsigned long long)sig64_round_bits(w, ew));
      }
      std::printf("\n");
    }
  }
}
"""


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("sig64")
    src = d / "h.cpp"
    # the exponential's table of 64-bit significands, from the generated coefficient header
    inc = open(os.path.join(os.path.dirname(HEADER), "boys_coeffs_f64.inc")).read()
    tab = next(line for line in inc.splitlines() if line.startswith("#define BOYS_EXP2_FRAC64_SIG "))
    src.write_text(tab + "\n" + HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)

    def call(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return out.stdout.split("\n")[: len(lines)]

    return call


def test_truncated_high_product_is_at_most_one_below_the_exact(run):
    rng = np.random.default_rng(7)
    pairs = [(int(a) | 1 << 63, int(b) | 1 << 63) for a, b in rng.integers(0, 2**63, size=(20000, 2), dtype=np.uint64)]
    edge = [1 << 63, (1 << 63) + 1, (1 << 64) - 1, 0xFFFFFFFF80000000, 0x80000000FFFFFFFF]
    pairs += [(a, b) for a in edge for b in edge]
    got = [int(v) for v in run([f"m {a} {b}" for a, b in pairs])]
    deficit = [(a * b >> 64) - g for (a, b), g in zip(pairs, got)]
    assert min(deficit) >= 0 and max(deficit) <= 1
    assert all(g >= 1 << 62 for g in got)


def _double(bits):
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def test_rounding_a_significand_to_a_double(run):
    rng = np.random.default_rng(8)
    cases = [(int(s) | 1 << 63, int(e)) for s, e in zip(rng.integers(0, 2**63, 5000, dtype=np.uint64),
                                                          rng.integers(-1022, 1023, 5000))]
    # halfway, just below halfway, and all ones (rounds up to the next power of two)
    cases += [((1 << 63) | (1 << 10), 0), ((1 << 63) | ((1 << 10) - 1), 5), ((1 << 64) - 1, -3), ((1 << 64) - 1, 1022)]
    got = [_double(int(v)) for v in run([f"r {s} {e}" for s, e in cases])]
    for (s, e), g in zip(cases, got):
        exact = Fraction(s) * Fraction(2) ** (e - 63)
        err = abs(Fraction(g) - exact)
        ulp = Fraction(2) ** (math.frexp(g)[1] - 53)
        assert err <= ulp / 2, (s, e, g)
        if (s & 0x7FF) != 0x400:  # away from ties the result is the nearest double
            assert err < ulp / 2 or g == float(exact), (s, e, g)


def test_half_odd_products_against_exact_fractions(run):
    got = [tuple(int(t) for t in line.split()) for line in run([f"h {m}" for m in range(0, 41)])]
    value = Fraction(1)
    for m, (s, e) in enumerate(got):
        if m:
            value *= Fraction(2 * m - 1, 2)
        assert 1 << 63 <= s < 1 << 64
        approx = Fraction(s) * Fraction(2) ** (e - 63)
        assert abs(approx / value - 1) <= m * Fraction(1, 2**64), m


def test_chain_bound_keeps_every_order_normal(run):
    """Below the bound, F_n's asymptote c_n x^-(n+1/2) (the smallest F_m of
    the row) is a normal double; the bound is a power of two and +inf for n=0."""
    got = [int(v) for v in run([f"x {n}" for n in range(0, 38)])]
    assert got[0] == 0x7FF0000000000000
    for n in range(1, 38):
        xmax = _double(got[n])
        assert xmax == math.ldexp(1.0, 2038 // (2 * n + 1))
        c_n = math.gamma(n + 0.5) / 2
        log2_fn = math.log2(c_n) - (n + 0.5) * math.log2(xmax)
        assert log2_fn > -1022, n
        assert 1.0 / xmax > np.finfo(np.float64).tiny


def _bits(v):
    return struct.unpack("<Q", struct.pack("<d", float(v)))[0]


def test_reciprocals_of_odd_numbers(run):
    # At x = 0 each step of the recursion is F_{k-1} = e^{-0} / (2k - 1): the
    # 2x F_k term (2x is 2^-1022 as the kernels form it) shifts out of the sum,
    # so every output is the constant 1/(2k - 1) times 1, rounded once, and
    # must be the correctly rounded double 1/(2k - 1), for k up to 41.
    lines = [f"d {m} {_bits(0.0)} {_bits(1.0 / (2 * m + 1))} {_bits(1.0)}" for m in range(1, 42)]
    for m, line in zip(range(1, 42), run(lines)):
        got = [_double(int(t)) for t in line.split()]
        want = [1.0 / (2 * k - 1) for k in range(m, 0, -1)]
        assert got == want, m


@pytest.mark.parametrize("top", [9, 18, 40])
def test_integer_recursion_against_the_oracle(run, oracle_mod, top):
    """The downward recursion (Eq. "r") on integer significands, from F_top and
    e^{-x} rounded to doubles as the kernels have them.  Each step is a
    weighted mean of the relative errors of F_m and e^{-x} (both terms are
    positive), so F_m carries at most the larger input rounding (2^-53) plus
    its own (2^-53) and the integer steps' truncation (below 2^-61 each):
    within 2.05 units of 2^-53 of the oracle's long double value.  The same
    recursion in double drifts further."""
    rng = np.random.default_rng(top)
    x = np.concatenate([[0.0, 5e-324, 1e-310, 1e-300, 1e-16], rng.uniform(0.0, 118.0, 3000),
                        np.exp(rng.uniform(-20, math.log(118.0), 1000))])
    ref = oracle_mod.boys_ld(x, top)  # F_0 .. F_top in long double
    ftop = ref[:, top].astype(np.float64)
    e = np.exp(-x)
    lines = [f"d {top} {_bits(v)} {_bits(f)} {_bits(ev)}" for v, f, ev in zip(x, ftop, e)]
    got = np.array([[_double(int(t)) for t in line.split()][::-1] for line in run(lines)])  # F_0 .. F_top-1
    rel = (np.abs(got - ref[:, :top]) / ref[:, :top]).astype(np.float64)
    assert rel.max() <= 2.05 * 2.0**-53, (top, rel.max() / 2.0**-53)
    # the same steps in double, for comparison
    f = ftop.copy()
    worst64 = 0.0
    for m in range(top, 0, -1):
        f = (2.0 * x * f + e) * (1.0 / (2 * m - 1))
        worst64 = max(worst64, float(np.max(np.abs(f - ref[:, m - 1]) / ref[:, m - 1])))
    assert rel.max() <= worst64


@pytest.mark.parametrize("n", [1, 8, 12, 16, 36])
def test_integer_chain_against_the_oracle(run, oracle_mod, n):
    """The asymptote's upward chain (Eq. "limf1") on integer significands from
    F_0 = c_0 / sqrt(x) and y = 1/x as doubles, for x above the cut-off and
    below the chain's range bound: F_m = F_0 y^m prod (k - 1/2) carries F_0's
    error (three roundings here), m times that of y (one rounding), its own
    rounding and the asymptote's distance from F_m (below 2^-53 above z): within
    3.5 + m units of 2^-53 of the oracle's long double value."""
    rng = np.random.default_rng(100 + n)
    xmax = _double(int(run([f"x {n}"])[0]))
    z = oracle_mod.cutoff(n, 53)
    x = np.exp(rng.uniform(math.log(z), math.log(min(xmax, 1e300)) - 1e-9, 2000))
    f0 = 0.88622692545275801365 / np.sqrt(x)
    y = 1.0 / x
    lines = [f"c {n} {_bits(a)} {_bits(b)}" for a, b in zip(f0, y)]
    got = np.array([[_double(int(t)) for t in line.split()] for line in run(lines)])  # F_1 .. F_n
    ref = oracle_mod.boys_ld(x, n)[:, 1:]
    rel = (np.abs(got - ref) / ref).astype(np.float64)
    bound = (3.5 + np.arange(1, n + 1)) * 2.0**-53
    assert np.all(rel.max(axis=0) <= bound), (rel.max(axis=0) / 2.0**-53)


def _float_bits(v):
    return struct.unpack("<I", struct.pack("<f", v))[0]


def _float(bits):
    return struct.unpack("<f", struct.pack("<I", bits))[0]


def _seeds(run, xs, rng, spread):
    """The kernels' seed: x = a 4^k, a's leading bits as a float (checked
    here), then a float approximation of 1/sqrt(a), here the nearest float
    moved by up to `spread` relative (the device's rsqrtf is within 2^-22)."""
    red = [line.split() for line in run([f"k {_bits(x)}" for x in xs])]
    seeds = []
    for x, (ab, k) in zip(xs, red):
        a = _float(int(ab))
        assert 1.0 <= a < 4.0 and abs(Fraction(a) * Fraction(4) ** int(k) / Fraction(float(x)) - 1) < Fraction(1, 2**23)
        r0 = np.float32(1.0 / math.sqrt(a) * (1.0 + rng.uniform(-spread, spread)))
        seeds.append(_float_bits(r0))
    return seeds


def test_reciprocal_square_root_by_newton_steps(run):
    """sig64_rsqrt from seeds within 2^-20 of 1/sqrt(a): within 2^-60 of
    1/sqrt(x) over the whole normal range, both exponent parities and the
    seeds' power-of-two edges (r = 1 exactly at a = 1)."""
    rng = np.random.default_rng(21)
    xs = list(np.exp(rng.uniform(math.log(2.3e-308), math.log(1.7e308), 4000)))
    xs += [1.0, 2.0, 4.0, 0.25, 0.5, 3.9999999999999996, 1.0000000000000002, 2.2250738585072014e-308,
           1.7976931348623157e308, 7.0, 110.0, 1e8]
    seeds = _seeds(run, xs, rng, 2.0**-20)
    got = [tuple(int(t) for t in line.split()) for line in run([f"q {_bits(x)} {s}" for x, s in zip(xs, seeds)])]
    for x, (s, e) in zip(xs, got):
        assert 1 << 63 <= s < 1 << 64
        r = Fraction(s) * Fraction(2) ** (e - 63)
        # r^2 x = (1 + eps)^2: |eps| <= 2^-60 within |r^2 x - 1| <= 2^-59 + 2^-120
        assert abs(r * r * Fraction(float(x)) - 1) <= Fraction(1, 2**59) + Fraction(1, 2**120), x


def test_powers_by_repeated_squaring(run):
    """sig64_pow: x^n for n = 0 .. 40 (the closed form's Q^n_top and
    w^n_top) within n 2^-62 relative of the exact power (each of its at most
    2 log2(n) products truncates below 2^-62)."""
    rng = np.random.default_rng(23)
    cases = [(int(s) | 1 << 63, int(e)) for s, e in zip(rng.integers(0, 2**63, 60, dtype=np.uint64),
                                                          rng.integers(-40, 40, 60))]
    cases += [(1 << 63, 0), ((1 << 64) - 1, 3), ((1 << 63) + 1, -5)]
    for (s0, e0), line in zip(cases, run([f"p {s} {e}" for s, e in cases])):
        t = [int(v) for v in line.split()]
        x = Fraction(s0) * Fraction(2) ** (e0 - 63)
        for n in range(41):
            s, e = t[2 * n], t[2 * n + 1]
            assert 1 << 63 <= s < 1 << 64
            got = Fraction(s) * Fraction(2) ** (e - 63)
            assert abs(got / x**n - 1) <= Fraction(max(n, 1), 2**61), (s0, e0, n)


def test_reciprocal_square_root_of_a_significand(run):
    """sig64_rsqrt_sig on values s 2^(e - 63) of either exponent parity (D of
    the closed form), seeded as the kernels seed it from sig64_rsqrt_seed_arg:
    within 2^-60 of 1/sqrt."""
    rng = np.random.default_rng(24)
    cases = [(int(s) | 1 << 63, int(e)) for s, e in zip(rng.integers(0, 2**63, 3000, dtype=np.uint64),
                                                          rng.integers(-300, 300, 3000))]
    cases += [(1 << 63, 0), (1 << 63, 1), ((1 << 64) - 1, -1), ((1 << 64) - 1, 2)]
    lines = []
    for s, e in cases:
        a = Fraction(s) * Fraction(2) ** ((e & 1) - 63)  # in [1, 4)
        seed = np.float32(1.0 / math.sqrt(float(a)) * (1.0 + rng.uniform(-(2.0**-20), 2.0**-20)))
        lines.append(f"s {s} {e} {_float_bits(seed)}")
    for (s0, e0), line in zip(cases, run(lines)):
        s, e, ab = (int(v) for v in line.split())
        a = _float(ab)
        assert 1.0 <= a < 4.0 and abs(Fraction(a) / (Fraction(s0) * Fraction(2) ** ((e0 & 1) - 63)) - 1) < Fraction(1, 2**23)
        r = Fraction(s) * Fraction(2) ** (e - 63)
        v = Fraction(s0) * Fraction(2) ** (e0 - 63)
        assert abs(r * r * v - 1) <= Fraction(1, 2**59) + Fraction(1, 2**120), (s0, e0)


def test_sqrt_pi_over_two_constant():
    # the 64-bit significand of c_0 = sqrt(pi)/2 in csrc/boys_sig64.cuh is the
    # nearest to 2^64 sqrt(pi)/2: its square times 4 brackets pi
    import re

    src = open(HEADER).read()
    s = int(re.search(r"kSig64C0s = (0x[0-9a-f]+)ull", src).group(1), 16)
    assert int(re.search(r"kSig64C0e = (-?\d+);", src).group(1)) == -1
    pi_lo, pi_hi = Fraction(314159265358979323846264338327950288, 10**35), Fraction(314159265358979323846264338327950289, 10**35)
    lo, hi = Fraction(s) - Fraction(1, 2), Fraction(s) + Fraction(1, 2)  # s 2^-64 within half a unit
    assert 4 * (lo / 2**64) ** 2 < pi_lo and pi_hi < 4 * (hi / 2**64) ** 2


@pytest.mark.parametrize("n", [0, 1, 8, 12, 16, 36])
def test_integer_asymptote_against_the_oracle(run, oracle_mod, n):
    """F_0 = c_0 / sqrt(x) and the chain, as the kernels form them above the
    cut-off on the integer pipes (sig64_rsqrt from a seed within 2^-21, y = r^2,
    F_0 = c_0 r, all to 64 bits): each F_m is one rounding (2^-53) from the
    exact asymptote, whose distance from F_m is below 2^-53 above z_{n,53},
    plus the 64-bit arithmetic (below m 2^-58): within 2 + m/32 units of 2^-53
    of the oracle's long double value."""
    rng = np.random.default_rng(200 + n)
    xmax = _double(int(run([f"x {max(n, 1)}"])[0])) if n else 1e300
    z = oracle_mod.cutoff(n, 53)
    x = np.exp(rng.uniform(math.log(z), math.log(min(xmax, 1e300)) - 1e-9, 2000))
    seeds = _seeds(run, list(x), rng, 2.0**-21)
    lines = [f"a {n} {_bits(a)} {s}" for a, s in zip(x, seeds)]
    got = np.array([[_double(int(t)) for t in line.split()] for line in run(lines)])  # F_0 .. F_n
    ref = oracle_mod.boys_ld(x, n)
    rel = (np.abs(got - ref) / ref).astype(np.float64)
    bound = (2.0 + np.arange(0, n + 1) / 32.0) * 2.0**-53
    assert np.all(rel.max(axis=0) <= bound), (rel.max(axis=0) / 2.0**-53)


def _exp2_sig_table():
    import re

    inc = open(os.path.join(os.path.dirname(HEADER), "boys_coeffs_f64.inc")).read()
    line = next(line for line in inc.splitlines() if line.startswith("#define BOYS_EXP2_FRAC64_SIG "))
    return [int(v, 16) for v in re.findall(r"0x([0-9a-f]+)ull", line)]


def test_exp2_significand_table_is_correctly_rounded():
    # s_j = round(2^(j/64) 2^63): (s_j -+ 1/2)^64 brackets 2^(j + 64*63) exactly
    tab = _exp2_sig_table()
    assert len(tab) == 64 and tab[0] == 1 << 63
    for j, s in enumerate(tab):
        assert 1 << 63 <= s < 1 << 64
        target = 1 << (j + 64 * 63)
        assert (2 * s - 1) ** 64 <= target * 2**64 <= (2 * s + 1) ** 64, j


def test_integer_exponential_against_mpmath(run):
    """sig64_exp_neg (Tang's method in 64-bit fixed point) on [0, 128): within
    2^-55 relative of e^{-x} (the closed form's arguments stay below 120), at
    zero, subnormals, the reduction's edges (x near (k + 1/2) ln2/64) and the
    fixed point's (x near 2^-57 and 2^-5)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    rng = np.random.default_rng(25)
    xs = list(np.exp(rng.uniform(math.log(1e-30), math.log(127.9), 3000))) + list(rng.uniform(0.0, 127.99, 3000))
    half = math.log(2) / 128
    xs += [(2 * k + 1) * half * (1 + d) for k in (0, 1, 63, 64, 5000, 11000) for d in (-1e-15, 0.0, 1e-15)]
    xs += [0.0, 5e-324, 2.2250738585072014e-308, 2.0**-61, 2.0**-57, 2.0**-56, 2.0**-5, 0.03125 * (1 - 2.0**-52),
           1.0, 60.0, 118.0, 127.99]
    got = [tuple(int(t) for t in line.split()) for line in run([f"E {_bits(x)}" for x in xs])]
    for x, (s, e) in zip(xs, got):
        assert 1 << 63 <= s < 1 << 64
        v = mpmath.mpf(s) * mpmath.mpf(2) ** (e - 63)
        assert abs(v / mpmath.exp(-mpmath.mpf(x)) - 1) <= mpmath.mpf(2) ** -55, x


@pytest.mark.parametrize("n_top", [1, 5, 9, 13, 20, 40])
def test_integer_closed_form_tail_against_mpmath(run, n_top):
    """The closed form after Q (Eq. "fq") as the kernels form it on the integer
    pipes: F = c (x + Q^s e)^{-s}, s = n_top + 1/2, from the doubles Q, e, x
    and c, with the powers, Q rsqrt(Q), D = x + T and D^{-1/2} on 64-bit
    significands and one rounding at the end.  About 2 s truncations of at
    most 2^-62 in T and in D^{-s}, amplified by the power s, and the final
    rounding: within 1 + s^2/256 units of 2^-53 of the exact value.  Q is drawn
    around the value that gives F_{n_top}(0) = 1/(2 n_top + 1), x over the
    range below the cut-off."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 150
    rng = np.random.default_rng(300 + n_top)
    s = n_top + 0.5
    c = math.gamma(s) / 2
    q0 = (c * (2 * n_top + 1)) ** (1 / (s * s))
    q = q0 * np.exp(rng.uniform(math.log(0.97), math.log(1.05), 600))
    x = np.concatenate([[0.0, 5e-324], rng.uniform(0.0, 3 * n_top + 40, 598)])
    e = np.exp(-x)
    lines = [f"T {n_top} {_bits(a)} {_bits(b)} {_bits(xx)} {_bits(c)}" for a, b, xx in zip(q, e, x)]
    got = [_double(int(v)) for v in run(lines)]
    sm = mpmath.mpf(n_top) + mpmath.mpf(1) / 2
    bound = (1 + s * s / 256) * mpmath.mpf(2) ** -53
    for a, b, xx, g in zip(q, e, x, got):
        ref = mpmath.mpf(c) * (mpmath.mpf(xx) + mpmath.mpf(a) ** sm * mpmath.mpf(b)) ** (-sm)
        assert abs(mpmath.mpf(g) / ref - 1) <= bound, (n_top, a, xx)
