"""The integer significand arithmetic of the asymptote's product chain
(csrc/boys_sig64.cuh), compiled for the host and checked against exact
integer and rational arithmetic: the truncated 64 x 64 high product, the
rounding of a significand to a double, the constants prod_{k<=m} (k - 1/2)
and the bound below which every F_m of the chain is a normal double."""
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
#include <cstdio>
using namespace boys;
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
    src.write_text(HARNESS)
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
