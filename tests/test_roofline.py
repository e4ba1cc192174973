"""The op-count model behind the FP64 roofline, against the code the kernels run.

`roofline.root_product_ops` is what the roofline charges for one evaluation of
the root products u(x), v(x) of Q~ (Eqs. "pz"/"qz"); here it is compared with
the floating-point operations written out in each generated `uv()` body of
`csrc/boys_coeffs_f64.inc`, and with the count the generator recorded beside
them.  The two-point count must be the two closed forms plus both
recursions and one exponential."""
import os
import re

import pytest

from paper_2504_07637_gb300 import roofline

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "paper_2504_07637_gb300", "csrc", "boys_coeffs_f64.inc")


def _uv_bodies():
    src = open(INC).read()
    out = {}
    for m in re.finditer(r"template <> struct BoysF64<(\d+)> \{(.*?)\n\};", src, re.S):
        n, body = int(m.group(1)), m.group(2)
        ops = int(re.search(r"kRootOps = (\d+);", body).group(1))
        uv = body[body.index("void uv("):]
        out[n] = (ops, uv)
    return out


def _count_fp_ops(code: str) -> int:
    # every fma(...) call and every binary +, -, * between operands (the
    # generator writes them with a space on each side; literals carry no sign)
    return code.count("fma(") + len(re.findall(r"\s[-+*]\s", code))


BODIES = _uv_bodies()


@pytest.mark.parametrize("n", sorted(BODIES))
def test_root_product_ops_match_generated_code(n):
    recorded, uv = BODIES[n]
    fit = roofline._fits(53)[n]
    model = roofline.root_product_ops(fit["u"]) + roofline.root_product_ops(fit["v"])
    assert _count_fp_ops(uv) == model
    assert recorded == model


def test_square_multiply_counts():
    # binary powering: squarings for the bits below the top one, a multiply
    # per further set bit (x^1 costs nothing, x^9 = ((x^2)^2)^2 x)
    assert [roofline.square_multiply_ops(k) for k in (0, 1, 2, 3, 4, 9, 15, 40)] == [0, 0, 1, 2, 2, 4, 6, 6]


def test_two_point_is_two_closed_forms_and_two_recursions():
    n_max, n_top, n_bar, n_top_lo = 36, 40, 18, 20
    one, above1 = roofline.f64_counts(n_max, n_top)
    lo, _ = roofline.f64_counts(n_bar, n_top_lo)
    two, above2 = roofline.f64_counts_two_point(n_max, n_top, n_bar, n_top_lo)
    assert above1 == above2
    assert two["exp"] == 1
    assert two["rsqrt"] == one["rsqrt"] + lo["rsqrt"] and two["div"] == one["div"] + lo["div"]
    # each one-point count holds its full recursion (2 n_top); the two-point
    # recursions run n_top -> n_bar + 1 and n_top_lo -> 0
    assert two["fma"] == (one["fma"] - 2 * n_top) + (lo["fma"] - 2 * n_top_lo) + 2 * (n_top - n_bar - 1) + 2 * n_top_lo
