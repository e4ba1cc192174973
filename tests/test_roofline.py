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
    one, above1 = roofline.f64_counts(n_max, n_top, int_chain=False)
    lo, _ = roofline.f64_counts(n_bar, n_top_lo, int_chain=False)
    two, above2 = roofline.f64_counts_two_point(n_max, n_top, n_bar, n_top_lo, int_chain=False)
    assert above1 == above2
    assert two["exp"] == 1
    assert two["rsqrt"] == one["rsqrt"] + lo["rsqrt"] and two["div"] == one["div"] + lo["div"]
    # each one-point count holds its full recursion (2 n_top); the two-point
    # recursions run n_top -> n_bar + 1 and n_top_lo -> 0
    assert two["fma"] == (one["fma"] - 2 * n_top) + (lo["fma"] - 2 * n_top_lo) + 2 * (n_top - n_bar - 1) + 2 * n_top_lo


def test_contraction_counts():
    # below the cut-off: the row plus an (n_max + 1)-term dot product; above it
    # with uniform weights: Horner in y = 1/x and the product with F_0, F_0 and
    # y from the integer start (in FP64: a reciprocal square root, F_0, and y
    # as rs^2 up to n_max = 12, else a division)
    for n_max, n_top in ((0, 0), (8, 9), (16, 18)):
        row_b, row_a = roofline.f64_counts(n_max, n_top)
        b, a = roofline.f64_counts_contract(n_max, n_top, uniform=True)
        assert b["fma"] == row_b["fma"] + n_max + 1 and b["exp"] == (0 if n_max <= 5 or n_max >= 12 else 1)
        assert a["fma"] == n_max + 1 and a["rsqrt"] == 0 and a["div"] == 0
        _, a64 = roofline.f64_counts_contract(n_max, n_top, uniform=True, int_chain=False)
        assert a64["fma"] == n_max + 2 + (1 if 1 <= n_max <= 12 else 0) and a64["rsqrt"] == 1
        assert a64["div"] == (1 if n_max > 12 else 0)
        # cheaper than the row and its dot product in FP64; with the row on the
        # integer pipes, no dearer than its dot product
        fp64_row = roofline.f64_counts(n_max, n_top, int_chain=False)[1]["fma"]
        assert a64["fma"] < fp64_row + n_max + 1 or n_max == 0
        assert a["fma"] <= row_a["fma"] + n_max + 1
    b, a = roofline.f64_counts_contract(36, 40, uniform=True)  # no Horner above n_max = 16
    assert a["fma"] == roofline.f64_counts(36, 40)[1]["fma"] + 37


def test_asymptote_leaves_the_fp64_pipe():
    # the upward chain's two multiplications per order, and F_0 = c_0 / sqrt(x)
    # and y = 1/x (Newton steps for 1/sqrt(x)), run on the integer pipes; the
    # all-FP64 form takes a reciprocal square root, F_0, y (rs^2 up to
    # n_max = 12, else a division) and the chain
    for n_max in (0, 1, 8, 12, 13, 36):
        _, a = roofline.f64_counts(n_max, n_max)
        _, a64 = roofline.f64_counts(n_max, n_max, int_chain=False)
        assert a == {"fma": 0, "div": 0, "sqrt": 0, "exp": 0, "rsqrt": 0}
        assert a64["fma"] == 1 + (1 if 1 <= n_max <= 12 else 0) + 2 * roofline.int_chain_orders(n_max)
        assert a64["rsqrt"] == 1 and a64["div"] == (1 if n_max > 12 else 0)


def test_integer_recursion_threshold_matches_the_kernels():
    # the kernels' rule (csrc/boys_f64.cuh) and the model's are the same
    import re

    src = open(os.path.join(os.path.dirname(roofline.__file__), "csrc", "boys_f64.cuh")).read()
    m = re.search(r"constexpr bool f64_int_recursion\(int steps\) \{ return steps <= (\d+); \}", src)
    assert m and int(m.group(1)) == roofline.INT_RECURSION_MAX_STEPS
    # in the row kernels every recursion leaves the FP64 pipe (from n_max = 12
    # on they loop over chunks of orders); in the unstaged epilogue kernels
    # only those of up to 18 steps
    for n_max, n_top in ((8, 9), (16, 18), (17, 19), (36, 40)):
        b, _ = roofline.f64_counts(n_max, n_top)
        b64, _ = roofline.f64_counts(n_max, n_top, int_chain=False)
        # the closed form's own difference below n_max = 12: rsqrt(Q) and
        # D^{-1/2} as integer Newton steps
        cf = roofline._closed_form_counts(n_top, False)["fma"] - roofline._closed_form_counts(n_top, True)["fma"]
        cf = cf if roofline.int_rsqrt(n_max) else 0
        assert b64["fma"] - b["fma"] == 2 * n_top + cf
        e, _ = roofline.f64_counts(n_max, n_top, rows=False)
        assert b64["fma"] - e["fma"] == cf + (2 * n_top if n_top <= 18 else 0)
    assert "f64_recurse_staged<NTOP, 0, NMAX, W, CH, K, true>" in src


def test_closed_form_newton_steps_leave_the_fp64_pipe():
    # below n_max = 12 and in the two-point rows everything after Q runs on
    # integer significands (the powers, Q rsqrt(Q), e^{-x}, + x, D^{-1/2} by
    # Newton steps): the FP64 pipe keeps Q~ and the division u/v; the FP64
    # form adds both powers (square and multiply), seven products and sums,
    # and the reciprocal square roots (and 1/D from n_top = 14 on)
    for n_top in (1, 9, 13, 14, 18, 40):
        c = roofline._closed_form_counts(n_top)
        c64 = roofline._closed_form_counts(n_top, False)
        assert c["rsqrt"] == 0 and c["div"] == 1
        assert c64["rsqrt"] == 2 and c64["div"] == (1 if n_top <= 13 else 2)
        assert c64["fma"] - c["fma"] == 2 * roofline.square_multiply_ops(n_top) + 7
    import re

    src = open(os.path.join(os.path.dirname(roofline.__file__), "csrc", "boys_f64.cuh")).read()
    m = re.search(r"constexpr bool f64_int_rsqrt\(int n_max, bool two\) \{ return two \|\| n_max < (\d+); \}", src)
    assert m and int(m.group(1)) == roofline.INT_RSQRT_BELOW
    for n_max, n_top in ((8, 9), (11, 12), (12, 13), (16, 18)):
        b, _ = roofline.f64_counts(n_max, n_top)
        assert b["rsqrt"] == (0 if n_max < 12 else 2)
        two, _ = roofline.f64_counts_two_point(n_max, n_top, n_max // 2, n_max // 2 + 1)
        assert two["rsqrt"] == 0


def test_integer_exponential_rule_matches_the_kernels():
    import re

    src = open(os.path.join(os.path.dirname(roofline.__file__), "csrc", "boys_f64.cuh")).read()
    m = re.search(r"constexpr bool f64_int_exp\(int n_max, bool two\) \{ return !two && \(n_max <= (\d+) \|\| n_max >= (\d+)\); \}", src)
    assert m and int(m.group(1)) == roofline.INT_EXP_UPTO and int(m.group(2)) == roofline.INT_RSQRT_BELOW
    for n_max in (0, 5, 6, 11, 12, 16, 36):
        b, _ = roofline.f64_counts(n_max, n_max + 1)
        assert b["exp"] == (0 if n_max <= 5 or n_max >= 12 else 1)
    two, _ = roofline.f64_counts_two_point(16, 18, 8, 9)
    assert two["exp"] == 1
