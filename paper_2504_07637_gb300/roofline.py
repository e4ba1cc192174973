"""Algorithmic work per argument of the Boys evaluation, for the roofline.

Counts follow the method (Sec. 2) as the double kernels evaluate it: below the
cut-off one evaluation of Q~ in root-product form, one division u/v, one
exponential (shared with the recursion, Eq. "r"), the half-integer powers
Q^{n+1/2} and D^{-(n+1/2)} as square-and-multiply plus a reciprocal square
root each (below n_max = 12 and in the two-point rows the kernels take
everything after Q~, and up to n_max = 5 and from n_max = 12 on the
exponential, from 64-bit integer significands), and two operations per step of
the downward recursion (on the integer pipes instead in the row kernels, and
for recursions of up to 18 steps elsewhere); above it (Eq. "limf1") nothing
on the FP64 pipe: F_0 and
1/x come from a reciprocal square root by Newton steps on 64-bit integer
significands, and the upward product chain runs there too.  The all-FP64
form (int_chain=False) counts one reciprocal square root, F_0, 1/x and the
chain's two products per order instead.  "fma" counts every add, multiply or
fused multiply-add (each one FP64-pipe instruction).  Bytes per argument are
the input value plus the n_max+1 outputs.
"""
from __future__ import annotations

import json
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def _fits(bits: int) -> dict:
    with open(os.path.join(_HERE, "coeffs", f"boys_fit_b{bits}.json")) as fh:
        return {r["n"]: r for r in json.load(fh)["fits"]}


def root_product_ops(fac: dict) -> int:
    """Adds/multiplies of one monic root-product polynomial as generated."""
    deg_poly = len(fac["poly"]) - 1
    ops = deg_poly  # Horner on the gathered polynomial (first step is an add)
    nfac = (1 if deg_poly >= 1 else 0) + len(fac["quad"]) + len(fac["lin"])
    ops += 2 * len(fac["quad"]) + len(fac["lin"])  # (x-y), fma(t,t,a) / (x-y)
    ops += max(0, nfac - 1)  # products joining the factors
    return ops


def square_multiply_ops(k: int) -> int:
    """Multiplications of x^k by repeated squaring."""
    if k <= 1:
        return 0
    return (k.bit_length() - 1) + (bin(k).count("1") - 1)


def int_rsqrt(n_max: int, two_point: bool = False) -> bool:
    """Whether the closed form takes its reciprocal square roots from integer
    Newton steps (f64_int_rsqrt in csrc/boys_f64.cuh): below n_max = 12 and
    in the two-point rows."""
    return two_point or n_max < INT_RSQRT_BELOW


INT_RSQRT_BELOW = 12
INT_EXP_UPTO = 5


def int_exp(n_max: int, two_point: bool = False) -> bool:
    """Whether e^{-x} runs on the integer pipes (f64_int_exp in
    csrc/boys_f64.cuh): the one-point rows up to n_max = 5 and from
    n_max = 12 on."""
    return not two_point and (n_max <= INT_EXP_UPTO or n_max >= INT_RSQRT_BELOW)


def _closed_form_counts(n_top: int, int_newton: bool = True) -> dict:
    """FP64 operations of F_{n_top} by the closed form (Eq. "fq") given
    e^{-x}: Q~ in root-product form with one division u/v, Q^n, sqrt(Q), D
    and D^{-s}.  int_newton: everything after Q on 64-bit integer
    significands (T = Q^n Q r_Q e^{-x}, D = x + T, r_D = D^{-1/2} by Newton
    steps, D^{-s} = r_D (r_D^2)^n times c), so the FP64 pipe keeps Q~ and
    the division.  In FP64 (int_newton False): Q^n, Q rsqrt(Q), and
    rsqrt(D)^{2n+1} for n_top <= 13, else (1/D)^n (1/D) rsqrt(1/D)."""
    rec = _fits(53)[n_top]
    pw = square_multiply_ops(n_top)
    fma = root_product_ops(rec["u"]) + root_product_ops(rec["v"]) + 4  # Q~ (given u/v)
    if int_newton:
        return {"fma": fma, "div": 1, "sqrt": 0, "exp": 0, "rsqrt": 0}
    fma += pw + 1 + 1 + 1 + 1  # Q^n, Q rsqrt(Q), product, times e^{-x}, plus x
    if n_top <= 13:
        fma += 1 + pw + 2  # rs^2, its power, c rs and the product
        rsq, div = 2, 1
    else:
        fma += pw + 1 + 2  # w^n, w rsqrt(w), c w^n and the product
        rsq, div = 2, 2
    return {"fma": fma, "div": div, "sqrt": 0, "exp": 0, "rsqrt": rsq}


_NONE = {"fma": 0, "div": 0, "sqrt": 0, "exp": 0, "rsqrt": 0}


def _asymptote_start_fp64(n_max: int) -> dict:
    """F_0 = c_0 rsqrt(x) and y = 1/x in FP64: one reciprocal square root,
    one product, y as rsqrt(x)^2 for n_max <= 12, else a division."""
    return {"fma": 1 + (1 if 1 <= n_max <= 12 else 0), "div": 1 if n_max > 12 else 0, "sqrt": 0, "exp": 0,
            "rsqrt": 1}


def _asymptote_counts(n_max: int, int_chain: bool = True) -> dict:
    """FP64 operations of the asymptote row (Eq. "limf1"): F_0 = c_0 / sqrt(x),
    y = 1/x and the upward chain F_m = F_{m-1} (m - 1/2) y.  The kernels form
    F_0 and y by Newton steps for 1/sqrt(x) and run the chain, all on 64-bit
    integer significands (csrc/boys_sig64.cuh), which leaves the FP64 pipe
    nothing; int_chain=False counts the FP64 forms instead: a reciprocal
    square root, F_0, y and two multiplications per order."""
    if int_chain:
        return dict(_NONE)
    c = _asymptote_start_fp64(n_max)
    c["fma"] += 2 * n_max
    return c


def int_chain_orders(n_max: int) -> int:
    """Orders of the asymptote row computed on the integer pipes (two 64-bit
    significand products and one rounding each)."""
    return n_max


# The kernels run the downward recursion on 64-bit integer significands when
# it unrolls at most this many steps (f64_int_recursion in csrc/boys_f64.cuh),
# and always in the one-point row kernels from n_max = 12 on, which stage
# their rows and loop over chunks of orders.
INT_RECURSION_MAX_STEPS = 18
STAGED_ROWS_FROM = 12


def int_recursion(steps: int, n_max: int | None = None) -> bool:
    """Whether a recursion of this many steps runs on the integer pipes; with
    n_max given, in the row kernel of that order, else in an unstaged one
    (the fused contraction and the gradient)."""
    return steps <= INT_RECURSION_MAX_STEPS or (n_max is not None and n_max >= STAGED_ROWS_FROM)


def f64_counts(n_max: int, n_top: int, int_chain: bool = True, rows: bool = True) -> tuple[dict, dict]:
    """(below-cut-off, above-cut-off) FP64 operation counts per argument, in
    the form the double kernels evaluate them: the closed form at n_top and
    one exponential below the cut-off, plus two operations per step of the
    downward recursion (Eq. "r") where it runs in FP64; the asymptote above
    it.  rows: the row kernel (else an unstaged epilogue kernel).  With
    int_chain False, the recursion and the asymptote's chain are both
    counted in FP64 (the all-FP64 kernel)."""
    below = _closed_form_counts(n_top, int_chain and int_rsqrt(n_max))
    below["exp"] = 0 if int_chain and int_exp(n_max) else 1  # else on the integer pipes
    if not (int_chain and int_recursion(n_top, n_max if rows else None)):
        below["fma"] += 2 * n_top  # recursion
    return below, _asymptote_counts(n_max, int_chain)


def f64_counts_two_point(n_max: int, n_top: int, n_bar: int, n_top_lo: int,
                         int_chain: bool = True) -> tuple[dict, dict]:
    """As f64_counts for the two-point evaluation (Trick B of Sec. 3): closed
    forms at n_top and at n_top_lo sharing one exponential, the recursion
    from n_top down to n_bar + 1 and the one from n_top_lo down to 0."""
    below = _closed_form_counts(n_top, int_chain)
    lo = _closed_form_counts(n_top_lo, int_chain)
    for k in below:
        below[k] += lo[k]
    below["exp"] = 1
    steps = (n_top - (n_bar + 1)) + n_top_lo
    if not (int_chain and int_recursion(steps)):  # the two-point rows keep the step rule
        below["fma"] += 2 * steps
    return below, _asymptote_counts(n_max, int_chain)


def f64_counts_contract(n_max: int, n_top: int, uniform: bool = True, int_chain: bool = True) -> tuple[dict, dict]:
    """As f64_counts for the fused contraction sum_m c_m F_m: below the
    cut-off the row as f64_counts plus the n_max + 1 term dot product; above
    it, with the same coefficients for every argument and n_max <= 16, the
    contraction of the asymptote as a polynomial in y = 1/x (Horner, n_max
    fused multiply-adds and the product with F_0, F_0 and y from the integer
    start, or in FP64 with int_chain False), else the asymptote row and the
    dot product."""
    below, above = f64_counts(n_max, n_top, int_chain, rows=False)
    below["fma"] += n_max + 1
    if uniform and n_max <= 16:
        above = dict(_NONE) if int_chain else _asymptote_start_fp64(n_max)
        above["fma"] += n_max + 1
    else:
        above = dict(above)
        above["fma"] += n_max + 1
    return below, above


def bytes_per_arg(n_max: int, elem: int = 8) -> int:
    return elem * (1 + n_max + 1)
