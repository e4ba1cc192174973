"""Pins for the CPU oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: a closed
form, a library special function, an independent evaluation branch, a limit
or an identity of Eq. "fn".  A plausible slip (a dropped term, a wrong sign,
an off-by-one order, a wrong denominator) fails at least one of them.
"""
import math

import numpy as np
import pytest

ORDERS = [0, 1, 2, 5, 8, 9, 13, 16, 17, 25, 36]


def _logspace(lo, hi, k):
    return np.exp(np.linspace(math.log(lo), math.log(hi), k))


def test_zero_argument_is_reciprocal_odd(oracle_mod):
    # Eq. "fn" at x = 0: int_0^1 t^{2m} dt = 1/(2m+1)
    f = oracle_mod.boys([0.0], 40)[0]
    assert np.array_equal(f, 1.0 / (2 * np.arange(41) + 1))


def test_small_argument_taylor(oracle_mod):
    # d/dx F_m(0) = -F_{m+1}(0) = -1/(2m+3);  second derivative 1/(2m+5)
    for x in (1e-300, 1e-30, 1e-12, 1e-6):
        f = oracle_mod.boys_ld([x], 30)[0]
        m = np.arange(31)
        taylor = 1.0 / (2 * m + 1) - x / (2 * m + 3) + x * x / 2 / (2 * m + 5)
        rel = np.abs(f.astype(np.float64) / taylor - 1)
        assert rel.max() < 1e-15, (x, rel.max())


def test_f0_closed_form_erf(oracle_mod):
    # F_0(x) = 1/2 sqrt(pi/x) erf(sqrt x)  (Eq. "fn" with n = 0); both branches
    x = np.concatenate([_logspace(1e-6, 2000, 400), [119.999, 120.0, 120.001, 1e5, 1e8]])
    got = oracle_mod.boys(x, 17)[:, 0]
    want = np.array([0.5 * math.sqrt(math.pi / v) * math.erf(math.sqrt(v)) for v in x])
    assert np.max(np.abs(got / want - 1)) < 1e-15  # a few ulp of the double reference


def test_regularized_gamma_scipy(oracle_mod):
    # x^{m+1/2} F_m(x) / c_m = P(m+1/2, x)  (regularized lower incomplete gamma),
    # c_m = Gamma(m+1/2)/2 (the c_n of Sec. 2); scipy is an independent library.
    sp = pytest.importorskip("scipy.special")
    x = _logspace(1e-3, 400, 300)
    n_max = 36
    f = oracle_mod.boys(x, n_max)
    for m in range(0, n_max + 1, 3):
        s = m + 0.5
        p = sp.gammainc(s, x)
        c = math.gamma(s) / 2
        got = x**s * f[:, m] / c
        ok = p > 1e-250
        assert np.max(np.abs(got[ok] / p[ok] - 1)) < 5e-13, m


def test_mpmath_40_digits(oracle_mod):
    # F_m(x) = gamma(m+1/2, x) / (2 x^{m+1/2}), evaluated by mpmath at 40 digits
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(7)
    x = np.concatenate([_logspace(1e-5, 1e4, 60), rng.uniform(0, 150, 40)])
    n_max = 37
    f = oracle_mod.boys_ld(x, n_max)
    eps = 2.0 ** (1 - oracle_mod.precision_bits())
    worst = 0.0
    for i, xv in enumerate(x):
        X = mp.mpf(float(xv))
        for m in range(0, n_max + 1, 4):
            s = mp.mpf(m) + mp.mpf(1) / 2
            ref = mp.gammainc(s, 0, X) / (2 * X**s)
            worst = max(worst, abs(float(mp.mpf(str(f[i, m])) / ref - 1)))
    assert worst < 2000 * eps, worst


def test_large_argument_limit(oracle_mod):
    # Eq. "limf1": F_m(x) -> c_m x^{-(m+1/2)}, c_m = (2m)! sqrt(pi) / (m! 2^{2m+1})
    for x in (2e3, 1e5, 1e7):
        f = oracle_mod.boys([x], 30)[0]
        for m in range(31):
            c = math.factorial(2 * m) * math.sqrt(math.pi) / (math.factorial(m) * 2 ** (2 * m + 1))
            assert abs(f[m] / (c * x ** -(m + 0.5)) - 1) < 1e-14


def test_c_constant_product_form(oracle_mod):
    c = oracle_mod.c_ld(30).astype(np.float64)
    for m in range(31):
        want = math.factorial(2 * m) * math.sqrt(math.pi) / (math.factorial(m) * 2 ** (2 * m + 1))
        assert abs(c[m] / want - 1) < 1e-15


@pytest.mark.parametrize("n", ORDERS)
def test_series_vs_quadrature(oracle_mod, n):
    # branch (2) against Gauss-Legendre quadrature of the definition itself
    x = np.concatenate([_logspace(1e-4, 300, 50), [0.3, 2.0, 57.7, 110.0]]).astype(np.longdouble)
    a = oracle_mod.series_ld(x, n)
    b = oracle_mod.quad_ld(x, n)
    eps = 2.0 ** (1 - oracle_mod.precision_bits())
    assert np.max(np.abs(a / b - 1)) < 4000 * eps


@pytest.mark.parametrize("n_max", [1, 8, 17, 36])
def test_branches_agree_in_overlap(oracle_mod, n_max):
    # erf + upward recursion vs series + downward recursion, where both are valid
    x = np.linspace(2 * n_max + 5, 300, 40).astype(np.longdouble)
    up = oracle_mod.erf_upward_ld(x, n_max)
    eps = 2.0 ** (1 - oracle_mod.precision_bits())
    for m in range(n_max + 1):
        s = oracle_mod.series_ld(x, m)
        assert np.max(np.abs(up[:, m] / s - 1)) < 4000 * eps, m


def test_recursion_identity(oracle_mod):
    # integration by parts of Eq. "fn":  (2m+1) F_m = 2x F_{m+1} + e^{-x}
    x = _logspace(1e-3, 500, 200).astype(np.longdouble)
    f = oracle_mod.boys_ld(x, 20)
    e = np.exp(-x)
    eps = 2.0 ** (1 - oracle_mod.precision_bits())
    for m in range(20):
        lhs = (2 * m + 1) * f[:, m]
        rhs = 2 * x * f[:, m + 1] + e
        assert np.max(np.abs(lhs / rhs - 1)) < 200 * eps


def test_derivative_is_minus_next_order(oracle_mod):
    # d/dx F_m = -F_{m+1}: fourth-order central differences in long double
    x = np.concatenate([_logspace(0.05, 300, 40)]).astype(np.longdouble)
    n_max = 12
    for xv in x:
        h = np.longdouble(1e-3) * max(np.longdouble(1), xv) ** np.longdouble(0.5)
        pts = np.array([xv - 2 * h, xv - h, xv + h, xv + 2 * h], dtype=np.longdouble)
        f = oracle_mod.boys_ld(pts, n_max + 1)
        fd = (8 * (f[2] - f[1]) - (f[3] - f[0])) / (12 * h)
        ref = -oracle_mod.boys_ld([xv], n_max + 1)[0]
        rel = np.abs(fd[: n_max + 1] / ref[1:] - 1)
        assert rel.max() < 1e-9, (xv, rel.max())


def test_monotone_in_x_and_order(oracle_mod):
    x = np.linspace(0, 200, 2001)
    f = oracle_mod.boys(x, 16)
    assert np.all(np.diff(f, axis=0) <= 0)
    assert np.all(np.diff(f, axis=1) < 0)


def test_domain_convention(oracle_mod):
    f = oracle_mod.boys([-1.0, -0.0, np.nan, np.inf, -np.inf], 5)
    assert np.all(np.isnan(f[0])) and np.all(np.isnan(f[2])) and np.all(np.isnan(f[4]))
    assert np.array_equal(f[1], 1.0 / (2 * np.arange(6) + 1))  # -0.0 == 0
    assert np.all(f[3] == 0.0)


def test_cutoff_matches_inverse_gamma(oracle_mod):
    # z_nb solves R(n+1/2, z) = 2^{-b}: scipy's inverse of the regularized upper gamma
    sp = pytest.importorskip("scipy.special")
    for b in (24, 53):
        for n in (0, 1, 4, 8, 9, 16, 17, 36):
            z = oracle_mod.cutoff(n, b)
            assert abs(z / sp.gammainccinv(n + 0.5, 2.0**-b) - 1) < 1e-10, (n, b)


def test_cutoff_satisfies_defining_equation(oracle_mod):
    # Sec. 2: z^{n+1/2} F_n(z) / c_n = 1 - 2^{-b}, with F from the oracle's own branches
    # (b = 53 would leave only ~10 bits of the x86 long double to resolve 1 - lhs)
    c = oracle_mod.c_ld(40)
    for b in (24, 40):
        for n in (0, 3, 8, 17, 30):
            z = np.longdouble(oracle_mod.cutoff(n, b))
            f = oracle_mod.boys_ld([z], n)[0, n]
            lhs = z ** (np.longdouble(n) + np.longdouble(0.5)) * f / c[n]
            assert abs(float((1 - lhs) / np.longdouble(2.0**-b)) - 1) < 2e-3, (n, b)


def test_upper_ratio_is_complement(oracle_mod):
    # R = 1 - P, with P from the oracle's F (independent code paths)
    c = oracle_mod.c_ld(20)
    x = _logspace(0.01, 30, 50).astype(np.longdouble)
    f = oracle_mod.boys_ld(x, 20)
    for n in (0, 5, 20):
        r = oracle_mod.upper_ratio_ld(n, x)
        p = x ** (np.longdouble(n) + np.longdouble(0.5)) * f[:, n] / c[n]
        assert np.max(np.abs(r + p - 1)) < 1e-17


def test_gradient_oracle(oracle_mod):
    # grad of sum_m w_m F_m is -sum_m w_m F_{m+1}; one-hot weights give -F_{m+1}
    rng = np.random.default_rng(3)
    x = _logspace(1e-3, 1e3, 64)
    n_max = 9
    f = oracle_mod.boys(x, n_max + 1)
    for m in range(n_max + 1):
        w = np.zeros(n_max + 1)
        w[m] = 1.0
        assert np.array_equal(oracle_mod.grad(x, w, n_max), -f[:, m + 1])
    g = rng.standard_normal((x.size, n_max + 1))
    got = oracle_mod.grad(x, g, n_max)
    want = -(g * f[:, 1:]).sum(axis=1)
    scale = (np.abs(g) * f[:, 1:]).sum(axis=1)
    assert np.max(np.abs(got - want) / scale) < 1e-15
