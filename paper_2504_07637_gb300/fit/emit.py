"""Generate the CUDA coefficient header from the fitted table (offline tool).

Sec. 3 of the paper proposes generating the evaluation code from the
coefficient dataset with all loops unrolled; this emits, per order n, a
device function that evaluates Q~_n(x) = q0 + q1 x + q2 x^2 u(x)/v(x) in the
root-product form of Eqs. "pz"/"qz": the gathered negative-real-part roots as
one Horner polynomial, then the quadratic factors (x - y)^2 + a, then the
linear factors (x - y).  Constants (cut-offs z_nb and c_n) are emitted as
template specialisations usable from device and host code.

Usage:  python -m paper_2504_07637_gb300.fit.emit
"""
from __future__ import annotations

import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
COEFF_DIR = os.path.join(PKG, "coeffs")
CSRC = os.path.join(PKG, "csrc")


def d(v: str) -> str:
    """Decimal string -> C double literal (correctly rounded by Python)."""
    f = float(v)
    r = repr(f)
    if "e" not in r and "." not in r and "inf" not in r:
        r += ".0"
    return r


def poly_lines(name: str, fac: dict, var: str = "x", fma: str = "fma", ty: str = "double", lit=None) -> list[str]:
    """Statements computing the monic root-product polynomial into `name`."""
    lit = lit or d
    poly = fac["poly"]  # low -> high, monic
    lines = [f"{ty} {name};"]
    state = {"first": True}

    def mul(expr: str, indent: str = "") -> None:
        if state["first"]:
            lines.append(f"{indent}{name} = {expr};")
            state["first"] = False
        else:
            lines.append(f"{indent}{name} = {name} * {expr};")

    if len(poly) > 1:
        # Horner on the gathered negative-real-part polynomial (leading coefficient 1)
        lines.append(f"{{ {ty} h = {var} + {lit(poly[-2])};")
        for c in reversed(poly[:-2]):
            lines.append(f"  h = {fma}(h, {var}, {lit(c)});")
        mul("h", "  ")
        lines.append("}")
    for y, a in fac["quad"]:
        lines.append(f"{{ const {ty} t = {var} - {lit(y)};")
        mul(f"{fma}(t, t, {lit(a)})", "  ")
        lines.append("}")
    for y in fac["lin"]:
        mul(f"({var} - {lit(y)})")
    if state["first"]:
        lines.append(f"{name} = 1;")
    return lines


def op_count(fac: dict) -> int:
    """FP64 operations of one root-product evaluation (for the roofline)."""
    deg_poly = len(fac["poly"]) - 1
    ops = max(0, deg_poly - 1) + (1 if deg_poly >= 1 else 0)
    nfac = (1 if deg_poly >= 1 else 0) + len(fac["quad"]) + len(fac["lin"])
    ops += 2 * len(fac["quad"]) + len(fac["lin"]) + max(0, nfac - 1)
    return ops


def emit_f64(table: dict) -> str:
    fits = {r["n"]: r for r in table["fits"]}
    nmax = max(fits)
    missing = [n for n in range(nmax + 1) if n not in fits]
    if missing:
        raise SystemExit(f"missing fits for n = {missing}")
    out = [
        "// Generated by paper_2504_07637_gb300/fit/emit.py from coeffs/boys_fit_b53.json; do not edit.",
        "// Per order n: the constrained minimax fit of Q_n (Sec. 2, Eqs. pqz/pz/qz) in root-product form,",
        "// its cut-off z_{n,53} and c_n = Gamma(n+1/2)/2.",
        "#pragma once",
        f"#define BOYS_F64_TABLE_MAX_N {nmax}",
        "",
        "template <int N> struct BoysF64;",
        "",
    ]
    host_z, host_c, host_eps, ops = [], [], [], []
    for n in range(nmax + 1):
        r = fits[n]
        host_z.append(d(r["z"]))
        host_c.append(d(r["c"]))
        host_eps.append(f"{r['eps_bits']:.3f}")
        ops.append(op_count(r["u"]) + op_count(r["v"]))
        body = ["    " + ln for ln in poly_lines("u", r["u"])]
        body += ["    " + ln for ln in poly_lines("v", r["v"])]
        out += [
            f"// n = {n}: N = {r['N']}, exact-arithmetic error 2^-{r['eps_bits']:.2f}",
            f"template <> struct BoysF64<{n}> {{",
            f"  static constexpr int kOrderN = {r['N']};",
            f"  static constexpr double kCutoff = {d(r['z'])};",
            f"  static constexpr double kC = {d(r['c'])};",
            f"  static constexpr double kQ0 = {d(r['q0'])};",
            f"  static constexpr double kQ1 = {d(r['q1'])};",
            f"  static constexpr double kQ2 = {d(r['q2'])};",
            f"  static constexpr int kRootOps = {ops[-1]};",
            "  // u(x) and v(x) as root products; returns u and v separately",
            "  static __device__ __forceinline__ void uv(double x, double &u_out, double &v_out) {",
            *body,
            "    u_out = u;",
            "    v_out = v;",
            "  }",
            "};",
            "",
        ]
    out += [
        "// 2^(j/64), j = 0..63 (table of the exponential used by the kernels)",
        f"#define BOYS_EXP2_FRAC64 {{{exp2_table()}}}",
        "// the same as 64-bit significands: round(2^(j/64) 2^63) (the integer exponential)",
        f"#define BOYS_EXP2_FRAC64_SIG {{{exp2_table_sig()}}}",
        f"static const double kBoysF64CutoffHost[{nmax + 1}] = {{" + ", ".join(host_z) + "};",
        f"static const double kBoysCHost[{nmax + 1}] = {{" + ", ".join(host_c) + "};",
        f"static const float kBoysF64FitBitsHost[{nmax + 1}] = {{" + ", ".join(e + "f" for e in host_eps) + "};",
        f"static const int kBoysF64RootOpsHost[{nmax + 1}] = {{" + ", ".join(map(str, ops)) + "};",
        "",
    ]
    return "\n".join(out)


def f(v: str) -> str:
    """Decimal string -> C float literal (correctly rounded)."""
    import numpy as np

    r = repr(float(np.float32(float(v))))
    if "e" not in r and "." not in r:
        r += ".0"
    return r + "f"


def f_split(v: str) -> tuple[str, str]:
    """Decimal string -> (hi, lo) float literals with hi + lo = v to ~48 bits."""
    from decimal import Decimal, getcontext

    import numpy as np

    getcontext().prec = 60
    dv = Decimal(v)
    hi = np.float32(float(dv))
    lo = np.float32(float(dv - Decimal(float(hi))))
    fmt = lambda q: (repr(float(q)) + ("" if ("e" in repr(float(q)) or "." in repr(float(q))) else ".0")) + "f"
    return fmt(hi), fmt(lo)


def ff_lit(v: str) -> str:
    """Decimal string -> ff{hi, lo} literal (float-float, about 48 bits)."""
    hi, lo = f_split(v)
    return f"ff{{{hi}, {lo}}}"


def poly_lines_ff(name: str, fac: dict) -> list[str]:
    """Statements computing the monic root-product polynomial into the
    float-float `name`, with float-float coefficients: the same factors as
    poly_lines, for the orders whose rounding is amplified beyond float."""
    poly = fac["poly"]
    lines = [f"ff {name};"]
    state = {"first": True}

    def mul(expr: str, indent: str = "") -> None:
        if state["first"]:
            lines.append(f"{indent}{name} = {expr};")
            state["first"] = False
        else:
            lines.append(f"{indent}{name} = ff_mul({name}, {expr});")

    if len(poly) > 1:
        # the gathered negative-real-part roots: positive coefficients
        lines.append(f"{{ ff h = ff_add_f({ff_lit(poly[-2])}, x);")
        for c in reversed(poly[:-2]):
            lines.append(f"  h = ff_add(ff_mul_f(h, x), {ff_lit(c)});")
        mul("h", "  ")
        lines.append("}")
    for y, a in fac["quad"]:
        lines.append(f"{{ const ff t = ff_sub_f({ff_lit(y)}, x);")  # x - y
        mul(f"ff_add(ff_sqr(t), {ff_lit(a)})", "  ")
        lines.append("}")
    for y in fac["lin"]:
        mul(f"ff_sub_f({ff_lit(y)}, x)")
    if state["first"]:
        lines.append(f"{name} = ff{{1.0f, 0.0f}};")
    return lines


def emit_f32(table: dict, source: str) -> str:
    fits = {r["n"]: r for r in table["fits"]}
    nmax = max(fits)
    out = [
        f"// Generated by paper_2504_07637_gb300/fit/emit.py from coeffs/{source}; do not edit.",
        "// Per order n: the constrained minimax fit of Q_n for 24-bit work (Sec. 2, Eqs. pqz/pz/qz) in",
        "// root-product form with float coefficients; q0, q1 and c_n as float-float pairs; cut-off z_{n,24}.",
        "#pragma once",
        f"#define BOYS_F32_TABLE_MAX_N {nmax}",
        "",
        "template <int N> struct BoysF32;",
        "",
    ]
    host_z = []
    for n in range(nmax + 1):
        r = fits[n]
        q0 = f_split(r["q0"])
        q1 = f_split(r["q1"])
        # c_n leaves the float range from n = 35 on; the kernels of high
        # orders use C = c_n^(1/(n+1/2)) instead, F_n = (C / D)^(n+1/2)
        c = f_split(r["c"]) if float(r["c"]) < 3.0e38 else ("0.0f", "0.0f")
        cs = f_split(c_root(r["c"], n))
        host_z.append(f(r["z"]))
        body = ["    " + ln for ln in poly_lines("u", r["u"], fma="fmaf", ty="float", lit=f)]
        body += ["    " + ln for ln in poly_lines("v", r["v"], fma="fmaf", ty="float", lit=f)]
        body_ff = ["    " + ln for ln in poly_lines_ff("u", r["u"])]
        body_ff += ["    " + ln for ln in poly_lines_ff("v", r["v"])]
        out += [
            f"// n = {n}: N = {r['N']}, exact-arithmetic error 2^-{r['eps_bits']:.2f}",
            f"template <> struct BoysF32<{n}> {{",
            f"  static constexpr int kOrderN = {r['N']};",
            f"  static constexpr float kCutoff = {f(r['z'])};",
            f"  static constexpr float kQ0hi = {q0[0]}, kQ0lo = {q0[1]};",
            f"  static constexpr float kQ1hi = {q1[0]}, kQ1lo = {q1[1]};",
            f"  static constexpr float kQ2 = {f(r['q2'])};",
            f"  static constexpr float kChi = {c[0]}, kClo = {c[1]};" + ("" if c[0] != "0.0f" else "  // beyond the float range"),
            f"  static constexpr float kCshi = {cs[0]}, kCslo = {cs[1]};  // c_n^(1/(n+1/2))",
            f"  static constexpr float kQ2lo = {f_split(r['q2'])[1]};  // q2 = kQ2 + kQ2lo",
            "  static BOYS_FF_HD void uv(float x, float &u_out, float &v_out) {",
            *body,
            "    u_out = u;",
            "    v_out = v;",
            "  }",
            "  // the same in float-float, coefficients to about 48 bits",
            "  static BOYS_FF_HD void uv_ff(float x, boys::ff &u_out, boys::ff &v_out) {",
            "    using namespace boys;",
            *body_ff,
            "    u_out = u;",
            "    v_out = v;",
            "  }",
            "};",
            "",
        ]
    out += [f"static const float kBoysF32CutoffHost[{nmax + 1}] = {{" + ", ".join(host_z) + "};", ""]
    return "\n".join(out)


def c_root(c: str, n: int) -> str:
    """c^(1/(n+1/2)) as a 40-digit decimal string."""
    import mpmath as mp

    mp.mp.dps = 50
    return mp.nstr(mp.mpf(c) ** (1 / (mp.mpf(n) + mp.mpf(1) / 2)), 40)


def exp2_table_ff(n: int = 32) -> str:
    """2^(j/n) as (hi, lo) float pairs, j = 0..n-1."""
    from decimal import Decimal, getcontext

    getcontext().prec = 60
    vals = []
    for j in range(n):
        hi, lo = f_split(str(Decimal(2) ** (Decimal(j) / Decimal(n))))
        vals.append(f"{hi}, {lo}")
    return ", ".join(vals)


def exp2_table_sig(n: int = 64) -> str:
    """round(2^(j/n) 2^63), j = 0..n-1: 2^(j/n) as a 64-bit significand of
    exponent 0, correctly rounded."""
    from decimal import ROUND_HALF_EVEN, Decimal, getcontext

    getcontext().prec = 80
    vals = []
    for j in range(n):
        v = (Decimal(2) ** (Decimal(j) / Decimal(n))) * (Decimal(2) ** 63)
        vals.append(f"0x{int(v.to_integral_value(rounding=ROUND_HALF_EVEN)):016x}ull")
    return ", ".join(vals)


def exp2_table(n: int = 64) -> str:
    """2^(j/n), j = 0..n-1, correctly rounded to double (table of Tang's
    table-driven exponential)."""
    from decimal import Decimal, getcontext

    getcontext().prec = 60
    vals = []
    for j in range(n):
        v = (Decimal(2) ** (Decimal(j) / Decimal(n)))
        vals.append(repr(float(v)))
    return ", ".join(vals)


F32_SOURCE = "boys_fit_b24_plus1.json"


def render_f64() -> str:
    """csrc/boys_coeffs_f64.inc from the committed 53-bit fits."""
    with open(os.path.join(COEFF_DIR, "boys_fit_b53.json")) as fh:
        return emit_f64(json.load(fh))


def render_f32() -> str | None:
    """csrc/boys_coeffs_f32.inc from the committed float fits (None without them)."""
    f32_path = os.path.join(COEFF_DIR, F32_SOURCE)
    if not os.path.exists(f32_path):
        return None
    with open(f32_path) as fh:
        src = emit_f32(json.load(fh), F32_SOURCE)
    src += "\n// 2^(j/32), j = 0..31, as (hi, lo) float pairs\n"
    src += f"#define BOYS_EXP2_FRAC32_FF {{{exp2_table_ff()}}}\n"
    return src


def main():
    path = os.path.join(CSRC, "boys_coeffs_f64.inc")
    with open(path, "w") as fh:
        fh.write(render_f64())
    print(f"wrote {path}")
    src = render_f32()
    if src is not None:
        path = os.path.join(CSRC, "boys_coeffs_f32.inc")
        with open(path, "w") as fh:
            fh.write(src)
        print(f"wrote {path}")


if __name__ == "__main__":
    main()
