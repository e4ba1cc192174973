"""Constrained uniform-relative minimax fit of the paper's Q_n (offline tool).

The paper's fitted coefficients are distributed as supplementary material that
is not available here, so this module regenerates them from the method of
Sec. 2:

* the closed form (Eq. "fq")  F_n = c_n / (x + Q_n^{s} e^{-x})^{s},  s = n + 1/2;
* the evaluation form (Eq. "pqz")  Q~_n = q0 + q1 x + q2 x^2 u(x)/v(x), with u,
  v monic of degrees N-1 and N given by their roots (Eqs. "pz", "qz");
* the four constraints built in (Eqs. "q0", "q1", "qa", "qb"):
  q0 = Q_n(0) and q1 = Q'_n(0) fix the first two terms, the slope alpha_n
  fixes q2 = alpha_n - q1 (u, v monic), and the intercept beta_n fixes
  sum(roots v) - sum(roots u) = (beta_n - q0)/q2;
* the objective E_n = max_{x>=0} |F~_n/F_n - 1| (Eq. "e").

To first order the relative error of F is  -s^2 (T/D) dQ/Q  with
T = Q^s e^{-x}, D = x + T, so the fit is a weighted rational minimax problem
for r = u/v against g = (Q - q0 - q1 x)/(q2 x^2).  It is solved by a
Lawson-weighted linearised least-squares start followed by Remez exchange
with a Newton solve of the levelled-error equations, all in mpmath.

The target is computed without cancellation from the regularized incomplete
gamma functions:  x^s F_n / c_n = P(s, x) = 1 - R(s, x), hence
T = x (P^{-1/s} - 1) = x expm1(-log(P)/s).
"""
from __future__ import annotations

import json
import math
import sys
import time
from dataclasses import dataclass, field

import mpmath as mp

# ----------------------------------------------------------------------------
# closed-form constants of Sec. 2


def constants(n: int) -> dict:
    """c_n, alpha_n, beta_n, q0, q1, q2 and the root-sum constraint kappa."""
    s = mp.mpf(n) + mp.mpf(1) / 2
    c_n = mp.factorial(2 * n) * mp.sqrt(mp.pi) / (mp.factorial(n) * mp.mpf(2) ** (2 * n + 1))
    c_n1 = mp.factorial(2 * n + 2) * mp.sqrt(mp.pi) / (mp.factorial(n + 1) * mp.mpf(2) ** (2 * n + 3))
    alpha = (2 * c_n1) ** (-mp.mpf(2) / (2 * n + 1))
    beta = mp.mpf(2 * n - 1) / (2 * n + 1) * alpha
    q0 = ((2 * n + 1) * c_n) ** (mp.mpf(4) / (2 * n + 1) ** 2)
    q1 = 2 * q0 / (2 * n + 1) * (mp.mpf(2 * n + 5) / (2 * n + 3) - ((2 * n + 1) * c_n) ** (-mp.mpf(2) / (2 * n + 1)))
    q2 = alpha - q1
    kappa = (beta - q0) / q2  # = (coef of x^{N-2} in u) - (coef of x^{N-1} in v)
    return dict(s=s, c=c_n, alpha=alpha, beta=beta, q0=q0, q1=q1, q2=q2, kappa=kappa)


def cutoff(n: int, bits: int) -> mp.mpf:
    """z_nb of Sec. 2: the root of R(n+1/2, z) = 2^{-b}."""
    s = mp.mpf(n) + mp.mpf(1) / 2
    target = mp.mpf(2) ** (-bits)
    f = lambda z: mp.log(mp.gammainc(s, z, mp.inf, regularized=True)) - mp.log(target)
    lo, hi = mp.mpf(0.5), mp.mpf(10)
    while f(hi) > 0:
        hi *= 2
    return mp.findroot(f, (lo, hi), solver="anderson")


def target(n: int, x: mp.mpf):
    """Exact Q_n(x), T = Q^s e^{-x} and D = x + T at x > 0."""
    s = mp.mpf(n) + mp.mpf(1) / 2
    p = mp.gammainc(s, 0, x, regularized=True)
    if p < mp.mpf(1) / 2:
        logp = mp.log(p)
    else:
        logp = mp.log1p(-mp.gammainc(s, x, mp.inf, regularized=True))
    t = x * mp.expm1(-logp / s)
    q = mp.exp((mp.log(t) + x) / s)
    return q, t, x + t


# ----------------------------------------------------------------------------
# the rational part r = u/v in the scaled variable t = x / X


@dataclass
class Problem:
    n: int
    N: int
    X: mp.mpf
    k: dict
    ts: list = field(default_factory=list)  # grid in t
    G: list = field(default_factory=list)  # X * g(x)
    W: list = field(default_factory=list)  # weight / X


def _poly(coefs_low, lead_deg, t):
    """Evaluate t^lead_deg + sum_k coefs_low[k] t^k (Horner, mp)."""
    acc = mp.mpf(1)
    for c in reversed(coefs_low):
        acc = acc * t + c
    return acc if len(coefs_low) == lead_deg else acc * t ** (lead_deg - len(coefs_low))


def split_theta(N: int, theta, kappa_over_X):
    """theta = [a_0..a_{N-3}, b_0..b_{N-2}, b_{N-1}] -> (a[0..N-2], b[0..N-1])."""
    a = list(theta[: N - 2])
    b = list(theta[N - 2 : 2 * N - 2])
    a.append(b[N - 1] + kappa_over_X)
    return a, b


def sample(prob: Problem, t: mp.mpf):
    """Exact G and W (scaled) at one t."""
    k = prob.k
    x = t * prob.X
    q, T, D = target(prob.n, x)
    g = (q - k["q0"] - k["q1"] * x) / (k["q2"] * x * x)
    w = k["s"] ** 2 * (T / D) * k["q2"] * x * x / q
    return prob.X * g, w / prob.X


def err_at(prob: Problem, theta, t, G, W):
    a, b = split_theta(prob.N, theta, prob.k["kappa"] / prob.X)
    u = _poly(a, prob.N - 1, t)
    v = _poly(b, prob.N, t)
    return W * (u / v - G)


def build_problem(n: int, N: int, X, m: int = 600) -> Problem:
    k = constants(n)
    prob = Problem(n=n, N=N, X=mp.mpf(X), k=k)
    for j in range(m):
        # Chebyshev-like points on (0, 1], skipping the exact zero
        t = (1 - mp.cos(mp.pi * (j + 1) / m)) / 2
        G, W = sample(prob, t)
        prob.ts.append(t)
        prob.G.append(G)
        prob.W.append(W)
    return prob


def lawson(prob: Problem, iters: int = 40, verbose: bool = False):
    """Lawson-weighted, Sanathanan-Koerner-linearised least squares."""
    N = prob.N
    kX = prob.k["kappa"] / prob.X
    m = len(prob.ts)
    lam = [mp.mpf(1) / m] * m
    vprev = [mp.mpf(1)] * m
    theta = None
    best = None
    for it in range(iters):
        rows, rhs = [], []
        for j in range(m):
            t, G, W = prob.ts[j], prob.G[j], prob.W[j]
            sc = mp.sqrt(lam[j]) * W / vprev[j]
            tp = [t**i for i in range(N + 1)]
            row = [sc * tp[i] for i in range(N - 2)]
            row += [-sc * G * tp[i] for i in range(N - 1)]
            row.append(sc * (tp[N - 2] - G * tp[N - 1]))
            rows.append(row)
            rhs.append(-sc * (tp[N - 1] + kX * tp[N - 2] - G * tp[N]))
        A = mp.matrix(rows)
        bvec = mp.matrix(rhs)
        AT = A.T
        theta_m = mp.lu_solve(AT * A, AT * bvec)
        theta = [theta_m[i] for i in range(2 * N - 2)]
        a, b = split_theta(N, theta, kX)
        errs = []
        for j in range(m):
            t = prob.ts[j]
            v = _poly(b, N, t)
            u = _poly(a, N - 1, t)
            vprev[j] = v
            errs.append(prob.W[j] * (u / v - prob.G[j]))
        emax = max(abs(e) for e in errs)
        if best is None or emax < best[0]:
            best = (emax, theta)
        tot = mp.fsum(lam[j] * abs(errs[j]) for j in range(m))
        lam = [lam[j] * abs(errs[j]) / tot for j in range(m)]
        if verbose:
            print(f"  lawson {it:3d}  max|e| = {float(emax):.4e}  (2^{float(mp.log(emax, 2)):.2f})", flush=True)
    return best[1], best[0]


def find_extrema(prob: Problem, theta):
    """Alternating extrema of the error on the grid (t, e) pairs."""
    m = len(prob.ts)
    e = [err_at(prob, theta, prob.ts[j], prob.G[j], prob.W[j]) for j in range(m)]
    ext = []
    for j in range(m):
        left = abs(e[j - 1]) if j > 0 else mp.mpf(0)
        right = abs(e[j + 1]) if j + 1 < m else mp.mpf(0)
        if abs(e[j]) >= left and abs(e[j]) >= right and e[j] != 0:
            ext.append((j, e[j]))
    # merge equal signs, keeping the larger magnitude
    merged = []
    for j, v in ext:
        if merged and mp.sign(merged[-1][1]) == mp.sign(v):
            if abs(v) > abs(merged[-1][1]):
                merged[-1] = (j, v)
        else:
            merged.append((j, v))
    return merged, e


def choose_reference(merged, K):
    ext = list(merged)
    while len(ext) > K:
        i = min(range(len(ext)), key=lambda q: abs(ext[q][1]))
        if i == 0 or i == len(ext) - 1 or len(ext) - K == 1:
            if len(ext) - K == 1 and 0 < i < len(ext) - 1:
                i = 0 if abs(ext[0][1]) < abs(ext[-1][1]) else len(ext) - 1
            ext.pop(i)
        else:
            ext.pop(i)
            # neighbours i-1 and i now share a sign: keep the larger
            if abs(ext[i - 1][1]) >= abs(ext[i][1]):
                ext.pop(i)
            else:
                ext.pop(i - 1)
    return ext


def refine_point(prob: Problem, theta, t_lo, t_hi, sign, iters: int = 30):
    """Golden-section maximisation of sign*e on [t_lo, t_hi] with exact samples."""
    gr = (mp.sqrt(5) - 1) / 2

    def f(t):
        G, W = sample(prob, t)
        return sign * err_at(prob, theta, t, G, W), G, W

    a, b = t_lo, t_hi
    c = b - gr * (b - a)
    d = a + gr * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        if fc[0] > fd[0]:
            b, d, fd = d, c, fc
            c = b - gr * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + gr * (b - a)
            fd = f(d)
    return (c, fc) if fc[0] > fd[0] else (d, fd)


def remez(prob: Problem, theta, iters: int = 20, tol=mp.mpf("1e-4"), verbose: bool = False):
    N = prob.N
    K = 2 * N - 1
    kX = prob.k["kappa"] / prob.X
    history = []
    for outer in range(iters):
        merged, e = find_extrema(prob, theta)
        if len(merged) < K:
            raise RuntimeError(f"only {len(merged)} alternations, need {K}")
        ref = choose_reference(merged, K)
        # refine each reference point to the true extremum
        pts = []
        m = len(prob.ts)
        for j, v in ref:
            lo = prob.ts[j - 1] if j > 0 else prob.ts[0] / 2
            hi = prob.ts[j + 1] if j + 1 < m else prob.ts[j]
            t, (val, G, W) = refine_point(prob, theta, lo, hi, mp.sign(v), iters=25)
            pts.append((t, G, W, mp.sign(v)))
        emax = max(abs(v) for _, v in ref)
        emax = max(emax, max(abs(p[3] * 0 + err_at(prob, theta, p[0], p[1], p[2])) for p in pts))
        emin = min(abs(err_at(prob, theta, p[0], p[1], p[2])) for p in pts)
        history.append(emax)
        if verbose:
            print(f"  remez {outer:2d}  max|e| = 2^{float(mp.log(emax, 2)):.3f}  min/max = {float(emin/emax):.5f}", flush=True)
        prob.ref_t = [p[0] for p in pts]
        if emin / emax > 1 - tol:
            break
        # Newton on the levelled equations E(t_i) = sigma_i h
        h = mp.fsum(p[3] * err_at(prob, theta, p[0], p[1], p[2]) for p in pts) / K
        th = list(theta)
        for _newton in range(12):
            a, b = split_theta(N, th, kX)
            J, F = [], []
            for (t, G, W, sg) in pts:
                tp = [t**i for i in range(N + 1)]
                u = _poly(a, N - 1, t)
                v = _poly(b, N, t)
                E = W * (u / v - G)
                row = [W * tp[i] / v for i in range(N - 2)]
                row += [-W * u * tp[i] / v**2 for i in range(N - 1)]
                row.append(W * (tp[N - 2] / v - u * tp[N - 1] / v**2))
                row.append(-sg)
                J.append(row)
                F.append(-(E - sg * h))
            delta = mp.lu_solve(mp.matrix(J), mp.matrix(F))
            th = [th[i] + delta[i] for i in range(2 * N - 2)]
            h = h + delta[2 * N - 2]
            if max(abs(delta[i]) for i in range(2 * N - 1)) < mp.mpf(10) ** (-(mp.mp.dps - 10)):
                break
        theta = th
    return theta, history


# ----------------------------------------------------------------------------
# root form (Eqs. "pz", "qz") and exact error


def to_roots(prob: Problem, theta):
    """Roots of u and v in the x variable."""
    N = prob.N
    a, b = split_theta(N, theta, prob.k["kappa"] / prob.X)
    # mp.polyroots wants the highest degree first
    ru = mp.polyroots([mp.mpf(1)] + list(reversed(a)), maxsteps=400, extraprec=400) if N > 1 else []
    rv = mp.polyroots([mp.mpf(1)] + list(reversed(b)), maxsteps=400, extraprec=400)
    return [r * prob.X for r in ru], [r * prob.X for r in rv]


def group_roots(roots):
    """Split roots into quadratic factors (x-y)^2+a (pairs, Re>=0), linear
    factors (x-y) (real, >=0) and the gathered negative-real-part polynomial."""
    quad, lin, neg = [], [], []
    used = [False] * len(roots)
    tol = mp.mpf(10) ** (-(mp.mp.dps // 2))
    for i, r in enumerate(roots):
        if used[i]:
            continue
        r = mp.mpc(r)
        if mp.re(r) < 0:
            used[i] = True
            neg.append(r)
            continue
        if abs(mp.im(r)) <= tol * max(1, abs(r)):
            used[i] = True
            lin.append(mp.re(r))
            continue
        # find the conjugate partner
        j = min((q for q in range(len(roots)) if not used[q] and q != i), key=lambda q: abs(mp.mpc(roots[q]) - mp.conj(r)))
        used[i] = used[j] = True
        quad.append((mp.re(r), mp.im(r) ** 2))
    # gathered polynomial with the negative-real-part roots: monic, coefficients low->high
    poly = [mp.mpc(1)]
    for r in neg:
        new = [mp.mpc(0)] * (len(poly) + 1)
        for i, c in enumerate(poly):
            new[i + 1] += c
            new[i] -= r * c
        poly = new
    poly = [mp.re(c) for c in poly]
    return quad, lin, poly


def eval_root_form(fac, x):
    """Evaluate a grouped root-product polynomial at x (mp)."""
    quad, lin, poly = fac
    acc = mp.mpf(0)
    for c in reversed(poly):
        acc = acc * x + c
    for y, a in quad:
        acc *= (x - y) ** 2 + a
    for y in lin:
        acc *= x - y
    return acc


def exact_error(n: int, k: dict, fu, fv, x):
    """F~/F - 1 at x with the grouped root form (Eq. "e")."""
    s = k["s"]
    q, T, D = target(n, x)
    qt = k["q0"] + k["q1"] * x + k["q2"] * x * x * eval_root_form(fu, x) / eval_root_form(fv, x)
    Dt = x + mp.exp(s * mp.log(qt) - x)
    return (D / Dt) ** s - 1


def max_exact_error(n, k, fu, fv, X, pts=4000):
    worst = mp.mpf(0)
    arg = None
    for j in range(1, pts + 1):
        x = X * (1 - mp.cos(mp.pi * j / pts)) / 2
        e = abs(exact_error(n, k, fu, fv, x))
        if e > worst:
            worst, arg = e, x
    return worst, arg


def level_at_reference(prob: Problem, ref_t):
    """Classical rational Remez step: on K = 2N-1 reference points solve
    u(t_i) - (G_i + sigma_i h / W_i) v(t_i) = 0 for the coefficients and the
    level h.  Linear in the coefficients for fixed h, it is the generalised
    eigenproblem (M0 + h M1) y = 0 with y = [theta, 1]; the admissible root
    is the real h of smallest magnitude whose v has no positive real zero."""
    N = prob.N
    kX = prob.k["kappa"] / prob.X
    K = 2 * N - 1
    assert len(ref_t) == K
    M0 = mp.matrix(K, K)
    M1 = mp.matrix(K, K)
    for i, t in enumerate(ref_t):
        G, W = sample(prob, t)
        sg = 1 if i % 2 == 0 else -1
        tp = [t**q for q in range(N + 1)]
        col = 0
        for q in range(N - 2):
            M0[i, col] = tp[q]
            col += 1
        for q in range(N - 1):
            M0[i, col] = -G * tp[q]
            M1[i, col] = -sg * tp[q] / W
            col += 1
        M0[i, col] = tp[N - 2] - G * tp[N - 1]
        M1[i, col] = -sg * tp[N - 1] / W
        col += 1
        M0[i, col] = tp[N - 1] + kX * tp[N - 2] - G * tp[N]
        M1[i, col] = -sg * tp[N] / W
    A = mp.inverse(M0) * M1
    ev, er = mp.eig(A)
    best = None
    for j, mu in enumerate(ev):
        if abs(mp.im(mu)) > abs(mu) * mp.mpf(10) ** (-(mp.mp.dps // 3)) or mu == 0:
            continue
        h = -1 / mp.re(mu)
        y = [mp.re(er[q, j]) for q in range(K)]
        if y[-1] == 0:
            continue
        theta = [y[q] / y[-1] for q in range(K - 1)]
        a, b = split_theta(N, theta, kX)
        rv = mp.polyroots([mp.mpf(1)] + list(reversed(b)), maxsteps=400, extraprec=400)
        if any(abs(mp.im(r)) < 1e-20 and mp.re(r) >= 0 for r in rv):
            continue
        if best is None or abs(h) < abs(best[0]):
            best = (h, theta)
    if best is None:
        raise RuntimeError("no admissible level on this reference")
    return best[1]


def theta_from_roots(prob: Problem, roots_u, roots_v):
    """Warm start: monic coefficients (in t = x/X) from roots in x, then the
    intercept constraint imposed on the x^{N-2} coefficient of u."""
    N = prob.N

    def coefs(roots):
        poly = [mp.mpc(1)]
        for r in roots:
            r = mp.mpc(r) / prob.X
            new = [mp.mpc(0)] * (len(poly) + 1)
            for i, c in enumerate(poly):
                new[i + 1] += c
                new[i] -= r * c
            poly = new
        return [mp.re(c) for c in poly[:-1]]

    a = coefs(roots_u)
    b = coefs(roots_v)
    return a[: N - 2] + b


def expand_roots(fac):
    """Grouped factors -> list of complex roots."""
    quad, lin, poly = fac
    roots = []
    for y, a in quad:
        roots += [mp.mpc(y, mp.sqrt(a)), mp.mpc(y, -mp.sqrt(a))]
    roots += [mp.mpc(y) for y in lin]
    if len(poly) > 1:
        roots += list(mp.polyroots(list(reversed(poly)), maxsteps=400, extraprec=400))
    return roots


def fit(n: int, N: int, bits: int, dps: int = 50, grid: int = 600, verbose: bool = False, lawson_iters: int = 40,
        warm=None):
    """Fit Q~_n of order N for b-bit work.  `warm` = (roots_u, roots_v) of a
    neighbouring order's solution starts the Remez exchange directly."""
    mp.mp.dps = dps
    t0 = time.time()
    z = cutoff(n, bits)
    X = z * mp.mpf("1.05") + 2
    prob = build_problem(n, N, X, m=grid)
    if warm is not None:
        # warm = reference points (x values) of a neighbouring order, rescaled
        ref_t = [mp.mpf(xr) / X for xr in warm]
        theta = level_at_reference(prob, ref_t)
    else:
        theta, e0 = lawson(prob, iters=lawson_iters, verbose=verbose)
    theta, hist = remez(prob, theta, verbose=verbose)
    ru, rv = to_roots(prob, theta)
    for r in rv:
        r = mp.mpc(r)
        if abs(mp.im(r)) < mp.mpf(10) ** (-(dps // 2)) and mp.re(r) >= 0:
            raise RuntimeError(f"pole on the positive axis at {r}")
    fu, fv = group_roots(ru), group_roots(rv)
    E, xE = max_exact_error(n, prob.k, fu, fv, X * 2, pts=3000)
    if verbose:
        print(f"n={n} N={N} b={bits}: -log2 E = {float(-mp.log(E, 2)):.3f} at x={float(xE):.3f} ({time.time()-t0:.1f}s)")
    ref_x = [t * X for t in getattr(prob, "ref_t", [])]
    return dict(n=n, N=N, bits=bits, z=z, X=X, k=prob.k, theta=theta, fu=fu, fv=fv, E=E, hist=hist, ref_x=ref_x)


if __name__ == "__main__":
    n, N, bits = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3])
    fit(n, N, bits, verbose=True)
