"""Seeded synthetic argument generators shaped like the paper's use case.

The Boys functions are evaluated inside one- and two-electron integral codes
over Gaussian basis functions (Sec. 1), where the argument is x = p R^2 for a
Gaussian exponent p and a distance R.  These generators hold none of the
method's arithmetic; they only draw arguments, and are shared by the tests,
the smoke check and the benchmark.  Seeds are fixed per workload.

Workloads:
  plain     65,536 arguments: 95% log-uniform on [1e-6, 300], the rest half
            exact zeros and half within +-1e-3 relative of the cut-offs z_{m,b},
            m = 0..8 round robin (b = 53, or 24 for the float path); shuffled.
  scale     x = p R^2, p log-uniform on [0.05, 1e4], R uniform on [0, 12].
  ragged    request counts log-uniform on [64, 65,536], n_max uniform on
            {0..16}, arguments drawn as in `plain`.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2504_07637


def cutoff_points(bits: int, orders=range(9)) -> np.ndarray:
    """z_{m,b}: where R(m+1/2, z) = 2^-b, from scipy's inverse incomplete gamma."""
    from scipy.special import gammainccinv

    return np.array([gammainccinv(m + 0.5, 2.0**-bits) for m in orders])


def plain(count: int = 65536, bits: int = 53, seed: int = SEED_BASE + 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n_main = int(round(0.95 * count))
    rest = count - n_main
    n_zero = rest // 2
    n_cut = rest - n_zero
    main = np.exp(rng.uniform(math.log(1e-6), math.log(300.0), n_main))
    zs = cutoff_points(bits)
    near = zs[np.arange(n_cut) % zs.size] * np.exp(rng.uniform(math.log(1 - 1e-3), math.log(1 + 1e-3), n_cut))
    x = np.concatenate([main, np.zeros(n_zero), near])
    rng.shuffle(x)
    return x


def scale(count: int = 1 << 26, seed: int = SEED_BASE + 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    p = np.exp(rng.uniform(math.log(0.05), math.log(1e4), count))
    r = rng.uniform(0.0, 12.0, count)
    return p * r * r


def ragged(num_requests: int = 4096, max_n: int = 16, seed: int = SEED_BASE + 3):
    """(x, offsets[R+1], n_max[R]) with x concatenated over requests."""
    rng = np.random.default_rng(seed)
    counts = np.floor(np.exp(rng.uniform(math.log(64), math.log(65536), num_requests))).astype(np.int64)
    n_max = rng.integers(0, max_n + 1, num_requests).astype(np.int32)
    offsets = np.zeros(num_requests + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    total = int(offsets[-1])
    x = plain(total, 53, seed=seed + 1000) if total > 0 else np.zeros(0)
    return x, offsets, n_max


def gradient_weights(n_max: int = 8, seed: int = SEED_BASE + 4) -> np.ndarray:
    """w_m ~ N(0, 1) for the loss sum_m w_m sum_i F_m(x_i)."""
    return np.random.default_rng(seed).standard_normal(n_max + 1)
