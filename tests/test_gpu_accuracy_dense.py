"""Table I's measurement, repeated on the GPU path.

Sec. 3 measures the finite-precision accuracy of each order n on 2^20
equally spaced points 0 <= x < z_nb: F_n by the approximation, F_m (m < n) by
the downward recursion, and the maximum relative error of each column,
reported as bits (-log2) for m = 0, n-1 and n (the eps_bar columns of
Table I).  Here the same grid goes through the library (n_max = n; the
library evaluates the closed form at n_top >= n and recurses, Trick A) and
the errors are measured against the oracle.  Each column must be within 1
bit of the paper's figure or better; the bits are recorded as test
properties (JUnit)."""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GRID = 1 << 20


def _table1():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_accuracy_bits.txt")
    rows = {}
    for line in open(path):
        f = line.split()
        if f and not line.startswith("#"):
            rows[int(f[0])] = f
    return rows


TABLE1 = _table1()


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07637_gb300.build import build_library

    build_library()
    import paper_2504_07637_gb300 as boys

    return boys


def _bits(rel_col):
    return -math.log2(max(float(rel_col.max()), 2.0**-64))


def _paper(n, f32):
    # columns: n, N, eps0_bar, eps_{n-1}_bar, eps_n_bar, eps_n (double), then the same for single
    f = TABLE1[n][6:] if f32 else TABLE1[n][1:6]
    e0, enm1, en = f[1], f[2], f[3]
    return float(e0), (None if enm1 == "-" else float(enm1)), float(en)


def _measure(lib, oracle_mod, n, f32, record_property):
    import torch

    bits = 24 if f32 else 53
    z = lib.cutoff(n, bits)
    x = np.arange(GRID, dtype=np.float64) * (z / GRID)  # 0 <= x < z, equally spaced
    if f32:
        x = x.astype(np.float32)
    got = lib.boys(torch.from_numpy(x).cuda(), n).cpu().numpy().astype(np.float64)
    ref = oracle_mod.boys_threaded(x.astype(np.float64), n, os.cpu_count() or 1)
    rel = np.abs(got - ref) / np.abs(ref)  # every F_m(x) > 0 on [0, z)
    ours = (_bits(rel[:, 0]), _bits(rel[:, n - 1]) if n >= 1 else None, _bits(rel[:, n]))
    record_property("bits_eps0_epsnm1_epsn", [round(b, 2) if b is not None else None for b in ours])
    return ours, rel


@pytest.mark.parametrize("n", list(range(0, 37)))
def test_double_columns_of_table1(lib, oracle_mod, n, record_property):
    ours, rel = _measure(lib, oracle_mod, n, False, record_property)
    assert rel.max() <= 2e-14
    for got_bits, paper_bits in zip(ours, _paper(n, False)):
        if paper_bits is not None and got_bits is not None:
            assert got_bits >= paper_bits - 1.0, (n, ours, _paper(n, False))


@pytest.mark.parametrize("n", list(range(0, 37)))
def test_single_columns_of_table1(lib, oracle_mod, n, record_property):
    ours, rel = _measure(lib, oracle_mod, n, True, record_property)
    assert rel.max() <= 2e-6
    for got_bits, paper_bits in zip(ours, _paper(n, True)):
        if paper_bits is not None and got_bits is not None:
            assert got_bits >= paper_bits - 1.0, (n, ours, _paper(n, True))


def test_f0_at_n36_meets_the_papers_17_bits_in_single(lib, oracle_mod, record_property):
    # Sec. 3 reports F_0 to no worse than 17 bits in single precision even for
    # n = 36; the float path (float-float on the amplified steps) is held to
    # the 2e-6 bound (18.9 bits) on Table I's grid
    ours, rel = _measure(lib, oracle_mod, 36, True, record_property)
    assert ours[0] >= 17.0 and ours[0] >= -math.log2(2e-6), ours
