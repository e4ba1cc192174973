"""Fused consumer: out = sum_m c_m F_m(x) computed inside the evaluation
kernel, against the oracle's rows contracted in long double.

Error measure: |out - ref| / sum_m |c_m| F_m(x) (signed coefficients cancel),
bounded by 2e-14 (FP64) and 2e-6 (FP32, where the terms are normal floats)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07637_gb300.build import build_library

    build_library()
    import paper_2504_07637_gb300 as boys

    return boys


def _ref(oracle_mod, x64, c, n_max):
    F = oracle_mod.boys_ld(x64, n_max)
    cl = np.broadcast_to(np.asarray(c, dtype=np.longdouble), F.shape)
    return (cl * F).sum(axis=1).astype(np.float64), (np.abs(cl) * F).sum(axis=1).astype(np.float64)


@pytest.mark.parametrize("n_max", [0, 5, 8, 16, 36])
@pytest.mark.parametrize("dense", [False, True])
def test_f64_against_oracle(lib, oracle_mod, n_max, dense):
    import torch

    rng = np.random.default_rng(n_max)
    x = np.concatenate([np.exp(rng.uniform(math.log(1e-7), math.log(1e4), 7000)), [0.0, 1e-300, 1e8]])
    c = rng.standard_normal((x.size, n_max + 1) if dense else n_max + 1)
    got = lib.boys_contract(torch.from_numpy(x).cuda(), n_max, torch.from_numpy(c).cuda()).cpu().numpy()
    want, scale = _ref(oracle_mod, x, c, n_max)
    assert (np.abs(got - want) / scale).max() <= 2e-14


@pytest.mark.parametrize("n_max", [0, 8, 16])
def test_f32_against_oracle(lib, oracle_mod, n_max):
    import torch

    rng = np.random.default_rng(50 + n_max)
    xf = np.exp(rng.uniform(math.log(1e-6), math.log(80.0), 9001)).astype(np.float32)  # normal-range values
    c = rng.standard_normal(n_max + 1).astype(np.float32)
    got = lib.boys_contract(torch.from_numpy(xf).cuda(), n_max, torch.from_numpy(c).cuda()).cpu().numpy()
    want, scale = _ref(oracle_mod, xf.astype(np.float64), c.astype(np.float64), n_max)
    assert (np.abs(got - want) / scale).max() <= 2e-6


def test_matches_rows_then_dot(lib):
    # the fused result equals contracting the stored rows, up to rounding:
    # with the same weights for every argument the asymptote's contribution
    # is a Horner polynomial, about (n_max + 3)/2 ulp of sum_m |w_m| F_m
    import torch

    from paper_2504_07637_gb300 import workloads

    x = torch.from_numpy(workloads.scale(1 << 20, seed=5)).cuda()
    c = torch.randn(9, dtype=torch.float64, device="cuda")
    fused = lib.boys_contract(x, 8, c)
    rows = lib.boys(x, 8)
    ref = rows @ c
    scale = rows @ c.abs()
    assert ((fused - ref).abs() / scale).max().item() <= 4e-15


@pytest.mark.parametrize("n_max", [12, 16, 23, 36])
@pytest.mark.parametrize("count", [5000, (1 << 20) + 3001])
def test_one_hot_contraction_equals_rows_bitwise(lib, n_max, count):
    # The contraction keeps each row in registers, the row store at n_max >= 12
    # stages it through shared memory: with c = e_m the contraction adds exact
    # zeros to F_m, so both paths must give the same bits (small and large
    # launch shapes, both lists of a tile, ragged tails) wherever they share
    # the recursion's arithmetic.  The staged rows always recurse on integer
    # significands; the contraction does so for up to 18 steps and in FP64
    # beyond (n_max >= 17), where the two agree to the FP64 recursion's
    # rounding (below 2.2e-15 relative over 40 steps).
    import torch

    from paper_2504_07637_gb300 import roofline, workloads

    x = torch.from_numpy(np.concatenate([workloads.scale(count - 3, seed=n_max), [0.0, 1e-300, 1e8]])).cuda()
    rows = lib.boys(x, n_max)
    for m in (0, n_max // 2, n_max):
        # coefficients given per argument ([count, n_max+1]): the contraction
        # then builds every row (uniform ones would take the asymptote's
        # contraction as a polynomial)
        c = torch.zeros((count, n_max + 1), dtype=torch.float64, device="cuda")
        c[:, m] = 1.0
        got = lib.boys_contract(x, n_max, c)
        if roofline.int_recursion(lib.top_order_f64(n_max)):
            assert torch.equal(got, rows[:, m]), m
        else:
            ref = rows[:, m]
            assert ((got - ref).abs() <= 4e-15 * ref.abs()).all().item(), m


@pytest.mark.parametrize("n_max", [0, 8, 13, 16])
def test_domain_convention_uniform_weights(lib, n_max):
    # the asymptote's contraction as a polynomial must follow the rows'
    # domain convention: negative or NaN x -> NaN, +inf -> 0
    import torch

    bad = np.tile([-1.0, -1e-300, np.nan, -np.inf, np.inf], 30)
    x = np.concatenate([bad, np.exp(np.random.default_rng(n_max).uniform(-5, 8, 200))])
    w = torch.linspace(-1.0, 2.0, n_max + 1, dtype=torch.float64, device="cuda")
    got = lib.boys_contract(torch.from_numpy(x).cuda(), n_max, w).cpu().numpy()
    nan_in = np.isnan(x) | (x < 0)
    assert np.all(np.isnan(got[nan_in]))
    assert np.all(got[x == np.inf] == 0.0)
    assert np.all(np.isfinite(got[~nan_in & np.isfinite(x)]))
