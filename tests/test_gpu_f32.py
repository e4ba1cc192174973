"""FP32 forward parity: the float CUDA path (through the C ABI) against the
oracle evaluated at the same (float) arguments.

Tolerance: max relative error 2e-6 for every m where the exact value is a
normal float (>= FLT_MIN); below that, |out - exact| <= 2e-6 |exact| + one
subnormal unit (2^-149): a float cannot carry more there.
"""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 2e-6
FLT_MIN = float(np.finfo(np.float32).tiny)
SUB = 2.0**-149


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07637_gb300.build import build_library

    build_library()
    import paper_2504_07637_gb300 as boys

    return boys


def _gpu(lib, x, n_max):
    import torch

    xf = np.ascontiguousarray(x, dtype=np.float32)
    return lib.boys(torch.from_numpy(xf).cuda(), n_max).cpu().numpy(), xf


def _check(got, ref):
    """Return the max relative error over normal-range references after
    asserting the exact/subnormal cases."""
    got = got.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    zero = ref == 0
    assert np.all(got[zero] == 0)
    small = ~nan & ~zero & (np.abs(ref) < FLT_MIN)
    assert np.all(np.abs(got[small] - ref[small]) <= TOL * np.abs(ref[small]) + SUB)
    norm = ~nan & ~zero & ~small
    rel = np.zeros_like(ref)
    rel[norm] = np.abs(got[norm] - ref[norm]) / np.abs(ref[norm])
    return rel


def _per_m(rel):
    # max relative error of each column F_m (normal-range values), as recorded in the test report
    return [float(f"{v:.3g}") for v in rel.max(axis=0)]


def _table1_eps_bar_n(n):
    """Table I's finite-precision accuracy of F_n (single column eps_n_bar, in
    bits): the paper's own rounding level after its recursion."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_accuracy_bits.txt")
    for line in open(path):
        f = line.split()
        if f and not line.startswith("#") and int(f[0]) == n:
            return float(f[9])
    raise KeyError(n)


def test_plain_workload_n8(lib, oracle_mod, record_property):
    from paper_2504_07637_gb300 import workloads

    got, xf = _gpu(lib, workloads.plain(65536, 24), 8)
    rel = _check(got, oracle_mod.boys(xf.astype(np.float64), 8))
    per_m = rel.max(axis=0)
    record_property("max_rel_err_per_m", _per_m(rel))
    assert per_m.max() <= TOL, per_m


@pytest.mark.parametrize("n_max", list(range(0, 37)))
def test_every_order(lib, oracle_mod, n_max, record_property):
    rng = np.random.default_rng(300 + n_max)
    z = lib.cutoff(lib.top_order_f32(n_max), 24)
    x = np.concatenate(
        [
            np.exp(rng.uniform(math.log(1e-8), math.log(2 * z), 3000)),
            rng.uniform(0, 1.2 * z, 1000),
            np.exp(rng.uniform(math.log(2 * z), math.log(1e30), 97)),
        ]
    )
    got, xf = _gpu(lib, x, n_max)
    rel = _check(got, oracle_mod.boys(xf.astype(np.float64), n_max))
    record_property("max_rel_err_per_m", _per_m(rel))
    assert rel.max() <= TOL
    # at least as accurate as the paper's own evaluation (Table I, eps_n_bar),
    # within 1 bit for the different sample points and rounding
    assert -math.log2(max(rel.max(), 2.0**-60)) >= _table1_eps_bar_n(n_max) - 1.0


def test_special_arguments(lib, oracle_mod):
    zs = [np.float32(lib.cutoff(n, 24)) for n in range(0, 38)]
    near = [np.nextafter(z, np.float32(0)) for z in zs] + zs + [np.nextafter(z, np.float32(np.inf)) for z in zs]
    x = np.array([0.0, -0.0, 1e-45, 1e-40, 1.1754944e-38, 1e-30, 1e-7, 1.0, 1e6, 1e20, 3.4e38] + near,
                 dtype=np.float32)
    for n_max in (0, 8, 16, 17, 24, 36):
        got, xf = _gpu(lib, x, n_max)
        rel = _check(got, oracle_mod.boys(xf.astype(np.float64), n_max))
        assert rel.max() <= TOL, (n_max, xf[np.argmax(rel.max(axis=1))])
    for n_max in (8, 16, 17, 36):  # every tile shape, and the compensated chain
        bad, _ = _gpu(lib, np.array([-1.0, -1e-30, np.nan, -np.inf, np.inf], dtype=np.float32), n_max)
        assert np.all(np.isnan(bad[:4])) and np.all(bad[4] == 0.0)


@pytest.mark.parametrize("count", [1, 2, 3, 31, 33, 255, 2047, 2048, 2049, 65537])
def test_tail_sizes(lib, oracle_mod, count):
    x = np.exp(np.random.default_rng(count).uniform(-10, 6, count))
    got, xf = _gpu(lib, x, 8)
    assert _check(got, oracle_mod.boys(xf.astype(np.float64), 8)).max() <= TOL


def test_misaligned_views_and_canaries(lib, oracle_mod):
    import torch

    from paper_2504_07637_gb300 import _capi

    n_max, count, pad = 8, 3001, 64
    xh = np.exp(np.random.default_rng(9).uniform(-12, 7, count)).astype(np.float32)
    xbuf = torch.zeros(count + 1, dtype=torch.float32, device="cuda")
    xbuf[1:] = torch.from_numpy(xh).cuda()
    sentinel = -12345.0
    obuf = torch.full((pad + count * (n_max + 1) + 1 + pad,), sentinel, dtype=torch.float32, device="cuda")
    _capi.call("boys_eval_f32", xbuf.data_ptr() + 4, count, n_max, obuf.data_ptr() + (pad + 1) * 4,
               torch.cuda.current_stream().cuda_stream)
    host = obuf.cpu().numpy()
    assert np.all(host[: pad + 1] == sentinel) and np.all(host[pad + 1 + count * (n_max + 1):] == sentinel)
    got = host[pad + 1: pad + 1 + count * (n_max + 1)].reshape(count, n_max + 1)
    assert _check(got, oracle_mod.boys(xh.astype(np.float64), n_max)).max() <= TOL


def test_full_size_scale_workload_sampled(lib, oracle_mod, record_property):
    # 2^26 float arguments, n_max = 8, in the benchmark's launch configuration
    import torch

    from paper_2504_07637_gb300 import workloads

    xf = workloads.scale(1 << 26).astype(np.float32)
    out = lib.boys(torch.from_numpy(xf).cuda(), 8)
    idx = np.sort(np.random.default_rng(8).choice(xf.size, 1 << 20, replace=False))  # a 2^20 sample
    idx = np.concatenate([idx, [0, xf.size - 1]])
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    rel = _check(got, oracle_mod.boys_threaded(xf[idx].astype(np.float64), 8, os.cpu_count() or 1))
    record_property("max_rel_err_per_m", _per_m(rel))
    assert rel.max() <= TOL
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n_max", [24, 36])
def test_full_size_high_order_sampled(lib, oracle_mod, n_max, record_property):
    # 2^24 float arguments of the scale workload at the high orders (float-float
    # rational part, paired recursion constants, compensated asymptote chain)
    import torch

    from paper_2504_07637_gb300 import workloads

    xf = workloads.scale(1 << 24, seed=36).astype(np.float32)
    out = lib.boys(torch.from_numpy(xf).cuda(), n_max)
    idx = np.sort(np.random.default_rng(n_max).choice(xf.size, 1 << 18, replace=False))
    idx = np.concatenate([idx, [0, xf.size - 1]])
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    rel = _check(got, oracle_mod.boys_threaded(xf[idx].astype(np.float64), n_max, os.cpu_count() or 1))
    record_property("max_rel_err_per_m", _per_m(rel))
    assert rel.max() <= TOL
    del out
    torch.cuda.empty_cache()


def test_contraction_order_limit(lib):
    # the fused float contraction stays at n_max <= 16 (plain FP32 Horner sums)
    import torch

    from paper_2504_07637_gb300 import _capi

    x = torch.ones(4, dtype=torch.float32, device="cuda")
    c = torch.ones(18, dtype=torch.float32, device="cuda")
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    rc = _capi.load().boys_eval_contract_f32(x.data_ptr(), 4, 17, c.data_ptr(), 0, 1, out.data_ptr(), None)
    assert rc == 3  # BOYS_ERR_NMAX


def test_host_pipeline_matches_device_path(lib):
    import torch

    from paper_2504_07637_gb300 import _capi, workloads

    n_max, count = 8, 70_000
    x = workloads.scale(count, seed=78).astype(np.float32)
    dev = lib.boys(torch.from_numpy(x).cuda(), n_max).cpu().numpy()
    xh = torch.from_numpy(x).pin_memory()
    out = torch.full((count, n_max + 1), -1.0, dtype=torch.float32).pin_memory()
    ws_bytes = _capi.load().boys_eval_f32_host_workspace(n_max, 8192)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    _capi.call("boys_eval_f32_host", xh.data_ptr(), count, n_max, out.data_ptr(), ws.data_ptr(), ws_bytes, s.cuda_stream)
    s.synchronize()
    assert np.array_equal(out.numpy(), dev)
