"""Backward (adjoint) parity: grad_x = -sum_m g_m F_{m+1} against the oracle
gradient and against central finite differences of the GPU forward.

Error measure: |grad_gpu - grad_ref| / sum_m |g_m| F_{m+1}(x), so signed
weights that cancel do not inflate it.  Bound 1e-12 against the oracle; the
finite-difference check (h = 1e-6 max(1, x), rounding noise ~1e-10) is a
sanity bound of 1e-7.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07637_gb300.build import build_library

    build_library()
    import paper_2504_07637_gb300 as boys

    return boys


def _x(n, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([np.exp(rng.uniform(math.log(1e-6), math.log(300.0), n - 4)), [0.0, 1e-300, 57.7, 1e6]])


def _ref(oracle_mod, x, g, n_max):
    grad, scale = oracle_mod.grad_ld(x, g, n_max)
    return grad.astype(np.float64), scale.astype(np.float64)


@pytest.mark.parametrize("n_max", [0, 1, 8, 9, 20, 35])
@pytest.mark.parametrize("mode", ["saved", "recompute"])
def test_against_oracle(lib, oracle_mod, n_max, mode):
    import torch

    x = _x(5000, n_max)
    g = np.random.default_rng(n_max + 7).standard_normal((x.size, n_max + 1))
    xd, gd = torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()
    F = lib.boys(xd, n_max + 1) if mode == "saved" else None
    got = lib.boys_backward(xd, gd, n_max, F).cpu().numpy()
    want, scale = _ref(oracle_mod, x, g, n_max)
    err = np.abs(got - want) / np.where(scale > 0, scale, 1.0)
    assert err.max() <= TOL, err.max()


def test_recompute_equals_saved_bitwise(lib):
    # per-argument weights: the recompute path builds every row, so both
    # paths sum the same products in the same order
    import torch

    x = torch.from_numpy(_x(20000, 3)).cuda()
    w = torch.randn(9, dtype=torch.float64, device="cuda")
    g = w.expand(x.numel(), 9).contiguous()
    a = lib.boys_backward(x, g, 8, lib.boys(x, 9))
    b = lib.boys_backward(x, g, 8, None)
    assert torch.equal(a, b)


@pytest.mark.parametrize("n_max", [0, 1, 8, 16, 20])
def test_recompute_with_broadcast_weights(lib, oracle_mod, n_max):
    # one weight vector for all arguments (row stride 0): above the cut-off the
    # recompute path takes the gradient of the asymptote as a polynomial in
    # 1/x (up to n_max = 16); against the oracle, and against the saved rows
    # within a few ulp of the weighted magnitude
    import torch

    x = _x(6000, 40 + n_max)
    w = np.random.default_rng(n_max).standard_normal(n_max + 1)
    xd = torch.from_numpy(x).cuda()
    g = torch.from_numpy(w).cuda().expand(x.size, n_max + 1)
    got = lib.boys_backward(xd, g, n_max, None).cpu().numpy()
    want, scale = _ref(oracle_mod, x, np.broadcast_to(w, (x.size, n_max + 1)).copy(), n_max)
    err = np.abs(got - want) / np.where(scale > 0, scale, 1.0)
    assert err.max() <= TOL, err.max()
    saved = lib.boys_backward(xd, g, n_max, lib.boys(xd, n_max + 1)).cpu().numpy()
    assert (np.abs(got - saved) / np.where(scale > 0, scale, 1.0)).max() <= 4e-15
    # domain convention through the polynomial: negative or NaN x -> NaN, +inf -> 0
    bad = torch.tensor([-1.0, float("nan"), float("inf")] * 40, dtype=torch.float64, device="cuda")
    gb = torch.from_numpy(w).cuda().expand(bad.numel(), n_max + 1)
    out = lib.boys_backward(bad, gb, n_max, None).cpu().numpy().reshape(40, 3)
    assert np.all(np.isnan(out[:, :2])) and np.all(out[:, 2] == 0.0)


def test_autograd_function_matches_oracle(lib, oracle_mod):
    import torch

    from paper_2504_07637_gb300 import workloads

    x_host = workloads.plain(1 << 14, 53)
    w = workloads.gradient_weights(8)
    x = torch.from_numpy(x_host).cuda().requires_grad_(True)
    F = lib.boys_autograd(x, 8)
    assert F.shape == (x.numel(), 9)
    loss = (F * torch.from_numpy(w).cuda()).sum()
    loss.backward()
    want, scale = _ref(oracle_mod, x_host, np.broadcast_to(w, (x_host.size, 9)), 8)
    err = np.abs(x.grad.cpu().numpy() - want) / scale
    assert err.max() <= TOL


def test_autograd_broadcast_gradient(lib, oracle_mod):
    # a weight vector expanded over the rows reaches the kernel with row stride 0
    import torch

    x_host = _x(10000, 5)
    w = np.random.default_rng(1).standard_normal(9)
    x = torch.from_numpy(x_host).cuda().requires_grad_(True)
    F = lib.boys_autograd(x, 8)
    torch.autograd.backward(F, torch.from_numpy(w).cuda().expand(x.numel(), 9))
    want, scale = _ref(oracle_mod, x_host, np.broadcast_to(w, (x_host.size, 9)), 8)
    assert (np.abs(x.grad.cpu().numpy() - want) / scale).max() <= TOL


def test_central_finite_differences(lib):
    # d/dx sum_m w_m F_m(x) by central differences of the GPU forward
    import torch

    x_host = np.exp(np.random.default_rng(2).uniform(math.log(0.01), math.log(200.0), 4000))
    w = np.random.default_rng(3).standard_normal(9)
    h = 1e-6 * np.maximum(1.0, x_host)
    wd = torch.from_numpy(w).cuda()
    f = lambda v: (lib.boys(torch.from_numpy(v).cuda(), 8) * wd).sum(dim=1).cpu().numpy()
    fd = (f(x_host + h) - f(x_host - h)) / (2 * h)
    x = torch.from_numpy(x_host).cuda().requires_grad_(True)
    (lib.boys_autograd(x, 8) * wd).sum().backward()
    Fn = lib.boys(torch.from_numpy(x_host).cuda(), 9).cpu().numpy()
    scale = (np.abs(w) * Fn[:, 1:]).sum(axis=1)
    assert (np.abs(fd - x.grad.cpu().numpy()) / scale).max() <= 1e-7


def test_torch_gradcheck(lib):
    import torch

    # central differences need x - eps >= 0 (negative arguments are outside the domain)
    x = torch.tensor([1e-3, 0.7, 3.0, 25.0, 60.0, 400.0], dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda v: lib.boys_autograd(v, 5), (x,), eps=1e-7, atol=1e-8, rtol=1e-5)


def test_full_size_differentiation_workload(lib, oracle_mod):
    # 2^24 arguments, forward to n_max = 9, loss sum_{m<=8} w_m sum_i F_m(x_i)
    import torch

    from paper_2504_07637_gb300 import workloads

    x_host = workloads.plain(1 << 24, 53)
    w = workloads.gradient_weights(8)
    x = torch.from_numpy(x_host).cuda().requires_grad_(True)
    F = lib.boys_autograd(x, 8)
    torch.autograd.backward(F, torch.from_numpy(w).cuda().expand(x.numel(), 9))
    idx = np.sort(np.random.default_rng(4).choice(x_host.size, 1 << 15, replace=False))
    got = x.grad[torch.from_numpy(idx).cuda()].cpu().numpy()
    want, scale = _ref(oracle_mod, x_host[idx], np.broadcast_to(w, (idx.size, 9)), 8)
    assert (np.abs(got - want) / np.where(scale > 0, scale, 1.0)).max() <= TOL
