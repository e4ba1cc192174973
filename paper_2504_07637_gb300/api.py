"""PyTorch-facing wrappers: torch supplies device memory and the stream;
every step of the evaluation runs in libboys.so's kernels."""
from __future__ import annotations

import torch

from . import _capi


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _check_input(x: torch.Tensor, dtypes) -> torch.Tensor:
    if not isinstance(x, torch.Tensor):
        raise TypeError("x must be a torch.Tensor")
    if not x.is_cuda:
        raise TypeError("x must be a CUDA tensor: the library has no CPU path")
    if x.dtype not in dtypes:
        raise TypeError(f"x must have dtype in {dtypes}, got {x.dtype}")
    return x.reshape(-1).contiguous()


def max_n(precision_bits: int = 53) -> int:
    return _capi.load().boys_max_n(precision_bits)


def cutoff(n: int, precision_bits: int = 53) -> float:
    """z_{n,b} used by the library (Sec. 2 cut-off)."""
    return _capi.load().boys_cutoff(n, precision_bits)


def top_order_f64(n_max: int) -> int:
    return _capi.load().boys_top_order_f64(n_max)


def top_order_f32(n_max: int) -> int:
    return _capi.load().boys_top_order_f32(n_max)


def boys(x: torch.Tensor, n_max: int, out: torch.Tensor | None = None) -> torch.Tensor:
    """F_0..F_{n_max} at every element of x: a [x.numel(), n_max+1] tensor of
    x's dtype (float64: 2e-14 max relative error; float32: 2e-6)."""
    xf = _check_input(x, (torch.float64, torch.float32))
    n = xf.numel()
    if out is None:
        out = torch.empty((n, n_max + 1), dtype=xf.dtype, device=xf.device)
    elif out.shape != (n, n_max + 1) or out.dtype != xf.dtype or not out.is_contiguous() or out.device != xf.device:
        raise ValueError("out must be a contiguous [count, n_max+1] tensor of x's dtype on x's device")
    fn = "boys_eval_f64" if xf.dtype == torch.float64 else "boys_eval_f32"
    with torch.cuda.device(xf.device):
        _capi.call(fn, xf.data_ptr(), n, int(n_max), out.data_ptr(), _stream_ptr(xf.device))
    return out


def boys_from_host(x: torch.Tensor, n_max: int, out: torch.Tensor | None = None,
                   workspace_bytes: int = 1 << 28, device: torch.device | int | None = None) -> torch.Tensor:
    """F_0..F_{n_max} for a CPU float64 tensor, streamed through the GPU.

    x and out live in host memory (pin them for overlapped copies); the
    device workspace is allocated by torch for the duration of the call.
    Returns out ([x.numel(), n_max+1], host) after the work has finished."""
    if not isinstance(x, torch.Tensor) or x.is_cuda or x.dtype != torch.float64:
        raise TypeError("x must be a CPU float64 tensor")
    xf = x.reshape(-1).contiguous()
    n = xf.numel()
    if out is None:
        out = torch.empty((n, n_max + 1), dtype=torch.float64, pin_memory=torch.cuda.is_available())
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
    ws = torch.empty(int(workspace_bytes), dtype=torch.uint8, device=dev)
    with torch.cuda.device(dev):
        s = torch.cuda.current_stream(dev)
        _capi.call("boys_eval_f64_host", xf.data_ptr(), n, int(n_max), out.data_ptr(), ws.data_ptr(),
                   int(workspace_bytes), s.cuda_stream)
        s.synchronize()
    return out
