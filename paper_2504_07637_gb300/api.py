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


def boys(x: torch.Tensor, n_max: int, out: torch.Tensor | None = None, two_point: bool = False) -> torch.Tensor:
    """F_0..F_{n_max} at every element of x: a [x.numel(), n_max+1] tensor of
    x's dtype (float64: 2e-14 max relative error; float32: 2e-6).
    two_point (float64): also evaluate the closed form at n_max/2 for more
    accurate low orders (Trick B of Sec. 3)."""
    xf = _check_input(x, (torch.float64, torch.float32))
    n = xf.numel()
    if out is None:
        out = torch.empty((n, n_max + 1), dtype=xf.dtype, device=xf.device)
    elif out.shape != (n, n_max + 1) or out.dtype != xf.dtype or not out.is_contiguous() or out.device != xf.device:
        raise ValueError("out must be a contiguous [count, n_max+1] tensor of x's dtype on x's device")
    if two_point and xf.dtype != torch.float64:
        raise TypeError("the two-point evaluation is a float64 path")
    fn = ("boys_eval_f64_two_point" if two_point else "boys_eval_f64") if xf.dtype == torch.float64 else "boys_eval_f32"
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


def boys_backward(x: torch.Tensor, g: torch.Tensor, n_max: int, F: torch.Tensor | None = None) -> torch.Tensor:
    """grad_x = -sum_m g[:, m] F_{m+1}(x) (float64).  g may be any 2-D view
    with non-negative strides, e.g. a weight vector expanded over the rows.
    F: saved forward rows with at least n_max+2 columns (else recomputed)."""
    xf = _check_input(x, (torch.float64,))
    n = xf.numel()
    if g.dim() != 2 or g.shape != (n, n_max + 1) or g.dtype != torch.float64 or not g.is_cuda:
        raise ValueError("g must be a float64 CUDA tensor of shape [count, n_max+1]")
    grad = torch.empty_like(xf)
    f_ptr, ld = 0, 0
    if F is not None:
        if F.dim() != 2 or F.shape[0] != n or F.shape[1] < n_max + 2 or F.stride(1) != 1 or F.dtype != torch.float64:
            raise ValueError("F must be float64 [count, >= n_max+2] with unit column stride")
        f_ptr, ld = F.data_ptr(), F.stride(0)
    with torch.cuda.device(xf.device):
        _capi.call("boys_eval_backward_f64", xf.data_ptr(), f_ptr, ld, g.data_ptr(), g.stride(0), g.stride(1), n,
                   int(n_max), grad.data_ptr(), _stream_ptr(xf.device))
    return grad


class BoysFunction(torch.autograd.Function):
    """F_0..F_{n_max}(x) with a hand-written adjoint.  The forward evaluates
    one order more (F_{n_max+1}) and keeps the rows, so the backward is the
    strided dot product grad_x = -sum_m g_m F_{m+1} read from HBM."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, n_max: int):
        F = boys(x, n_max + 1)
        ctx.save_for_backward(F)
        ctx.n_max = n_max
        ctx.x_shape = x.shape
        return F[:, : n_max + 1]

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (F,) = ctx.saved_tensors
        n_max = ctx.n_max
        if g.stride(0) < 0 or g.stride(1) < 0:
            g = g.contiguous()
        grad = torch.empty(F.shape[0], dtype=F.dtype, device=F.device)
        with torch.cuda.device(F.device):
            _capi.call("boys_eval_backward_f64", 0, F.data_ptr(), F.stride(0), g.data_ptr(), g.stride(0), g.stride(1),
                       F.shape[0], int(n_max), grad.data_ptr(), _stream_ptr(F.device))
        return grad.view(ctx.x_shape), None


def boys_autograd(x: torch.Tensor, n_max: int) -> torch.Tensor:
    """Differentiable F_0..F_{n_max}(x) for a float64 CUDA tensor."""
    if x.dtype != torch.float64:
        raise TypeError("the differentiable path is float64")
    return BoysFunction.apply(x, n_max)


class RaggedBatch:
    """A ragged batch laid out for boys_eval_ragged_f64.

    offsets (R+1) and n_max (R) describe the requests over a concatenated
    argument array; out_offsets and the output size follow from them and are
    computed once on the host.  All arrays are kept on the device, so the
    evaluation call itself needs no host synchronisation and can be captured
    in a CUDA graph (see capture())."""

    def __init__(self, offsets, n_max, device=None):
        import numpy as np

        offsets = np.asarray(offsets, dtype=np.int64)
        n_max = np.asarray(n_max, dtype=np.int32)
        if offsets.ndim != 1 or n_max.ndim != 1 or offsets.size != n_max.size + 1:
            raise ValueError("offsets must have one more entry than n_max")
        counts = np.diff(offsets)
        out_offsets = np.zeros_like(offsets)
        np.cumsum(counts * (n_max.astype(np.int64) + 1), out=out_offsets[1:])
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        self.num_requests = int(n_max.size)
        self.x_size = int(offsets[-1]) if offsets.size else 0
        self.out_size = int(out_offsets[-1]) if out_offsets.size else 0
        self.offsets = torch.from_numpy(offsets).to(dev)
        self.n_max = torch.from_numpy(n_max).to(dev)
        self.out_offsets = torch.from_numpy(out_offsets).to(dev)
        self.out_offsets_host = out_offsets
        ws = _capi.load().boys_ragged_workspace_bytes(self.num_requests)
        self.workspace = torch.empty(int(ws), dtype=torch.uint8, device=dev)

    def __call__(self, x: torch.Tensor, out: torch.Tensor | None = None, variant: int = -1) -> torch.Tensor:
        """Evaluate every request; returns the flat output (out_size doubles)."""
        xf = _check_input(x, (torch.float64,))
        if xf.numel() < self.x_size:
            raise ValueError("x is shorter than offsets[-1]")
        if out is None:
            out = torch.empty(self.out_size, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _capi.call("boys_eval_ragged_f64", xf.data_ptr(), xf.numel(), self.offsets.data_ptr(),
                       self.n_max.data_ptr(), self.out_offsets.data_ptr(), self.num_requests, out.data_ptr(),
                       out.numel(), self.workspace.data_ptr(), self.workspace.numel(), int(variant),
                       _stream_ptr(self.device))
        return out

    def errors(self) -> int:
        """Invalid requests seen by the last call (synchronises)."""
        import ctypes

        n = ctypes.c_int64(0)
        _capi.call("boys_ragged_errors", self.workspace.data_ptr(), ctypes.addressof(n), _stream_ptr(self.device))
        return int(n.value)

    def request_rows(self, out: torch.Tensor, r: int) -> torch.Tensor:
        """Rows of request r as a [count_r, n_max_r + 1] view of the flat output."""
        lo, hi = int(self.out_offsets_host[r]), int(self.out_offsets_host[r + 1])
        return out[lo:hi].view(-1, int(self.n_max[r].item()) + 1)

    def capture(self, x: torch.Tensor, out: torch.Tensor, variant: int = -1):
        """A CUDA graph replaying this batch's evaluation (x and out are fixed buffers)."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self(x, out, variant)  # first call sets up the kernels outside the capture
        torch.cuda.current_stream(self.device).wait_stream(s)
        with torch.cuda.graph(g):
            self(x, out, variant)
        return g


def ragged_variants() -> list[tuple[int, int]]:
    """(block size, tile) of each launch configuration of the ragged kernel."""
    import ctypes

    lib = _capi.load()
    out = []
    for v in range(lib.boys_ragged_num_variants()):
        b, t = ctypes.c_int(0), ctypes.c_int(0)
        _capi.call("boys_ragged_variant_info", v, ctypes.addressof(b), ctypes.addressof(t))
        out.append((b.value, t.value))
    return out


def boys_contract(x: torch.Tensor, n_max: int, c: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """out[i] = sum_m c[i, m] F_m(x_i) (c of shape [n_max+1], broadcast over
    the arguments, or [count, n_max+1]), with the F_m kept in registers.
    float64 or float32, following x."""
    xf = _check_input(x, (torch.float64, torch.float32))
    n = xf.numel()
    if c.dtype != xf.dtype or not c.is_cuda or c.device != xf.device:
        raise TypeError("c must be a CUDA tensor of x's dtype on x's device")
    if c.dim() == 1:
        if c.numel() != n_max + 1:
            raise ValueError("c must have n_max+1 entries")
        c_row, c_col = 0, c.stride(0)
    elif c.dim() == 2 and c.shape == (n, n_max + 1):
        c_row, c_col = c.stride(0), c.stride(1)
    else:
        raise ValueError("c must be [n_max+1] or [count, n_max+1]")
    if c_row < 0 or c_col < 0:
        c = c.contiguous()
        c_row, c_col = (0, 1) if c.dim() == 1 else (c.stride(0), c.stride(1))
    if out is None:
        out = torch.empty(n, dtype=xf.dtype, device=xf.device)
    fn = "boys_eval_contract_f64" if xf.dtype == torch.float64 else "boys_eval_contract_f32"
    with torch.cuda.device(xf.device):
        _capi.call(fn, xf.data_ptr(), n, int(n_max), c.data_ptr(), c_row, c_col, out.data_ptr(),
                   _stream_ptr(xf.device))
    return out
