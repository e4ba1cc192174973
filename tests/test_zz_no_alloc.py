"""The ragged entry point that allocates nothing.

Some callers cannot provide device scratch memory (their device memory is
held by a pool the library may not touch, or they have no allocator at hand);
boys_eval_ragged_f64_noalloc serves them from a fixed array inside the
library.  Here it must reproduce boys_eval_ragged_f64 (caller workspace) on
two calls in a row, and refuse batches larger than its array.  This file is
collected last so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 2e-14  # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07637_gb300 import _capi, workloads
    from paper_2504_07637_gb300.build import build_library

    build_library()
    return torch, _capi, workloads


def _batch(workloads, seed, num_requests=257):
    rng = np.random.default_rng(seed)
    counts = np.floor(np.exp(rng.uniform(0, np.log(9000), num_requests))).astype(np.int64)
    n_max = rng.integers(0, 17, num_requests).astype(np.int32)
    offsets = np.zeros(num_requests + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    out_offsets = np.zeros_like(offsets)
    np.cumsum(counts * (n_max.astype(np.int64) + 1), out=out_offsets[1:])
    x = workloads.plain(int(offsets[-1]), 53, seed=seed)
    return x, offsets, n_max, out_offsets


def _rel(a, b):
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(b != 0, np.abs(a - b) / np.abs(b), np.abs(a - b))
    return float(np.nanmax(r)) if r.size else 0.0


def test_matches_workspace_entry_point_twice(env):
    torch, capi, workloads = env
    lib = capi.load()
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((11, 12)):  # two calls in a row, different batches
        x, offsets, n_max, out_offsets = _batch(workloads, seed)
        R, total = n_max.size, int(out_offsets[-1])
        xd = torch.from_numpy(x).cuda()
        od, nd, ood = (torch.from_numpy(a).cuda() for a in (offsets, n_max, out_offsets))
        ws_bytes = lib.boys_ragged_workspace_bytes(R)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        want = torch.empty(total, dtype=torch.float64, device="cuda")
        capi.call("boys_eval_ragged_f64", xd.data_ptr(), x.size, od.data_ptr(), nd.data_ptr(), ood.data_ptr(), R,
                  want.data_ptr(), total, ws.data_ptr(), ws_bytes, -1, stream)
        got = torch.full((total,), -7.0, dtype=torch.float64, device="cuda")
        capi.call("boys_eval_ragged_f64_noalloc", xd.data_ptr(), x.size, od.data_ptr(), nd.data_ptr(),
                  ood.data_ptr(), R, got.data_ptr(), total, -1, stream)
        torch.cuda.synchronize()
        g, w = got.cpu().numpy(), want.cpu().numpy()
        assert not np.any(g == -7.0), call
        assert _rel(g, w) <= TOL, call


def test_refuses_batches_beyond_its_array(env):
    torch, capi, _ = env
    f = capi.load().boys_eval_ragged_f64_noalloc
    too_many = 65536 + 1
    # refused on the host before any pointer is used
    assert f(8, 10, 8, 4, 8, too_many, 8, 10, -1, None) == 5
