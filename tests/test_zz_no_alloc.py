"""The ragged entry point that allocates nothing.

Some callers cannot provide device scratch memory (their device memory is
held by a pool the library may not touch, or they have no allocator at hand);
boys_eval_ragged_f64_noalloc serves them from a fixed array inside the
library.  Here it must reproduce boys_eval_ragged_f64 (caller workspace) bit
for bit on two calls in a row, match the oracle, fill its whole array of
requests, and refuse batches larger than the array.  This file is
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


def _run_both(torch, capi, x, offsets, n_max, out_offsets):
    """(no-allocation result, workspace result) of one batch, as host arrays."""
    lib = capi.load()
    stream = torch.cuda.current_stream().cuda_stream
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
    return got.cpu().numpy(), want.cpu().numpy()


def _oracle_error(oracle_mod, x, offsets, n_max, out_offsets, got):
    """Max relative error of every request's rows against the oracle."""
    worst = 0.0
    for n in np.unique(n_max):
        reqs = np.nonzero(n_max == n)[0]
        xs = np.concatenate([x[offsets[r]:offsets[r + 1]] for r in reqs])
        rows = np.concatenate([got[out_offsets[r]:out_offsets[r + 1]] for r in reqs]).reshape(-1, int(n) + 1)
        ref = oracle_mod.boys(xs, int(n))
        nz = ref != 0
        assert np.all(rows[~nz] == 0)
        worst = max(worst, float(np.max(np.abs(rows[nz] - ref[nz]) / ref[nz], initial=0.0)))
    return worst


def test_matches_workspace_entry_point_twice(env, oracle_mod):
    torch, capi, workloads = env
    for call, seed in enumerate((11, 12)):  # two calls in a row, different batches
        x, offsets, n_max, out_offsets = _batch(workloads, seed)
        got, want = _run_both(torch, capi, x, offsets, n_max, out_offsets)
        # the same kernels and launch variant: the same bits, and every element written
        assert not np.any(got == -7.0), call
        assert np.array_equal(got, want, equal_nan=False), call
        if call == 0:
            assert _oracle_error(oracle_mod, x, offsets, n_max, out_offsets, got) <= TOL


def test_full_array_of_requests(env):
    # exactly BOYS_RAGGED_NOALLOC_MAX_REQUESTS small requests: the tile prefix
    # then lives in the array's last bytes (beyond the shared-memory copy)
    torch, capi, workloads = env
    R = 65536
    rng = np.random.default_rng(21)
    counts = rng.integers(0, 4, R).astype(np.int64)
    n_max = rng.integers(0, 17, R).astype(np.int32)
    offsets = np.zeros(R + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    out_offsets = np.zeros_like(offsets)
    np.cumsum(counts * (n_max.astype(np.int64) + 1), out=out_offsets[1:])
    x = workloads.plain(int(offsets[-1]), 53, seed=21)
    got, want = _run_both(torch, capi, x, offsets, n_max, out_offsets)
    assert not np.any(got == -7.0)
    assert np.array_equal(got, want, equal_nan=False)


def test_refuses_batches_beyond_its_array(env):
    torch, capi, _ = env
    f = capi.load().boys_eval_ragged_f64_noalloc
    too_many = 65536 + 1
    # refused on the host before any pointer is used
    assert f(8, 10, 8, 4, 8, too_many, 8, 10, -1, None) == 5
