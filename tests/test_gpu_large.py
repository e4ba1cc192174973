"""Maximum sizes: argument counts past 2^31 (64-bit indexing everywhere) and
ragged batches large enough to leave the shared-memory tile prefix."""
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


def _rel(got, ref):
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(ref != 0, np.abs(got - ref) / np.abs(ref), np.abs(got))


@pytest.mark.parametrize("dtype,tol", [("float64", 2e-14), ("float32", 2e-6)])
def test_count_beyond_int32(lib, oracle_mod, dtype, tol):
    # 2^31 + 3 arguments drawn on the device (seeded), n_max = 0 and 1
    import torch

    count = (1 << 31) + 3
    tdt = getattr(torch, dtype)
    g = torch.Generator(device="cuda").manual_seed(2504_07637)
    x = torch.rand(count, generator=g, dtype=torch.float32, device="cuda").mul_(60.0).to(tdt)
    for n_max in (0, 1):
        out = lib.boys(x, n_max)
        assert out.shape == (count, n_max + 1)
        idx = np.concatenate([np.arange(5), np.random.default_rng(n_max).integers(0, count, 4000),
                              np.arange(count - 5, count), [(1 << 31) - 1, 1 << 31]])
        it = torch.from_numpy(idx).cuda()
        got = out[it].cpu().numpy().astype(np.float64)
        ref = oracle_mod.boys(x[it].cpu().numpy().astype(np.float64), n_max)
        assert _rel(got, ref).max() <= tol, (dtype, n_max)
        del out
    del x
    torch.cuda.empty_cache()


def test_ragged_beyond_shared_prefix(lib):
    # 20,000 requests: the tile prefix no longer fits in shared memory and is
    # searched in global memory; rows must equal one plain launch per n_max group
    import torch

    from paper_2504_07637_gb300 import workloads

    rng = np.random.default_rng(9)
    R = 20000
    counts = rng.integers(0, 60, R)
    n_max = rng.integers(0, 17, R).astype(np.int32)
    offsets = np.zeros(R + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    x = workloads.plain(int(offsets[-1]), 53, seed=10)
    batch = lib.RaggedBatch(offsets, n_max)
    out = batch(torch.from_numpy(x).cuda()).cpu().numpy()
    assert batch.errors() == 0
    for n in range(17):
        rs = np.nonzero(n_max == n)[0]
        xs = np.concatenate([x[offsets[r]:offsets[r + 1]] for r in rs])
        rows = lib.boys(torch.from_numpy(xs).cuda(), n).cpu().numpy().reshape(-1)
        got = np.concatenate([out[batch.out_offsets_host[r]:batch.out_offsets_host[r + 1]] for r in rs])
        assert np.array_equal(got, rows), n


def test_full_size_ragged_configuration_sampled(lib, oracle_mod):
    # the benchmark's batch: 4,096 requests, counts log-uniform on [64, 65536], n_max 0..16
    import torch

    from paper_2504_07637_gb300 import workloads

    x, offsets, n_max = workloads.ragged(4096, 16)
    batch = lib.RaggedBatch(offsets, n_max)
    out = batch(torch.from_numpy(x).cuda())
    assert batch.errors() == 0
    rng = np.random.default_rng(4)
    for r in rng.choice(4096, 48, replace=False):
        rows = batch.request_rows(out, int(r)).cpu().numpy()
        lo, hi = int(offsets[r]), int(offsets[r + 1])
        pick = rng.choice(hi - lo, min(256, hi - lo), replace=False)
        ref = oracle_mod.boys(x[lo:hi][pick], int(n_max[r]))
        assert _rel(rows[pick], ref).max() <= 2e-14, r
