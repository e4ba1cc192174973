"""Ragged batches: one call over many requests with their own n_max must give
exactly (bitwise) the rows the plain FP64 path gives each request, for every
launch configuration, inside a CUDA graph, and must contain bad requests."""
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


def _batch(num_requests, seed, max_count=20000):
    from paper_2504_07637_gb300 import workloads

    rng = np.random.default_rng(seed)
    counts = np.floor(np.exp(rng.uniform(np.log(1), np.log(max_count), num_requests))).astype(np.int64)
    counts[:3] = [0, 1, 2049]  # empty, single and one-past-a-tile requests
    n_max = rng.integers(0, 17, num_requests).astype(np.int32)
    offsets = np.zeros(num_requests + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    x = workloads.plain(int(offsets[-1]), 53, seed=seed)
    return x, offsets, n_max


def _per_request(lib, x, offsets, n_max):
    import torch

    rows = []
    xd = torch.from_numpy(x).cuda()
    for r in range(n_max.size):
        lo, hi = int(offsets[r]), int(offsets[r + 1])
        rows.append(lib.boys(xd[lo:hi], int(n_max[r])).reshape(-1))
    return torch.cat(rows)


@pytest.mark.parametrize("variant", [-1, 0, 1, 2, 3, 4])
def test_matches_plain_launches_bitwise(lib, variant):
    import torch

    x, offsets, n_max = _batch(300, 1)
    batch = lib.RaggedBatch(offsets, n_max)
    out = batch(torch.from_numpy(x).cuda(), variant=variant)
    assert batch.errors() == 0
    assert torch.equal(out, _per_request(lib, x, offsets, n_max))


def test_against_oracle(lib, oracle_mod):
    import torch

    x, offsets, n_max = _batch(64, 2, max_count=3000)
    batch = lib.RaggedBatch(offsets, n_max)
    out = batch(torch.from_numpy(x).cuda())
    for r in range(64):
        got = batch.request_rows(out, r).cpu().numpy()
        ref = oracle_mod.boys(x[offsets[r]:offsets[r + 1]], int(n_max[r]))
        with np.errstate(invalid="ignore", divide="ignore"):
            rel = np.where(ref != 0, np.abs(got - ref) / np.abs(ref), np.abs(got))
        assert rel.max(initial=0) <= 2e-14, r


def test_graph_capture_and_replay(lib):
    import torch

    x, offsets, n_max = _batch(200, 3)
    batch = lib.RaggedBatch(offsets, n_max)
    xd = torch.from_numpy(x).cuda()
    out = torch.full((batch.out_size,), -1.0, dtype=torch.float64, device="cuda")
    g = batch.capture(xd, out)
    out.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    want = _per_request(lib, x, offsets, n_max)
    assert torch.equal(out, want)
    # replay on new arguments in the same buffer
    x2 = x * 0.5
    xd.copy_(torch.from_numpy(x2))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, _per_request(lib, x2, offsets, n_max))


def test_invalid_requests_are_counted_and_contained(lib):
    import torch

    from paper_2504_07637_gb300 import _capi

    x, offsets, n_max = _batch(40, 4, max_count=500)
    batch = lib.RaggedBatch(offsets, n_max)
    good = batch(torch.from_numpy(x).cuda()).clone()
    bad_n = n_max.copy()
    bad_n[5] = 17  # above the supported order
    bad_n[9] = -1
    batch.n_max.copy_(torch.from_numpy(bad_n))
    out = batch(torch.from_numpy(x).cuda())
    assert batch.errors() == 2
    for r in range(40):
        lo, hi = int(batch.out_offsets_host[r]), int(batch.out_offsets_host[r + 1])
        if r in (5, 9):
            assert torch.all(torch.isnan(out[lo:hi]))
        else:
            assert torch.equal(out[lo:hi], good[lo:hi])
    # an output range beyond out_size produces nothing and is counted
    oo = batch.out_offsets.clone()
    batch.n_max.copy_(torch.from_numpy(n_max))
    short = torch.full((batch.out_size - 1,), 7.0, dtype=torch.float64, device="cuda")
    _capi.call("boys_eval_ragged_f64", torch.from_numpy(x).cuda().data_ptr(), x.size, batch.offsets.data_ptr(),
               batch.n_max.data_ptr(), oo.data_ptr(), 40, short.data_ptr(), short.numel(),
               batch.workspace.data_ptr(), batch.workspace.numel(), -1, torch.cuda.current_stream().cuda_stream)
    assert batch.errors() >= 1


def test_autotuner_picks_a_variant(lib, tmp_path, monkeypatch):
    import torch

    from paper_2504_07637_gb300 import autotune

    monkeypatch.setenv("BOYS_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    x, offsets, n_max = _batch(100, 5)
    batch = lib.RaggedBatch(offsets, n_max)
    res = autotune.tune_ragged(batch, torch.from_numpy(x).cuda(), reps=2)
    assert 0 <= res["variant"] < len(lib.ragged_variants())
    assert len(res["all"]) == len(lib.ragged_variants())
    again = autotune.tune_ragged(batch, torch.from_numpy(x).cuda())
    assert again == res  # served from the cache
