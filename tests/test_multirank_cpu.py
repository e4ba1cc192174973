"""The N > 1 benchmark path on CPU: two gloo ranks draw distinct shards,
cover a split array exactly once, and agree on the slowest rank's time."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_2504_07637_gb300 import shard, workloads

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x = workloads.scale(1000, seed=shard.shard_seed(workloads.SEED_BASE + 1, rank))
        lo, hi = shard.shard_range(10_001, rank, world)
        t = shard.max_over_ranks(float(rank + 1) * 1.5)
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([x[:8], [lo, hi, t]]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    r0, r1 = (np.load(tmp_path / f"r{r}.npy") for r in range(world))
    assert not np.array_equal(r0[:8], r1[:8])  # independent shards
    assert r0[8] == 0 and r0[9] == r1[8] and r1[9] == 10_001  # contiguous cover
    assert r0[10] == r1[10] == 3.0  # slowest rank's time on every rank


def test_shard_range_covers_once():
    from paper_2504_07637_gb300 import shard

    for count in (0, 1, 7, 100, 12345):
        for world in (1, 2, 3, 8):
            seen = np.zeros(count, dtype=int)
            for r in range(world):
                lo, hi = shard.shard_range(count, r, world)
                seen[lo:hi] += 1
            assert np.all(seen == 1)
