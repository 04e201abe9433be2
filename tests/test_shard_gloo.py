"""The multi-rank partition on CPU: two gloo ranks each compute their shard
with the oracle at the shard's word offset, all-gather, and the
concatenation must equal the unsharded oracle fill (no data-path collective
exists in the library; the gather here is only the test's check)."""

import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2109_01329_gb300 import shard

CASES = [(0, 1, 1, 0.0, 1.0), (1, 2, 1, 0.0, 1.0), (0, 2, 2, 0.0, 1.0), (1, 0, 0, 0.0, 0.0)]


@pytest.fixture(scope="module", autouse=True)
def _library():
    # shard.py takes word offsets from grng_words_for, so the library must exist
    from paper_2109_01329_gb300 import build

    build.build()


def _worker(rank, world, port, n, q):
    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ok = True
        for engine, kind, dtype, p0, p1 in CASES:
            start, count, woff = shard.shard_range(rank, world, n, kind, dtype)
            part = oracle.generate(engine, 31, 7 + woff, kind, dtype, p0, p1, count)
            t = torch.from_numpy(part.view(np.uint8).copy())
            sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
            dist.all_gather(sizes, torch.tensor([t.numel()], dtype=torch.int64))
            mx = int(max(s.item() for s in sizes))
            padded = torch.zeros(mx, dtype=torch.uint8)
            padded[: t.numel()] = t
            bufs = [torch.zeros(mx, dtype=torch.uint8) for _ in range(world)]
            dist.all_gather(bufs, padded)
            if rank == 0:
                cat = np.concatenate([b[: int(s.item())].numpy() for b, s in zip(bufs, sizes)])
                full = oracle.generate(engine, 31, 7, kind, dtype, p0, p1, n).view(np.uint8)
                ok = ok and np.array_equal(cat, full)
        if rank == 0:
            q.put(ok)
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_concatenate():
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    n = 100_003
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=10) is True


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_ranges_tile(world):
    for n in [0, 1, 5, 1000, 10**6 + 3]:
        pos = 0
        for r in range(world):
            start, count, woff = shard.shard_range(r, world, n, 2, 2)
            assert start == pos and count >= 0 and start % 4 == 0 or start == n
            assert woff == 2 * start
            pos += count
        assert pos == n
