"""Replica-parallel host logic on CPU: two gloo ranks, no GPU.

The bounding path shards by subdomain with no exchange during the
iterations; what crosses ranks is the partition of the subdomain list, the
optional all-gather of the bounds and the max-over-ranks step time.
"""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from paper_2104_06718_gb300.replicas import block_range, gather_rows, max_over_ranks


@pytest.mark.parametrize("n_total", [0, 1, 7, 8, 2048, 2049])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_blocks_partition_the_subdomains(n_total, world):
    seen = []
    sizes = []
    for r in range(world):
        s, c = block_range(n_total, world, r)
        seen.extend(range(s, s + c))
        sizes.append(c)
    assert seen == list(range(n_total))
    assert max(sizes) - min(sizes) <= 1
    assert sizes == sorted(sizes, reverse=True)


def test_block_range_rejects_bad_arguments():
    for args in [(4, 0, 0), (4, 2, 2), (4, 2, -1), (-1, 2, 0)]:
        with pytest.raises(ValueError):
            block_range(*args)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_total, results):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        start, count = block_range(n_total, world, rank)
        # this rank's "bounds": a value that identifies the subdomain, plus a
        # second column, as for rho rows
        local = torch.stack([torch.arange(start, start + count, dtype=torch.float64),
                             -torch.arange(start, start + count, dtype=torch.float64)], dim=1)
        full = gather_rows(local, n_total)
        t = max_over_ranks([1.0 + rank, 10.0 - rank])
        results[rank] = (full.tolist(), t)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_total", [7, 8])
def test_two_gloo_ranks_gather_bounds_and_time(n_total):
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, n_total, results)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        for p in procs:
            if p.is_alive():
                p.kill()
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        got = dict(results)
    expect = [[float(i), -float(i)] for i in range(n_total)]
    for r in range(world):
        full, t = got[r]
        assert full == expect
        assert t == [2.0, 10.0]
