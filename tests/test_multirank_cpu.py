"""The benchmark's multi-rank path on CPU: two gloo ranks.

Chains are independent Markov chains, so ranks exchange nothing on the data
path; the only collective is the max-reduction of the timed region.  Checks
that the ranks' Philox chain words are disjoint, that the reduction returns
the slowest rank's time on every rank, and the whole-job rate."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n_chains, q):
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ids = bench.rank_chain_ids(rank, n_chains)
        t_ms = 100.0 * (rank + 1)  # this rank's timed region
        mx = bench.max_over_ranks(torch, dist, t_ms, "cpu")
        rate = bench.aggregate_rate(world, 1000, 4, mx)
        q.put((rank, ids, mx, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, n_chains = 2, 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n_chains, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    all_ids = out[0][1] + out[1][1]
    assert sorted(all_ids) == list(range(world * n_chains))
    for _, _, mx, rate in out:
        assert mx == 200.0
        assert rate == pytest.approx(world * 1000 * 4 / 0.2)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(torch, None, 3.5, "cpu") == 3.5
    assert bench.rank_chain_ids(2, 3) == [6, 7, 8]
