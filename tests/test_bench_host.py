"""Host-side logic of bench.py: the multi-rank aggregation (replicas, no
collective on the data path) over gloo with two CPU ranks, and the
algorithmic byte / MAC counts of the HomConv launch."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    secs, units = bench.aggregate(1.0 + rank, 10.0 * (rank + 1), world)
    q.put((rank, secs, units))
    dist.destroy_process_group()


def test_aggregate_takes_slowest_rank_and_sums_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, secs, units in res:
        assert secs == 2.0 and units == 30.0


def test_homconv_counts():
    import bench
    import fdsc_inputs as FI

    ls = FI.CONFIGS["cfg1"].layers[0]
    byts, macs = bench.layer_counts(ls, 32, 1, 1, 2048, addends=0)
    assert macs == 2 * 64 * 64 * 32 * 32  # equals the useful MACs: g_c H W = S
    assert byts == 8 * 64 * 32 * 2048 + 8 * (2 * 32 * 2048 + 3 * 64 * 2048)
