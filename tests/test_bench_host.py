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

    ls = FI.CONFIGS["cifar_32x32x64_b1"].layers[0]
    byts, macs = bench.layer_counts(ls, 32, 1, 1, 2048, addends=0)
    assert macs == 2 * 64 * 64 * 32 * 32  # equals the useful MACs: g_c H W = S
    assert byts == 8 * 64 * 32 * 2048 + 8 * (2 * 32 * 2048 + 3 * 64 * 2048)


def test_reference_arm_line():
    """bench.py --impl reference times the oracle on the host and prints one
    JSON line with the contract's keys (no GPU involved)."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3"],
                         cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "layers/s" and d["steps"] == 3 and d["warmup"] == 3
    # ms_per_step is the measured wall time of a step; a step is a stated fraction of a layer
    frac = d["layer_fraction_per_step"]
    assert 0 < frac <= 1 and d["value"] > 0
    assert abs(d["value"] - frac * 1e3 / d["ms_per_step"]) < 1e-6 * d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "layers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
