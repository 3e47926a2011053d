"""The replicas-only multi-GPU path of bench.py, on CPU: two gloo ranks (no GPU).

Each rank reports its own step times; the job's step time is the slowest rank's, and
the throughput counts the units of every rank.
"""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    step_ms = [10.0 + rank, 12.0 + 3 * rank]  # rank 1 is the slow one
    ms, value = bench.replica_throughput(step_ms, 1000, dist, "cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    slow = (11.0 + 15.0) / 2
    for r in range(world):
        ms, value = res[r]
        assert ms == pytest.approx(slow)
        assert value == pytest.approx(world * 1000 / (slow * 1e-3))


def test_single_replica():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ms, value = bench.replica_throughput([2.0, 4.0], 600)
    assert ms == 3.0 and value == pytest.approx(2e5)


def test_clock_summary_reads_throttle_reasons():
    """The bench's clock record: median SM clock under load, the maximum clock, and every
    throttle reason seen Active in any sample (nvidia-smi csv rows, faked here)."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    cs = bench.ClockSampler(None)
    assert cs.summary()["reasons"] == ["unavailable"]
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    cs.rows = [[p.strip() for p in r.split(",")] for r in rows]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    cs.rows.append([p.strip() for p in "0, 1500, 2070, 700, 0x40, Not Active, Active, Not Active, Not Active".split(",")])
    assert cs.summary()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
