"""Option B on CPU ranks (paper Sec. 5): the lattice cut into z-slabs, one per rank, each
rank's deposit summed over the ranks.  Two gloo ranks; the per-rank deposit is a host-side
stand-in (the oracle on the rank's cubes, inside this test only: the partition and reduction
code in paper_1612_09491_gb300.shard imports no oracle).  The summed grid must equal the
one-rank deposit of the whole lattice; a rank that leaves between steps, or never arrives,
makes the other raise RankLost at its next check-in instead of waiting in the collective."""
from __future__ import annotations

import os
import socket
from datetime import timedelta

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1612_09491_gb300 import shard  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slab_bounds_cover_the_lattice_once():
    for n in (1, 5, 16, 17):
        for world in (1, 2, 3, 4, 7):
            spans = [shard.slab_bounds(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [k1 - k0 for k0, k1 in spans]
            assert max(sizes) - min(sizes) <= 1
    ids = shard.slab_cube_ids((4, 3, 5), 1, 3)
    assert ids.tolist() == list(range(12, 36))


def _setup(rank, world, port, sport):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=30))
    store = dist.TCPStore("127.0.0.1", sport, world, rank == 0, timeout=timedelta(seconds=30))
    return store


def _oracle_slab(pos, n, g):
    import oracle

    def slab(k0, k1):
        m, _ = oracle.deposit_lattice(pos, n, g, cube_ids=shard.slab_cube_ids(n, k0, k1), nthreads=1)
        return torch.from_numpy(m.copy())
    return slab


def _rank_sum(rank, world, port, sport, out):
    from pse_inputs import zeldovich_positions
    store = _setup(rank, world, port, sport)
    n, g = 12, 20
    pos = zeldovich_positions(n, -2.0, 1.5, seed=31)
    grids = []
    for step in range(2):
        grids.append(shard.deposit_sharded(_oracle_slab(pos, n, g), n, dist, store=store, step=step, timeout_s=20.0))
    out[rank] = [x.numpy().copy() for x in grids]
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sum_to_the_whole_deposit():
    import oracle
    from pse_inputs import zeldovich_positions
    world, port, sport = 2, _free_port(), _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_rank_sum, args=(world, port, sport, out), nprocs=world, join=True)
        res = dict(out)
    n, g = 12, 20
    ref, _ = oracle.deposit_lattice(zeldovich_positions(n, -2.0, 1.5, seed=31), n, g)
    for r in range(world):
        for grid in res[r]:
            np.testing.assert_allclose(grid, ref, rtol=1e-12, atol=1e-18)
            assert abs(grid.sum() - 1.0) < 1e-13


def _rank_leaves(rank, world, port, sport, out, announce):
    from pse_inputs import zeldovich_positions
    store = _setup(rank, world, port, sport)
    n, g = 8, 12
    pos = zeldovich_positions(n, -2.0, 1.0, seed=5)
    shard.deposit_sharded(_oracle_slab(pos, n, g), n, dist, store=store, step=0, timeout_s=20.0)
    if rank == 1:
        # rank 1 leaves between steps, with none of its work in flight
        if announce:
            shard.leave(store, 1)
        out[rank] = "left"
        return
    try:
        shard.deposit_sharded(_oracle_slab(pos, n, g), n, dist, store=store, step=1, timeout_s=2.0)
        out[rank] = "waited"
    except shard.RankLost as e:
        out[rank] = ("lost", e.missing, e.step)


@pytest.mark.parametrize("announce", [True, False])
def test_a_rank_that_leaves_stops_the_others(announce):
    world, port, sport = 2, _free_port(), _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_rank_leaves, args=(world, port, sport, out, announce), nprocs=world, join=True)
        res = dict(out)
    assert res[1] == "left"
    assert res[0] == ("lost", [1], 1)
