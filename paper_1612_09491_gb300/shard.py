"""Several GPUs by the paper's option B (Sec. 5): the Lagrangian lattice is cut into z-slabs
of cube layers, one slab per rank; every rank deposits the tetrahedra of its slab onto the
whole deposit grid (or the whole set of octree leaf blocks), and the grids are summed over
the ranks.  Tetrahedra are independent, so the sum is the one-rank deposit; the only
exchange is the reduction of the float64 grid.

* Each rank holds the whole position array (the cubes of its slab read one particle layer
  beyond it, and an octree built from tetrahedron sizes is then the same on every rank: its
  histograms count integers, so the tree is identical without an exchange).
* The reduction is ``torch.distributed.all_reduce(SUM)`` on the grid tensor: NCCL on GPUs,
  gloo on CPU tensors.  FP32 deposits are renormalised per rank to the mass of that rank's
  tetrahedra, so the sum keeps the total mass.
* Before each reduction the ranks check in through a key-value store with a deadline: a
  rank that has left (or that never arrives) makes the others raise ``RankLost`` instead of
  waiting in the collective.
"""
from __future__ import annotations

import time
from datetime import timedelta


class RankLost(RuntimeError):
    """A rank did not check in before the reduction."""

    def __init__(self, missing, step):
        super().__init__(f"rank(s) {sorted(missing)} did not reach step {step}")
        self.missing = sorted(missing)
        self.step = step


def slab_bounds(n_layers: int, world: int, rank: int) -> tuple[int, int]:
    """Cube layers [k0, k1) of `rank` out of `world` (contiguous, sizes differ by at most one)."""
    if not (0 <= rank < world) or n_layers < 0:
        raise ValueError("rank out of range")
    base, extra = divmod(n_layers, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def slab_cube_ids(nc, k0: int, k1: int):
    """Cube ids (i + nc0 (j + nc1 k), x fastest) of the cube layers k0 <= k < k1 of a lattice of
    nc = (nc0, nc1, nc2) cubes (an int: the same on every axis), as an int64 numpy array."""
    import numpy as np
    nc0, nc1 = (nc, nc) if isinstance(nc, int) else (int(nc[0]), int(nc[1]))
    return np.arange(k0 * nc0 * nc1, k1 * nc0 * nc1, dtype=np.int64)


def leave(store, rank: int) -> None:
    """Announce that `rank` leaves the job (between steps): the others stop at their next
    check-in instead of waiting for it."""
    store.set(f"left/{rank}", "1")


def check_in(store, step: int, world: int, rank: int, timeout_s: float = 10.0, poll_s: float = 0.01) -> None:
    """Mark `rank` as arrived at `step`, then wait until every rank has, raising RankLost when a
    rank has left or `timeout_s` passes first."""
    store.set(f"step{step}/{rank}", "1")
    keys = [f"step{step}/{r}" for r in range(world)]
    deadline = time.monotonic() + timeout_s
    while True:
        missing = [r for r, k in enumerate(keys) if not store.check([k])]
        if not missing:
            return
        left = [r for r in range(world) if store.check([f"left/{r}"])]
        if left or time.monotonic() >= deadline:
            raise RankLost(left or missing, step)
        time.sleep(poll_s)


def deposit_sharded(deposit_slab, n_layers: int, dist, *, store=None, step: int = 0, timeout_s: float = 10.0):
    """One sharded deposit: this rank deposits cube layers slab_bounds(n_layers, world, rank)
    with ``deposit_slab(k0, k1)`` (which returns the whole grid as a tensor holding only this
    slab's deposits), checks in through `store` (if given), and sums the grids over the ranks.
    Returns the summed grid (every rank holds it)."""
    rank, world = dist.get_rank(), dist.get_world_size()
    k0, k1 = slab_bounds(n_layers, world, rank)
    grid = deposit_slab(k0, k1)
    if store is not None:
        check_in(store, step, world, rank, timeout_s)
    dist.all_reduce(grid, op=dist.ReduceOp.SUM)
    return grid


def default_timeout(seconds: float) -> timedelta:
    """A process-group timeout for init_process_group: a collective that a lost rank never
    joins fails after this long instead of waiting."""
    return timedelta(seconds=seconds)


def deposit_uniform_sharded(pos, n: int, grid_n, dist, *, store=None, step: int = 0, timeout_s: float = 10.0, **kw):
    """pse_deposit_uniform of a periodic n^3 lattice, sharded over the ranks of `dist` by
    z-slabs (each rank on its own GPU, `pos` the whole lattice on that GPU); keyword
    arguments go to deposit_uniform."""
    import torch

    from . import deposit_uniform

    def slab(k0, k1):
        ids = torch.from_numpy(slab_cube_ids(n, k0, k1)).to(pos.device)
        return deposit_uniform(pos, n, grid_n, cube_ids=ids, **kw)
    return deposit_sharded(slab, n, dist, store=store, step=step, timeout_s=timeout_s)


def deposit_octree_sharded(pos, n: int, octree, dist, *, store=None, step: int = 0, timeout_s: float = 10.0, **kw):
    """pse_deposit_octree of a periodic n^3 lattice sharded the same way (every rank holds the
    same octree); keyword arguments go to deposit_octree."""
    import torch

    from . import deposit_octree

    def slab(k0, k1):
        ids = torch.from_numpy(slab_cube_ids(n, k0, k1)).to(pos.device)
        return deposit_octree(pos, n, octree, cube_ids=ids, **kw)
    return deposit_sharded(slab, n, dist, store=store, step=step, timeout_s=timeout_s)
