"""Slab streaming from host memory (pse_*_streamed) against the one-shot deposits.

The streamed deposit visits the same cubes as the one-shot one, slab by slab, so the
counters must agree exactly and the masses to FP32 rounding (FP64 path: to 1e-12).
Slab sizes that do not divide the lattice, single-layer slabs and one slab covering
the whole lattice are all exercised; the halo row wraps around the periodic box.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1612_09491_gb300 as pse  # noqa: E402
from paper_1612_09491_gb300.metrics import cell_errors  # noqa: E402
from pse_inputs import CONFIGS, config_positions, lattice_positions, zeldovich_positions  # noqa: E402

pytestmark = pytest.mark.gpu

COUNTERS = ("tets", "bbox_cells", "inside_cells", "partial_clips", "fp64_redos", "degenerate_tets",
            "single_cell_tets")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1612_09491_gb300 import build
    build.build()
    pse._lib.load()
    yield


@pytest.mark.parametrize("slab", [1, 5, 32, 40])
@pytest.mark.parametrize("sched", [pse.PSE_WARP_COOPERATIVE, pse.PSE_BINNED_PERSISTENT])
def test_uniform_streamed_equals_one_shot(slab, sched):
    cfg = CONFIGS[1]
    pos = config_positions(cfg)
    ref, sr = pse.deposit_uniform(torch.from_numpy(pos).cuda(), cfg.n, cfg.grid_n, schedule=sched, stats=True)
    h = torch.from_numpy(pos).pin_memory()
    got, sg = pse.deposit_uniform_streamed(h, cfg.n, cfg.grid_n, slab, schedule=sched, stats=True)
    for k in COUNTERS:
        assert sr[k] == sg[k], k
    e = cell_errors(got.cpu().numpy(), ref.cpu().numpy())
    assert e["max_rel"] <= 2e-6 and e["mass"] <= 1e-13, e


def test_uniform_streamed_fp64_matches_oracle_from_pageable_memory():
    n, g = 12, 20
    pos = zeldovich_positions(n, -2.0, 1.5, seed=31)
    ref, _ = oracle.deposit_lattice(pos, n, g)
    got = pse.deposit_uniform_streamed(pos, n, g, 5, precision=pse.PSE_FP64_PLAIN,
                                       schedule=pse.PSE_THREAD_PER_TET).cpu().numpy()
    e = cell_errors(got, ref)
    assert e["max_rel"] <= 1e-9 and e["mass"] <= 1e-13, e


def _squeezed(n, seed=0):
    q = lattice_positions(n).astype(np.float64)
    c = np.array([0.3, 0.6, 0.9])  # near the top of the box: slabs and the halo wrap cross it
    d = q - c
    d -= np.round(d)
    r = np.linalg.norm(d, axis=1, keepdims=True)
    p = np.where(r < 0.25, c + d * 0.3, q)
    p = p + np.random.default_rng(seed).normal(0, 0.2 / n, p.shape)
    return np.mod(p, 1.0).astype(np.float32)


def test_octree_streamed_build_and_deposit_equal_one_shot():
    n, bc, ml = 16, 4, 4
    pos = _squeezed(n)
    dpos = torch.from_numpy(pos).cuda()
    one = pse.build_octree_from_tet_sizes(dpos, n, bc, ml, 2.0)
    h = torch.from_numpy(pos).pin_memory()
    for slab in (1, 3, 16):
        st = pse.build_octree_streamed(h, n, bc, ml, slab, 2.0)
        np.testing.assert_array_equal(st.leaves(), one.leaves())
    assert len(set(one.leaves()[:, 0].tolist())) > 1
    ref, sr = pse.deposit_octree(dpos, n, one, stats=True)
    for slab in (3, 7):
        got, sg = pse.deposit_octree_streamed(h, n, one, slab, stats=True)
        for k in COUNTERS:
            assert sr[k] == sg[k], k
        e = cell_errors(got.cpu().numpy(), ref.cpu().numpy())
        assert e["max_rel"] <= 2e-6 and e["mass"] <= 1e-13, e
    # and the octree deposit against the oracle
    o, _ = oracle.deposit_octree(pos, n, one.leaves(), bc, ml)
    assert cell_errors(got.cpu().numpy(), o)["max_rel"] <= 1e-5


def test_streamed_rejects():
    pos = lattice_positions(8)
    with pytest.raises(pse.PseError):
        pse.deposit_uniform_streamed(pos, 8, 8, 0)  # slab_cubes < 1
    with pytest.raises(pse.PseError):
        pse.deposit_uniform_streamed(pos, 8, 8, 2, tuning={"use_graph": 1}, schedule=pse.PSE_BINNED_PERSISTENT)
