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


def test_uniform_streamed_compensated_equals_one_shot():
    """Compensated accumulation across slabs: the float pairs persist over every slab and are
    converted once at the end."""
    cfg = CONFIGS[1]
    pos = config_positions(cfg)
    ref = pse.deposit_uniform(torch.from_numpy(pos).cuda(), cfg.n, cfg.grid_n,
                              precision=pse.PSE_FP32_COMPENSATED).cpu().numpy()
    got = pse.deposit_uniform_streamed(torch.from_numpy(pos).pin_memory(), cfg.n, cfg.grid_n, 5,
                                       precision=pse.PSE_FP32_COMPENSATED).cpu().numpy()
    e = cell_errors(got, ref)
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


def _max_displacement(pos, n):
    """Largest |x - q| per axis over the lattice, nearest periodic image (positions on the GPU)."""
    p = pos.view(n, n, n, 3)
    q = torch.arange(n, device=pos.device, dtype=torch.float32) / n
    out = 0.0
    for a, shape in enumerate(((1, 1, n), (1, n, 1), (n, 1, 1))):
        d = p[..., a] - q.view(*shape)
        d -= torch.round(d)
        out = max(out, float(d.abs().max()))
    return out


def _cubes_reaching(posh, n, cell, g, psi_max):
    """Cubes whose corner bounding box (corners taken at the image nearest corner 0) touches `cell`
    of a periodic g^3 grid: the Lagrangian window that displacements up to psi_max allow, then
    the exact box test on the cubes of that window."""
    h = 1.0 / n
    ax = []
    for a in range(3):
        lo = int(np.floor((cell[a] / g - h - psi_max) * n)) - 1
        hi = int(np.ceil(((cell[a] + 1) / g + psi_max) * n)) + 1
        ax.append(np.unique(np.arange(lo, hi + 1) % n))
    kk, jj, ii = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    p0 = posh[ii + n * (jj + n * kk)].astype(np.float64)
    lo = p0.copy()
    hi = p0.copy()
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                c = posh[(ii + dx) % n + n * ((jj + dy) % n + n * ((kk + dz) % n))].astype(np.float64)
                d = c - p0
                d -= np.floor(d + 0.5)
                lo = np.minimum(lo, p0 + d)
                hi = np.maximum(hi, p0 + d)
    blo = np.floor(lo * g).astype(np.int64)
    ext = np.floor(hi * g).astype(np.int64) - blo
    sel = np.all(np.mod(np.asarray(cell) - blo, g) <= ext, axis=1)
    return (ii + n * (jj + n * kk))[sel]


def test_config5_streamed_full_size_sampled_cells():
    """1024^3 particles (6.4B tetrahedra), k^-2, rms 3 spacings, streamed from pinned host memory in
    z-slabs of 64 cube layers onto the octree of 128^3-cell blocks, levels 0-4 (2048^3 finest), in
    the bench's launch configuration: the whole deposit conserves mass and counts every
    tetrahedron; 6 random leaf cells match the oracle's exact overlaps (FP64) of every
    tetrahedron that can reach them."""
    from pse_inputs import zeldovich_positions_device
    cfg = CONFIGS[5]
    n, bc = cfg.n, cfg.bc
    pos = zeldovich_positions_device(n, cfg.spectral_index, cfg.rms_disp, cfg.seed, device="cuda")
    psi_max = _max_displacement(pos, n) + 1.0 / n
    h = torch.empty((n ** 3, 3), dtype=torch.float32).pin_memory()
    h.copy_(pos)
    del pos
    torch.cuda.empty_cache()
    oct_ = pse.build_octree_streamed(h, n, bc, cfg.max_level, 64, 2.0)
    leaves = oct_.leaves()
    assert sum(8.0 ** -int(l) for l in leaves[:, 0]) == pytest.approx(1.0, abs=1e-12)
    out, st = pse.deposit_octree_streamed(h, n, oct_, 64, stats=True, tuning={"blocks_per_sm": 4})
    assert st["tets"] == cfg.n_tets
    assert abs(float(out.sum()) - 1.0) <= 1e-12
    posh = h.numpy()
    mt = 1.0 / (6 * n ** 3)
    rng = np.random.default_rng(55)
    for _ in range(6):
        li = int(rng.integers(0, len(leaves)))
        lvl, lx, ly, lz = (int(v) for v in leaves[li])
        cx, cy, cz = (int(v) for v in rng.integers(0, bc, 3))
        g = bc << lvl
        cell = np.array([lx * bc + cx, ly * bc + cy, lz * bc + cz])
        got = float(out[li, cz, cy, cx])
        exp = 0.0
        for c in _cubes_reaching(posh, n, cell, g, psi_max):
            for s in range(6):
                tet = oracle.lattice_tet(posh, n, int(c), s)
                vol = oracle.tet_volume(tet)
                if vol == 0.0:  # degenerate: all its mass goes to the cell of the vertex centroid
                    exp += mt * bool(np.all(np.mod(np.floor(tet.mean(0) * g), g) == cell))
                    continue
                cells, vols = oracle.tet_cells(tet, np.full(3, 1.0 / g))
                hit = np.all(np.mod(cells, g) == cell, axis=1)
                exp += mt * vols[hit].sum() / vol
        assert abs(got - exp) <= 1e-5 * max(exp, 1e-3 / g ** 3), (cell, lvl, got, exp)
