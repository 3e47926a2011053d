"""Octree (adaptive deposit grid, Sec. 4) on the GPU against the oracle.

* deposit: the same leaf set is given to the CUDA path (pse_octree_from_leaves) and to
  the oracle; leaf-block masses compared cell by cell (C13 measures).
* build: the CUDA builder decides refinement from a 64-bin histogram (lower-median
  bin edge); the oracle uses the exact lower median.  Both must agree on every node
  whose exact median is not within one bin width of the threshold.
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

PATHS = [
    ("fp64-thread", pse.PSE_FP64_PLAIN, pse.PSE_THREAD_PER_TET, 1e-9),
    ("fp32-thread", pse.PSE_FP32_FP64ACC, pse.PSE_THREAD_PER_TET, 1e-5),
    ("fp32-warp", pse.PSE_FP32_FP64ACC, pse.PSE_WARP_COOPERATIVE, 1e-5),
    ("fp32c-warp", pse.PSE_FP32_COMPENSATED, pse.PSE_WARP_COOPERATIVE, 1e-5),
]
BIN = 10 ** (6 / 64)  # ratio of one histogram bin


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1612_09491_gb300 import build
    build.build()
    pse._lib.load()
    yield


def squeezed_lattice(n, center=(0.3, 0.6, 0.4), radius=0.22, factor=0.3, jitter=0.2, seed=0):
    q = lattice_positions(n).astype(np.float64)
    c = np.asarray(center)
    d = q - c
    r = np.linalg.norm(d, axis=1, keepdims=True)
    p = np.where(r < radius, c + d * factor, q)
    p = p + np.random.default_rng(seed).normal(0, jitter / n, p.shape)
    return np.mod(p, 1.0).astype(np.float32)


def gpu_octree_deposit(pos, n, leaves, bc, max_level, prec, sched, **kw):
    oct_ = pse.octree_from_leaves(leaves, bc, max_level)
    out = pse.deposit_octree(torch.from_numpy(pos).cuda(), n, oct_, precision=prec, schedule=sched, **kw)
    if isinstance(out, tuple):
        return out[0].cpu().numpy(), out[1]
    return out.cpu().numpy()


@pytest.mark.parametrize("name,prec,sched,tol", PATHS)
def test_single_leaf_equals_uniform(name, prec, sched, tol):
    n, bc = 12, 24
    pos = zeldovich_positions(n, -2.0, 1.0, seed=4)
    m = gpu_octree_deposit(pos, n, np.array([[0, 0, 0, 0]], np.int32), bc, 0, prec, sched)
    ref, _ = oracle.deposit_lattice(pos, n, bc)
    e = cell_errors(m[0], ref)
    assert e["max_rel"] <= tol, e


@pytest.mark.parametrize("name,prec,sched,tol", PATHS)
def test_adaptive_tree_matches_oracle(name, prec, sched, tol):
    n, bc, ml = 16, 4, 4
    pos = squeezed_lattice(n)
    leaves, _ = oracle.build_octree(pos, n, bc, ml)
    assert len(set(leaves[:, 0].tolist())) > 1
    ref, _ = oracle.deposit_octree(pos, n, leaves, bc, ml)
    m, st = gpu_octree_deposit(pos, n, leaves, bc, ml, prec, sched, stats=True)
    e = cell_errors(m, ref)
    assert e["max_rel"] <= tol, e
    assert e["mass"] <= (1e-13 if prec == pse.PSE_FP64_PLAIN else 1e-12), e
    assert st["tets"] == 6 * n ** 3


@pytest.mark.parametrize("name,prec,sched,tol", PATHS)
def test_shell_crossed_tree_matches_oracle(name, prec, sched, tol):
    n, bc, ml = 16, 4, 3
    pos = zeldovich_positions(n, -1.5, 3.0, seed=8)
    leaves = np.array([[1, x, y, z] for z in range(2) for y in range(2) for x in range(2)][:7] +
                      [[2, 2 * 1 + (c & 1), 2 * 1 + ((c >> 1) & 1), 2 * 1 + (c >> 2)] for c in range(8)], np.int32)
    ref, _ = oracle.deposit_octree(pos, n, leaves, bc, ml)
    m = gpu_octree_deposit(pos, n, leaves, bc, ml, prec, sched)
    e = cell_errors(m, ref)
    assert e["max_rel"] <= tol, e


def test_cube_subset_and_accumulate():
    n, bc, ml = 16, 4, 4
    pos = squeezed_lattice(n, seed=3)
    leaves, _ = oracle.build_octree(pos, n, bc, ml)
    ids = np.random.default_rng(0).permutation(n ** 3)
    a, b = np.sort(ids[:1000]), np.sort(ids[1000:])
    ref, _ = oracle.deposit_octree(pos, n, leaves, bc, ml)
    oct_ = pse.octree_from_leaves(leaves, bc, ml)
    dpos = torch.from_numpy(pos).cuda()
    out = pse.deposit_octree(dpos, n, oct_, cube_ids=torch.from_numpy(a).cuda())
    pse.deposit_octree(dpos, n, oct_, cube_ids=torch.from_numpy(b).cuda(), out=out, accumulate=True)
    e = cell_errors(out.cpu().numpy(), ref)
    assert e["max_rel"] <= 1e-5, e


def _tree_agreement(pos, n, bc, ml, threshold=2.0):
    got = pse.build_octree_from_tet_sizes(torch.from_numpy(pos).cuda(), n, bc, ml, threshold).leaves()
    exp, nodes = oracle.build_octree(pos, n, bc, ml, threshold_cells=threshold)
    near = [tuple(int(v) for v in r[:4]) for r in nodes
            if r[4] > 0 and r[0] < ml and threshold / BIN <= r[5] < threshold * BIN]
    return got, exp, near


@pytest.mark.parametrize("n,bc,ml", [(32, 4, 6), (32, 8, 6), (16, 4, 1)])
def test_build_undisplaced_closed_form(n, bc, ml):
    got, exp, near = _tree_agreement(lattice_positions(n), n, bc, ml)
    mean_edge = (3 + 2 * np.sqrt(2) + np.sqrt(3)) / 6 / n
    lev = 0
    while lev < ml and mean_edge < 2.0 / (bc * 2 ** lev):
        lev += 1
    assert set(got[:, 0].tolist()) == {lev}
    assert len(got) == 8 ** lev


def test_build_matches_oracle_away_from_threshold():
    n, bc, ml = 16, 4, 4
    pos = squeezed_lattice(n, seed=5)
    got, exp, near = _tree_agreement(pos, n, bc, ml)
    if not near:
        np.testing.assert_array_equal(got, exp)
    else:  # nodes within a bin of the threshold may go either way; everything else must match
        gs = {tuple(r) for r in got.tolist()}
        es = {tuple(r) for r in exp.tolist()}

        def under(leaf, node):
            return leaf[0] >= node[0] and all((leaf[1 + a] >> (leaf[0] - node[0])) == node[1 + a] for a in range(3))
        diff = gs ^ es
        assert all(any(under(l, nd) for nd in near) for l in diff), (diff, near)


def test_build_rejects_open_lattice_and_bad_args():
    pos = torch.from_numpy(lattice_positions(4)).cuda()
    with pytest.raises(pse.PseError):
        pse.octree_from_leaves(np.array([[1, 0, 0, 0]], np.int32), 4, 1)  # does not tile
    with pytest.raises(pse.PseError):
        pse.build_octree_from_tet_sizes(pos, 4, 4, 11)


def test_config3_full_size_sampled():
    """256^3 particles (100.7M tetrahedra), k^-1.5, rms 4 spacings, octree of 16^3 blocks, levels 0-4:
    GPU-built tree; the plain FP64 GPU path agrees with the oracle on 2048 random cubes deposited
    alone, and the FP32 path agrees with the FP64 path on every cell of the full deposit."""
    cfg = CONFIGS[3]
    pos = config_positions(cfg)
    dpos = torch.from_numpy(pos).cuda()
    oct_ = pse.build_octree_from_tet_sizes(dpos, cfg.n, cfg.bc, cfg.max_level, 2.0)
    leaves = oct_.leaves()
    # the leaves tile the box (with 16^3 blocks, 256^3 particles are ~1.3 finest cells apart,
    # so the size rule refines nearly everywhere down to level 4)
    assert sum(8.0 ** -int(l) for l in leaves[:, 0]) == pytest.approx(1.0, abs=1e-12)
    out, st = pse.deposit_octree(dpos, cfg.n, oct_, stats=True)
    assert st["tets"] == cfg.n_tets
    assert abs(float(out.sum()) - 1.0) <= 1e-12
    ids = np.sort(np.random.default_rng(33).choice(cfg.n ** 3, 2048, replace=False))
    ref, _ = oracle.deposit_octree(pos, cfg.n, leaves, cfg.bc, cfg.max_level, cube_ids=ids, nthreads=8)
    sub = pse.deposit_octree(dpos, cfg.n, oct_, cube_ids=torch.from_numpy(ids).cuda(),
                             precision=pse.PSE_FP64_PLAIN, schedule=pse.PSE_THREAD_PER_TET).cpu().numpy()
    # floor: 1e-3 of the mean occupied cell of the FULL deposit (the sample alone is sparse)
    full = out.cpu().numpy()
    e = cell_errors(sub, ref, floor_mass=1e-3 * full.sum() / np.count_nonzero(full))
    assert e["max_rel"] <= 1e-9, e
    full64 = pse.deposit_octree(dpos, cfg.n, oct_, precision=pse.PSE_FP64_PLAIN,
                                schedule=pse.PSE_THREAD_PER_TET).cpu().numpy()
    e = cell_errors(full, full64)
    assert e["max_rel"] <= 1e-5, e
    assert e["mass"] <= 1e-12, e


def test_octree_graph_replay():
    """use_graph on the octree deposit: replays equal plain calls, also after the positions change."""
    n, bc, ml = 16, 4, 4
    pos = torch.from_numpy(squeezed_lattice(n, seed=7)).cuda()
    oct_ = pse.build_octree_from_tet_sizes(pos, n, bc, ml, 2.0)
    ws = torch.empty(pse.workspace_size(pse._lib.PSE_OP_DEPOSIT_OCTREE), dtype=torch.uint8, device="cuda")
    out = torch.empty((oct_.n_leaves, bc, bc, bc), dtype=torch.float64, device="cuda")
    for seed in (7, 8):
        pos.copy_(torch.from_numpy(squeezed_lattice(n, seed=seed)))
        ref = pse.deposit_octree(pos, n, oct_).cpu().numpy()
        for _ in range(2):
            pse.deposit_octree(pos, n, oct_, out=out, workspace=ws, tuning={"use_graph": 1})
            e = cell_errors(out.cpu().numpy(), ref)
            assert e["max_rel"] <= 2e-6 and e["mass"] <= 1e-13, e


def test_restriction_equals_coarse_uniform_deposits():
    """Every node of levels 0..max_level-1 (pse_octree_restrict) holds the deposit on the
    uniform grid of its level restricted to the node; nodes below a leaf hold 0."""
    n, bc, ml = 16, 4, 4
    pos = squeezed_lattice(n)
    leaves, _ = oracle.build_octree(pos, n, bc, ml)
    assert len(set(leaves[:, 0].tolist())) > 1
    oct_ = pse.octree_from_leaves(leaves, bc, ml)
    m = pse.deposit_octree(torch.from_numpy(pos).cuda(), n, oct_, precision=pse.PSE_FP64_PLAIN,
                           schedule=pse.PSE_THREAD_PER_TET)
    pyr = pse.octree_restrict(oct_, m).cpu().numpy()
    row = 0
    for l in range(ml):
        nn = 2 ** l
        ref, _ = oracle.deposit_lattice(pos, n, bc * nn)
        floor = 1e-3 * ref.mean()
        for z in range(nn):
            for y in range(nn):
                for x in range(nn):
                    blk = pyr[row + x + nn * (y + nn * z)]
                    # where is this node: a leaf, an inner node, or below a coarser leaf?
                    below = any(L[0] < l and all((c >> (l - L[0])) == L[1 + a] for a, c in enumerate((x, y, z)))
                                for L in leaves)
                    if below:
                        assert not blk.any()
                        continue
                    r = ref[z * bc:(z + 1) * bc, y * bc:(y + 1) * bc, x * bc:(x + 1) * bc]
                    assert np.max(np.abs(blk - r) / np.maximum(r, floor)) <= 1e-9, (l, x, y, z)
        row += nn ** 3


def test_count_rule_build_matches_oracle():
    """The paper's count criterion on the GPU against the float64 restatement: identical
    leaves wherever no node's estimate lies within 1e-9 of the threshold."""
    n, bc, ml = 16, 4, 4
    for seed, thr in ((3, 600.0), (4, 100.0)):
        pos = squeezed_lattice(n, seed=seed)
        exp, est = oracle.build_octree_count(pos, n, bc, ml, count_threshold=thr, subblock=4)
        near = [k for k, v in est.items() if abs(v - thr) <= 1e-9 * thr]
        got = pse.build_octree_count(torch.from_numpy(pos).cuda(), n, bc, ml, thr, subblock=4).leaves()
        assert not near
        np.testing.assert_array_equal(got, exp)
        assert len(set(exp[:, 0].tolist())) > 1  # the squeezed region refines deeper


def test_collapsed_regions_give_an_adaptive_tree_and_match_the_oracle():
    """The collapsed-region input of workload 7 at a small size (4 finest cells per lattice
    spacing): the field's tetrahedra stop refining a level above the finest, the collapsed
    cores refine to the finest level, the GPU build agrees with the oracle away from the
    threshold, and the deposit on that mixed-level tree matches the oracle's."""
    from pse_inputs import collapse_positions
    n, bc, ml = 32, 8, 4
    pos = collapse_positions(zeldovich_positions(n, -2.0, 1.5 * (n / 256) ** 0.5, seed=1007), 8, 0.1, 0.16, 0.35,
                             1008)
    got, exp, near = _tree_agreement(pos, n, bc, ml)
    levels = np.bincount(got[:, 0], minlength=ml + 1)
    assert levels[ml] > 0 and levels[ml - 1] > 0, levels  # mixed levels
    gs, es = {tuple(r) for r in got.tolist()}, {tuple(r) for r in exp.tolist()}

    def under(leaf, node):
        return leaf[0] >= node[0] and all((leaf[1 + a] >> (leaf[0] - node[0])) == node[1 + a] for a in range(3))
    assert all(any(under(l, nd) for nd in near) for l in gs ^ es), (gs ^ es, near)
    ref, _ = oracle.deposit_octree(pos, n, got, bc, ml)
    m, st = gpu_octree_deposit(pos, n, got, bc, ml, pse.PSE_FP32_FP64ACC, pse.PSE_WARP_COOPERATIVE, stats=True)
    e = cell_errors(m, ref)
    assert e["max_rel"] <= 1e-5 and e["mass"] <= 1e-12, e
