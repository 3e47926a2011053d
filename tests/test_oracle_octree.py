"""Pins of the oracle's octree (adaptive deposit grid of Sec. 4): leaf tilings, the
coarsening identity against the pinned uniform deposit, and closed-form refinement
of the undisplaced lattice."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from pse_inputs import lattice_positions, zeldovich_positions


def coarsen_to_uniform(mass, leaves, bc, g):
    """Sum every leaf cell into the uniform grid of g cells per side (g <= bc at the coarsest leaf level)."""
    out = np.zeros((g, g, g))
    for l, (lev, ix, iy, iz) in enumerate(leaves):
        fine = bc * 2 ** lev              # cells per side at this leaf's level
        r = fine // g                     # leaf cells per uniform cell
        blk = mass[l]                     # [bc(z), bc(y), bc(x)]
        b = blk.reshape(bc // r, r, bc // r, r, bc // r, r).sum(axis=(1, 3, 5))
        o = np.array([ix, iy, iz]) * (bc // r)
        out[o[2]:o[2] + bc // r, o[1]:o[1] + bc // r, o[0]:o[0] + bc // r] += b
    return out


def test_single_root_leaf_equals_uniform_grid():
    n, bc = 8, 16
    pos = zeldovich_positions(n, -2.0, 1.0, seed=3)
    leaves = np.array([[0, 0, 0, 0]], np.int32)
    m, _ = oracle.deposit_octree(pos, n, leaves, bc, 0, nthreads=2)
    u, _ = oracle.deposit_lattice(pos, n, bc, nthreads=2)
    np.testing.assert_allclose(m[0], u, rtol=1e-13, atol=1e-19)


def test_fully_refined_tree_equals_fine_uniform_grid():
    n, bc, lev = 8, 4, 2
    pos = zeldovich_positions(n, -2.0, 1.0, seed=5)
    leaves = np.array([[lev, x, y, z] for z in range(4) for y in range(4) for x in range(4)], np.int32)
    m, _ = oracle.deposit_octree(pos, n, leaves, bc, lev, nthreads=2)
    u, _ = oracle.deposit_lattice(pos, n, bc * 2 ** lev, nthreads=2)
    np.testing.assert_allclose(coarsen_to_uniform(m, leaves, bc, bc * 2 ** lev), u, rtol=1e-12, atol=1e-19)


def squeezed_lattice(n, center=(0.25, 0.25, 0.25), radius=0.2, factor=0.3, jitter=0.0, seed=0):
    """Undisplaced lattice with a ball compressed by `factor` (small tetrahedra there)."""
    q = lattice_positions(n).astype(np.float64)
    c = np.asarray(center)
    d = q - c
    r = np.linalg.norm(d, axis=1, keepdims=True)
    p = np.where(r < radius, c + d * factor, q)
    if jitter:
        p = p + np.random.default_rng(seed).normal(0, jitter / n, p.shape)
    return np.mod(p, 1.0).astype(np.float32)


def test_mixed_tree_coarsens_to_uniform():
    """Any tree: summing leaf cells onto the coarsest common grid reproduces the uniform deposit."""
    n, bc = 16, 4
    pos = squeezed_lattice(n, jitter=0.2, seed=1)
    leaves, _ = oracle.build_octree(pos, n, bc, 4, threshold_cells=2.0)
    assert len(set(leaves[:, 0])) > 1  # genuinely adaptive
    m, st = oracle.deposit_octree(pos, n, leaves, bc, 4, nthreads=2)
    assert abs(m.sum() - 1.0) < 1e-13
    g = bc * 2 ** int(leaves[:, 0].min())
    u, _ = oracle.deposit_lattice(pos, n, g, nthreads=2)
    np.testing.assert_allclose(coarsen_to_uniform(m, leaves, bc, g), u, rtol=1e-11, atol=1e-18)


def test_leaves_tile_the_box():
    n, bc = 12, 8
    pos = zeldovich_positions(n, -1.5, 3.0, seed=9)
    leaves, nodes = oracle.build_octree(pos, n, bc, 4)
    vol = sum(8.0 ** -int(l[0]) for l in leaves)
    assert vol == pytest.approx(1.0, abs=1e-15)
    # depth-first order, children x fastest: a refined node is immediately followed by its first child
    refined = nodes[nodes[:, 6] == 1]
    assert len(refined) == sum(1 for _ in refined)


@pytest.mark.parametrize("n,bc,max_level", [(32, 4, 6), (32, 8, 6), (16, 4, 1)])
def test_undisplaced_lattice_refines_uniformly(n, bc, max_level):
    """Every Kuhn tetrahedron has mean edge (3 + 2 sqrt2 + sqrt3)/6 spacings: refinement stops at the
    first level l where that is >= 2 h_l, h_l = 1/(bc 2^l), or at max_level."""
    pos = lattice_positions(n)
    leaves, _ = oracle.build_octree(pos, n, bc, max_level, threshold_cells=2.0)
    mean_edge = (3 + 2 * np.sqrt(2) + np.sqrt(3)) / 6 / n
    lev = 0
    while lev < max_level and mean_edge < 2.0 / (bc * 2 ** lev):
        lev += 1
    assert set(leaves[:, 0].tolist()) == {lev}
    assert len(leaves) == 8 ** lev


def test_refinement_follows_small_tetrahedra():
    """A compressed region (small tetrahedra) is refined, the rest is not."""
    n, bc = 16, 4
    c = np.array([0.25, 0.25, 0.25])
    pos = squeezed_lattice(n, center=c)
    leaves, _ = oracle.build_octree(pos, n, bc, 4, threshold_cells=2.0)
    side = 1.0 / 2.0 ** leaves[:, 0]
    centers = (leaves[:, 1:] + 0.5) * side[:, None]
    deep = leaves[:, 0] == leaves[:, 0].max()
    assert np.all(np.linalg.norm(centers[deep] - c, axis=1) < 0.3)
    assert leaves[:, 0].max() > leaves[:, 0].min()


def test_bad_leaf_sets_are_rejected():
    pos = lattice_positions(4)
    with pytest.raises(RuntimeError):
        oracle.deposit_octree(pos, 4, np.array([[1, 0, 0, 0]], np.int32), 4, 1)  # does not tile
    with pytest.raises(RuntimeError):
        oracle.deposit_octree(pos, 4, np.array([[0, 0, 0, 0], [1, 0, 0, 0]], np.int32), 4, 1)  # overlaps


# ------------------------------------------------------------- count criterion (Sec. 4) --
def test_count_rule_root_estimate_is_every_tetrahedron():
    """Every subblock box lies inside the periodic root, so the root's estimate is 6 n^3."""
    n = 16
    pos = zeldovich_positions(n, -2.0, 1.0, seed=5)
    _, est = oracle.build_octree_count(pos, n, 4, 2, count_threshold=1e30, subblock=4)
    assert est[(0, 0, 0, 0)] == pytest.approx(6 * n ** 3, rel=1e-12)


@pytest.mark.parametrize("thr", [6 * 16 ** 3 / 8 - 1, 6 * 16 ** 3 / 64 - 1, 6 * 16 ** 3 / 64 + 1])
def test_count_rule_undisplaced_lattice_closed_form(thr):
    """Undisplaced lattice: the subblock boxes tile the box, so a node at level l is
    estimated at 6 n^3 / 8^l and the tree refines uniformly while that exceeds the threshold."""
    n, ml = 16, 4
    leaves, est = oracle.build_octree_count(lattice_positions(n), n, 4, ml, count_threshold=thr, subblock=4)
    for (l, x, y, z), v in est.items():
        assert v == pytest.approx(6 * n ** 3 / 8 ** l, rel=1e-12)
    lev = 0
    while lev < ml and 6 * n ** 3 / 8 ** lev > thr:
        lev += 1
    assert set(leaves[:, 0].tolist()) == {lev}
    assert len(leaves) == 8 ** lev


def test_large_tetrahedra_over_deep_tree_keep_every_leaf():
    """Eq. 1 on an octree: a tetrahedron covers every leaf its volume reaches, however many.
    A 3^3 lattice has tetrahedra a third of the box wide; on a tree refined to level 5 each
    one's bounding box spans about 11^3 finest nodes (over a thousand leaves).  Summed onto
    the finest uniform grid the leaves must give the uniform deposit, and the total mass 1."""
    n, bc, lev = 3, 2, 5
    pos = zeldovich_positions(n, -2.0, 0.3, seed=21)
    side = 2 ** lev
    leaves = np.array([[lev, x, y, z] for z in range(side) for y in range(side) for x in range(side)], np.int32)
    m, _ = oracle.deposit_octree(pos, n, leaves, bc, lev, nthreads=4)
    assert abs(m.sum() - 1.0) < 1e-12
    g = bc * side
    u, _ = oracle.deposit_lattice(pos, n, g, nthreads=4)
    np.testing.assert_allclose(coarsen_to_uniform(m, leaves, bc, g), u, rtol=1e-11, atol=1e-18)
