"""The per-cell error floor bench.py uses for sparse (sampled) deposits, on CPU tensors:
the Kuhn tetrahedra it forms from a lattice match the oracle's, and the vectorised floor
(the mass of a whole cell at the density of the densest tetrahedron whose bounding box
covers the cell) matches a plain loop over the tetrahedra."""
from __future__ import annotations

import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from pse_inputs.lattice import zeldovich_positions  # noqa: E402


def test_lattice_tets_match_oracle():
    n = 8
    pos = zeldovich_positions(n, -1.5, 1.5, seed=3)
    cubes = torch.tensor([0, 7, 63, 100, 511])
    v = bench.lattice_tets_cells(torch.from_numpy(pos), (n, n, n), cubes, 1.0, periodic=True).numpy()
    # the helper orders tetrahedra s-major: [s * len(cubes) + c]
    for s in range(6):
        for c, cube in enumerate(cubes.tolist()):
            ref = oracle.lattice_tet(pos, n, cube, s)
            np.testing.assert_allclose(v[s * len(cubes) + c], ref, rtol=0, atol=1e-12)


def test_density_floor_matches_loop():
    n, g = 6, 12
    pos = zeldovich_positions(n, -1.5, 1.0, seed=5)
    cubes = torch.arange(n ** 3)
    v = bench.lattice_tets_cells(torch.from_numpy(pos), (n, n, n), cubes, float(g), periodic=True)
    m_t = 1.0 / (6 * n ** 3)

    def index(ix, iy, iz):
        return (ix % g) + g * ((iy % g) + g * (iz % g))
    got = bench.density_floor_cells(v, m_t, index, g ** 3).numpy()
    ref = np.zeros(g ** 3)
    for t in v.numpy():
        vol = abs(np.linalg.det(t[1:] - t[0])) / 6.0
        lo, hi = np.floor(t.min(0)).astype(int), np.floor(t.max(0)).astype(int)
        for z in range(lo[2], hi[2] + 1):
            for y in range(lo[1], hi[1] + 1):
                for x in range(lo[0], hi[0] + 1):
                    k = (x % g) + g * ((y % g) + g * (z % g))
                    ref[k] = max(ref[k], m_t / vol)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    assert np.count_nonzero(ref) == g ** 3


class _FakeOctree:
    """Two levels of 4^3-cell leaf blocks: every leaf at level 1 (8^3 finest cells)."""
    bc, max_level = 4, 1

    def leaves(self):
        return np.array([(1, i, j, k) for k in range(2) for j in range(2) for i in range(2)], np.int32)


def test_octree_subset_floor_matches_global_floor():
    n, g = 4, 8
    pos = zeldovich_positions(n, -1.5, 1.0, seed=9)
    cubes = torch.tensor([0, 5, 21, 42, 63])
    oc = _FakeOctree()
    touched = torch.tensor([0, 3, 5, 6])
    got = bench.octree_subset_floor(torch.from_numpy(pos), n, cubes, oc, touched).reshape(len(touched), 4, 4, 4)
    v = bench.lattice_tets_cells(torch.from_numpy(pos), (n, n, n), cubes, float(g), periodic=True)
    full = bench.density_floor_cells(v, 1.0 / (6 * n ** 3), lambda x, y, z: (x % g) + g * ((y % g) + g * (z % g)),
                                     g ** 3).numpy().reshape(g, g, g)
    leaves = oc.leaves()
    for p, lf in enumerate(touched.tolist()):
        _, i, j, k = leaves[lf]
        np.testing.assert_array_equal(got[p], full[4 * k:4 * k + 4, 4 * j:4 * j + 4, 4 * i:4 * i + 4])
    assert np.count_nonzero(got) > 0
