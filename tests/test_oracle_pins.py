"""Pins of the FP64 CPU oracle against what the geometry and the paper fix.

Each test checks the oracle against something other than itself: a closed form,
an exact rational evaluation by a different algorithm, a symmetry, Monte Carlo,
or an invariant of Eq. 1 (mass conservation, partition of unity).  A plausible
slip anywhere in the oracle (a dropped prism piece, a wrong side of a plane, a
transposed axis, a missed periodic image) fails at least one of them.
"""
from __future__ import annotations

import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact
from pse_inputs import jitter_positions, lattice_positions, random_dyadic_tets, zeldovich_positions

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- P1 -------
def test_kuhn_simplex_worked_example():
    """The Kuhn simplex on unit cells: closed-form volumes from tests/golden."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "kuhn_simplex.txt")) if l.strip() and l[0] != "#"]
    expect = {(int(r[0]), int(r[1]), int(r[2])): int(r[3]) / int(r[4]) for r in rows}
    tet = np.array([[0, 0, 0], [0, 0, 2], [0, 2, 2], [2, 2, 2]], dtype=np.float64)
    cells, vols = oracle.tet_cells(tet, 1.0)
    got = {tuple(int(c) for c in cell): v for cell, v in zip(cells, vols)}
    assert set(got) == set(expect)
    for k, v in expect.items():
        assert got[k] == pytest.approx(v, abs=1e-15)


# ---------------------------------------------------------------- P2 -------
@pytest.mark.parametrize("n,g,offset", [(8, 8, 0.0), (8, 16, 0.0), (8, 4, 0.0), (8, 12, 0.0),
                                        (8, 5, 0.0), (8, 16, 0.5), (8, 9, 0.25)])
def test_undisplaced_lattice_is_uniform(n, g, offset):
    """Every tetrahedron of the undisplaced lattice has density exactly 1, so every cell gets 1/G^3."""
    pos = lattice_positions(n, offset=offset)
    m, st = oracle.deposit_lattice(pos, n, g, nthreads=2)
    assert st["degenerate_tets"] == 0
    np.testing.assert_allclose(m, 1.0 / g ** 3, rtol=1e-13, atol=0)


# ---------------------------------------------------------------- P3/P4 ----
def test_tet_inside_one_cell_deposits_there():
    g = 8
    h = 1.0 / g
    base = np.array([3, 2, 5]) * h
    tet = base + h * np.array([[0.1, 0.2, 0.3], [0.9, 0.15, 0.2], [0.3, 0.8, 0.25], [0.4, 0.4, 0.95]])
    m, st = oracle.deposit_tets(tet[None], 0.37, g)
    assert m[5, 2, 3] == pytest.approx(0.37, rel=1e-15)
    assert np.count_nonzero(m) == 1


def test_cell_inside_tet_gets_density_times_cell_volume():
    g = 16
    h = 1.0 / g
    tet = np.array([[0.05, 0.05, 0.05], [0.95, 0.1, 0.08], [0.1, 0.9, 0.1], [0.12, 0.11, 0.93]])
    vol = float(exact._vol(exact.tet_halfspaces([[Fraction(float(c)) for c in v] for v in tet]), 3))
    m, _ = oracle.deposit_tets(tet[None], 1.0, g)
    # cell (2,2,2) = [0.125,0.1875]^3 is deep inside this tetrahedron
    corners = np.array(list(itertools.product([2 * h, 3 * h], repeat=3)))
    # double-check containment with barycentric coordinates (independent of the oracle)
    T = np.column_stack([tet[1] - tet[0], tet[2] - tet[0], tet[3] - tet[0]])
    lam = np.linalg.solve(T, (corners - tet[0]).T)
    assert np.all(lam > 0) and np.all(lam.sum(axis=0) < 1)
    assert m[2, 2, 2] == pytest.approx(h ** 3 / vol, rel=1e-12)


# ---------------------------------------------------------------- P5 -------
@pytest.mark.parametrize("n,g,rms", [(16, 32, 0.5), (16, 16, 2.0), (12, 20, 1.5)])
def test_mass_conservation_periodic(n, g, rms):
    pos = zeldovich_positions(n, -2.0, rms, seed=7 + n)
    m, st = oracle.deposit_lattice(pos, n, g, nthreads=4)
    assert st["degenerate_tets"] == 0
    assert abs(m.sum() - 1.0) <= 1e-13
    assert np.all(m >= 0)


# ---------------------------------------------------------------- P6 -------
def test_partition_of_unity_per_tet():
    rng = np.random.default_rng(3)
    for t in range(40):
        tet = rng.uniform(-0.3, 0.3, size=(4, 3)) * rng.uniform(0.05, 1.0) + rng.uniform(0, 1, 3)
        h = rng.uniform(0.02, 0.2)
        _, vols = oracle.tet_cells(tet, h)
        ref = float(exact._vol(exact.tet_halfspaces([[Fraction(float(c)) for c in v] for v in tet]), 3))
        assert vols.sum() == pytest.approx(ref, rel=1e-12)


# ---------------------------------------------------------------- P7 -------
def test_exact_rational_lasserre_agrees():
    """Oracle (recursive split, FP64) vs exact rational Lasserre recursion on dyadic tetrahedra."""
    tets = random_dyadic_tets(12, seed=11, span=3.0, denom_bits=5, origin=0.0)
    nchecked = 0
    for tet in tets:
        ftet = [[Fraction(float(c)) for c in v] for v in tet]
        lo = np.floor(tet.min(axis=0)).astype(int)
        hi = np.floor(tet.max(axis=0)).astype(int)
        for ix in range(lo[0], hi[0] + 1):
            for iy in range(lo[1], hi[1] + 1):
                for iz in range(lo[2], hi[2] + 1):
                    c = (ix, iy, iz)
                    ex = exact.tet_box_volume(ftet, c, tuple(x + 1 for x in c))
                    got = oracle.tet_box_volume(tet, c, [x + 1 for x in c])
                    assert abs(got - float(ex)) <= 1e-14, (tet, c, got, float(ex))
                    nchecked += 1
    assert nchecked > 50


def test_lasserre_textbook_values():
    """The checker itself: unit cube, and the Kuhn simplex, by Lasserre."""
    cube = exact._vol(exact.box_halfspaces([0, 0, 0], [1, 1, 1]), 3)
    assert cube == 1
    kuhn = [[0, 0, 0], [0, 0, 2], [0, 2, 2], [2, 2, 2]]
    assert exact._vol(exact.tet_halfspaces([[Fraction(c) for c in v] for v in kuhn]), 3) == Fraction(4, 3)
    assert exact.tet_box_volume(kuhn, (0, 0, 1), (1, 1, 2)) == Fraction(1, 2)


# ---------------------------------------------------------------- P8 -------
def test_inclusion_exclusion_over_orthants():
    """vol(T ∩ box) = sum over box corners of ±vol(T ∩ orthant) (3-plane clips only)."""
    rng = np.random.default_rng(5)
    for _ in range(30):
        tet = rng.uniform(0, 2, size=(4, 3))
        lo = rng.uniform(0.2, 0.9, 3)
        hi = lo + rng.uniform(0.2, 0.9, 3)
        six = oracle.tet_box_volume(tet, lo, hi)
        acc = 0.0
        for bits in itertools.product([0, 1], repeat=3):
            corner = [hi[a] if bits[a] else lo[a] for a in range(3)]
            sign = (-1) ** (3 - sum(bits))
            acc += sign * oracle.tet_halfspaces_volume(tet, [(a, 1, corner[a]) for a in range(3)])
        assert six == pytest.approx(acc, abs=1e-12)


# ---------------------------------------------------------------- P9 -------
def test_monte_carlo_fractions():
    rng = np.random.default_rng(9)
    tet = np.array([[0.11, 0.07, 0.13], [0.83, 0.21, 0.09], [0.27, 0.71, 0.31], [0.35, 0.29, 0.88]])
    h = 0.25
    cells, vols = oracle.tet_cells(tet, h)
    ns = 10_000_000
    # uniform points in the tetrahedron: sorted-uniform barycentric coordinates
    u = np.sort(rng.random((ns, 3)), axis=1)
    bary = np.column_stack([u[:, 0], u[:, 1] - u[:, 0], u[:, 2] - u[:, 1], 1 - u[:, 2]])
    pts = bary @ tet
    idx = np.floor(pts / h).astype(np.int64)
    keys = (idx[:, 0] * 1000 + idx[:, 1]) * 1000 + idx[:, 2]
    uk, cnt = np.unique(keys, return_counts=True)
    mc = dict(zip(uk.tolist(), cnt.tolist()))
    V = vols.sum()
    for cell, v in zip(cells, vols):
        k = (int(cell[0]) * 1000 + int(cell[1])) * 1000 + int(cell[2])
        p = v / V
        sigma = np.sqrt(p * (1 - p) / ns)
        assert abs(mc.get(k, 0) / ns - p) <= 4 * sigma + 1e-12


# ---------------------------------------------------------------- P10 ------
def test_translation_by_whole_cells_is_exact_shift():
    n, g = 8, 16
    pos = zeldovich_positions(n, -2.0, 0.4, seed=21).astype(np.float64)
    pos = (np.round(pos * 2 ** 20) / 2 ** 20) % 1.0  # coarse dyadic values: the shift below is exact
    m0, _ = oracle.deposit_lattice(pos.astype(np.float32), n, g, nthreads=1)
    shift = np.array([3, 5, 7]) / g
    pos2 = np.mod(pos + shift, 1.0)
    assert np.all(pos2.astype(np.float32).astype(np.float64) == pos2)
    m1, _ = oracle.deposit_lattice(pos2.astype(np.float32), n, g, nthreads=1)
    expect = np.roll(m0, shift=(7, 5, 3), axis=(0, 1, 2))
    np.testing.assert_allclose(m1, expect, rtol=1e-12, atol=1e-18)


def test_axis_permutation_symmetry():
    """Swapping x and y of every particle (and the lattice axes) transposes the grid."""
    n, g = 8, 12
    pos = zeldovich_positions(n, -2.0, 1.0, seed=23)
    m0, _ = oracle.deposit_lattice(pos, n, g, nthreads=1)
    # new lattice index (i', j', k) = (j, i, k): reorder particles and swap coordinates
    p3 = pos.reshape(n, n, n, 3)  # [k, j, i, a]
    q3 = np.transpose(p3, (0, 2, 1, 3))[..., [1, 0, 2]]
    m1, _ = oracle.deposit_lattice(np.ascontiguousarray(q3.reshape(-1, 3)), n, g, nthreads=1)
    # the Kuhn split is symmetric as a set under any axis permutation, so the deposit is too
    np.testing.assert_allclose(m1, np.transpose(m0, (0, 2, 1)), rtol=1e-11, atol=1e-18)


# ---------------------------------------------------------------- P11 ------
def test_one_plane_truncated_power_formula():
    """vol(T ∩ {x_a <= s}) = V * sum_i (s - x_i)_+^3 / prod_{j != i} (x_j - x_i)."""
    rng = np.random.default_rng(13)
    for _ in range(60):
        tet = rng.uniform(0, 1, size=(4, 3))
        V = oracle.tet_volume(tet)
        for a in range(3):
            x = tet[:, a]
            for s in rng.uniform(x.min() - 0.05, x.max() + 0.05, 3):
                ref = 0.0
                for i in range(4):
                    den = np.prod([x[j] - x[i] for j in range(4) if j != i])
                    ref += max(s - x[i], 0.0) ** 3 / den
                ref *= V
                got_below = oracle.tet_halfspaces_volume(tet, [(a, 1, s)])
                got_above = oracle.tet_halfspaces_volume(tet, [(a, 0, s)])
                assert got_below == pytest.approx(ref, abs=1e-12)
                assert got_above == pytest.approx(V - ref, abs=1e-12)


# ---------------------------------------------------------------- P12 ------
def test_paper_jitter_distribution_conserves_mass():
    """The weak-scaling input of Sec. 7.2: lattice + uniform offsets of up to one spacing."""
    n, g = 12, 24
    pos = jitter_positions(n, seed=31, amp=1.0)
    m, st = oracle.deposit_lattice(pos, n, g, nthreads=4)
    assert abs(m.sum() - 1.0) <= 1e-13
    assert np.all(m >= 0)


# ---------------------------------------------------------------- edge cases
def test_degenerate_tet_goes_to_centroid_cell():
    g = 4
    tet = np.array([[0.1, 0.1, 0.3], [0.6, 0.1, 0.3], [0.1, 0.6, 0.3], [0.35, 0.35, 0.3]])  # flat: z = 0.3
    m, st = oracle.deposit_tets(tet[None], 0.5, g)
    assert st["degenerate_tets"] == 1
    c = (tet.mean(axis=0) * g).astype(int)
    assert m[c[2], c[1], c[0]] == pytest.approx(0.5)
    assert np.count_nonzero(m) == 1


def test_periodic_wrap_equals_shifted_deposit():
    g = 8
    tet = np.array([[0.95, 0.40, 0.40], [1.10, 0.42, 0.45], [0.97, 0.60, 0.41], [1.02, 0.45, 0.62]])
    m, _ = oracle.deposit_tets(tet[None], 1.0, g, periodic=True)
    m2, _ = oracle.deposit_tets((tet - [0.5, 0, 0])[None], 1.0, g, periodic=True)
    np.testing.assert_allclose(m, np.roll(m2, 4, axis=2), rtol=1e-12, atol=1e-16)
    assert m.sum() == pytest.approx(1.0, abs=1e-14)
    assert m[..., 7].sum() > 0 and m[..., 0].sum() > 0


def test_open_boundary_loses_outside_mass():
    g = 8
    tet = np.array([[0.95, 0.40, 0.40], [1.10, 0.42, 0.45], [0.97, 0.60, 0.41], [1.02, 0.45, 0.62]])
    m, st = oracle.deposit_tets(tet[None], 1.0, g, periodic=False)
    assert m.sum() + st["lost_mass"] == pytest.approx(1.0, abs=1e-14)
    assert st["lost_mass"] > 0


def test_lattice_tets_tile_each_cube():
    """The 6 Kuhn tetrahedra of a cube have volume cube/6 each and fill it (undisplaced)."""
    n = 4
    pos = lattice_positions(n)
    for cube in (0, 5, 63):
        vols = [oracle.tet_volume(oracle.lattice_tet(pos, n, cube, s)) for s in range(6)]
        np.testing.assert_allclose(vols, (1 / n) ** 3 / 6, rtol=1e-14)


def test_thread_count_does_not_change_result():
    n, g = 12, 24
    pos = zeldovich_positions(n, -2.0, 2.0, seed=41)
    m1, _ = oracle.deposit_lattice(pos, n, g, nthreads=1)
    m4, _ = oracle.deposit_lattice(pos, n, g, nthreads=4)
    np.testing.assert_allclose(m1, m4, rtol=1e-13, atol=1e-19)


def test_cube_subset_sums_to_whole():
    n, g = 8, 16
    pos = zeldovich_positions(n, -2.0, 1.0, seed=43)
    full, _ = oracle.deposit_lattice(pos, n, g, nthreads=2)
    ids = np.arange(n ** 3)
    a, _ = oracle.deposit_lattice(pos, n, g, cube_ids=ids[::2], nthreads=2)
    b, _ = oracle.deposit_lattice(pos, n, g, cube_ids=ids[1::2], nthreads=2)
    np.testing.assert_allclose(a + b, full, rtol=1e-12, atol=1e-19)
