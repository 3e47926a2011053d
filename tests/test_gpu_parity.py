"""Parity of the CUDA deposit (through the C ABI) with the FP64 CPU oracle.

Tolerances (the C13 measures of paper_1612_09491_gb300.metrics):
  * FP64 plain path:     max_rel <= 1e-9 (different clip algorithm, both float64; sliver
                         tetrahedra amplify float64 rounding on both sides);
  * FP32 + FP64-redo:    max_rel <= 1e-5 per cell, total mass <= 1e-12 relative.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1612_09491_gb300 as pse  # noqa: E402
from paper_1612_09491_gb300.metrics import cell_errors  # noqa: E402
from pse_inputs import (CONFIGS, config_positions, jitter_positions, lattice_positions,  # noqa: E402
                        random_dyadic_tets, zeldovich_positions)

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32 = 1e-5
MASS32 = 1e-12
# Isolated tetrahedra and cube subsets leave cells that hold only a sliver of one
# tetrahedron.  A clip's FP32 rounding is a fraction of a FULL cell at that
# tetrahedron's density, however thin the sliver, so sparse cases are measured against
# the per-cell floor of density_floor() (same TOL32).

PATHS = [
    ("fp64-thread", pse.PSE_FP64_PLAIN, pse.PSE_THREAD_PER_TET),
    ("fp32-thread", pse.PSE_FP32_FP64ACC, pse.PSE_THREAD_PER_TET),
    ("fp32-warp", pse.PSE_FP32_FP64ACC, pse.PSE_WARP_COOPERATIVE),
    ("fp32-binned", pse.PSE_FP32_FP64ACC, "binned"),
    ("fp32-warp-per-tet", pse.PSE_FP32_FP64ACC, pse.PSE_WARP_PER_TET),
    ("fp32c-warp", pse.PSE_FP32_COMPENSATED, pse.PSE_WARP_COOPERATIVE),
    ("fp32c-binned", pse.PSE_FP32_COMPENSATED, "binned"),
]
# the binned schedule with tiny thresholds, so that small cases go through the split
# work items (every tetrahedron with more than 4 bounding-box cells, 8 cells per item)
SPLIT_TUNING = {"split_cells": 4, "chunk_cells": 8}


def sched_kw(sched):
    if sched == "binned":
        return {"schedule": pse.PSE_BINNED_PERSISTENT, "tuning": SPLIT_TUNING}
    return {"schedule": sched}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1612_09491_gb300 import build
    build.build()
    pse._lib.load()
    yield


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_lattice(pos, n, g, prec, sched, **kw):
    out = pse.deposit_uniform(dev(pos), n, g, precision=prec, **sched_kw(sched), **kw)
    if isinstance(out, tuple):
        return out[0].cpu().numpy(), out[1]
    return out.cpu().numpy()


def gpu_tets(verts, mass, g, prec, sched, **kw):
    out = pse.deposit_tets(dev(np.asarray(verts, np.float32)), dev(np.asarray(mass, np.float64)), g,
                           precision=prec, **sched_kw(sched), **kw)
    if isinstance(out, tuple):
        return out[0].cpu().numpy(), out[1]
    return out.cpu().numpy()


def tol_for(prec):
    return TOL64 if prec == pse.PSE_FP64_PLAIN else TOL32


def density_floor(tets, mass, g):
    """Per cell: the mass of a whole cell at the density of the densest tetrahedron whose
    bounding box covers it ([z, y, x] like the deposit; periodic box of side 1)."""
    f = np.zeros((g, g, g))
    for t, m in zip(np.asarray(tets, np.float64), np.asarray(mass, np.float64)):
        v = t * g
        vol = abs(np.linalg.det(v[1:] - v[0])) / 6.0
        if vol == 0.0:
            continue
        lo = np.floor(v.min(0)).astype(int)
        hi = np.floor(v.max(0)).astype(int)
        ix, iy, iz = (np.arange(lo[a], hi[a] + 1) % g for a in range(3))
        blk = np.ix_(iz, iy, ix)
        f[blk] = np.maximum(f[blk], m / vol)
    return f


def subset_tets(pos, n, ids):
    return np.array([oracle.lattice_tet(pos, n, int(c), s) for c in ids for s in range(6)])


def f32(a):
    """Coordinates as the GPU sees them: rounded to float32 (the oracle gets the same values)."""
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def explain(tets, mass, g, prec, sched, e):
    """Failure message: the tetrahedron whose lone deposit disagrees most with the oracle."""
    worst = (-1.0, -1, None)
    for t in range(len(tets)):
        r, _ = oracle.deposit_tets(tets[t:t + 1], mass[t:t + 1], g)
        m, st = gpu_tets(tets[t:t + 1], mass[t:t + 1], g, prec, sched, stats=True)
        d = float(np.abs(m - r).max() / max(np.abs(r).max(), 1e-300))
        if d > worst[0]:
            worst = (d, t, st)
    t = worst[1]
    return f"{e}; worst tet {t} rel {worst[0]:.3g} verts {tets[t].tolist()} stats {worst[2]}"


# ------------------------------------------------------------ closed forms --
@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_kuhn_simplex(name, prec, sched):
    tet = np.array([[[0, 0, 0], [0, 0, 2], [0, 2, 2], [2, 2, 2]]], dtype=np.float32) / 2.0  # box 1, grid 2
    m = gpu_tets(tet, [1.0], 2, prec, sched)
    expect = np.zeros((2, 2, 2))
    for (ix, iy, iz), v in {(0, 0, 0): 1 / 6, (0, 0, 1): 1 / 2, (0, 1, 1): 1 / 2, (1, 1, 1): 1 / 6}.items():
        expect[iz, iy, ix] = v * 0.75  # mass 1 over volume 4/3 (cell units)
    np.testing.assert_allclose(m, expect, rtol=0, atol=1e-7 if prec else 1e-15)


@pytest.mark.parametrize("name,prec,sched", PATHS)
@pytest.mark.parametrize("n,g,offset", [(8, 8, 0.0), (8, 16, 0.0), (8, 4, 0.0), (16, 24, 0.0), (8, 5, 0.0),
                                        (8, 16, 0.5), (16, 32, 0.25)])
def test_undisplaced_lattice_uniform(name, prec, sched, n, g, offset):
    """Every vertex on cell planes: the degenerate worst case; must stay exactly uniform."""
    pos = lattice_positions(n, offset=offset)
    m, st = gpu_lattice(pos, n, g, prec, sched, stats=True)
    tol = 1e-13 if prec == pse.PSE_FP64_PLAIN else 1e-6
    np.testing.assert_allclose(m, 1.0 / g ** 3, rtol=tol, atol=0)
    assert st["tets"] == 6 * n ** 3


@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_tet_inside_one_cell(name, prec, sched):
    g = 8
    h = 1.0 / g
    tet = f32((np.array([3, 2, 5]) * h + h * np.array([[0.1, 0.2, 0.3], [0.9, 0.15, 0.2], [0.3, 0.8, 0.25],
                                                       [0.4, 0.4, 0.95]]))[None])
    m = gpu_tets(tet, [0.37], g, prec, sched)
    assert m[5, 2, 3] == pytest.approx(0.37, rel=1e-15)
    assert np.count_nonzero(m) == 1


@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_cell_inside_tet(name, prec, sched):
    g = 16
    tet = f32([[[0.05, 0.05, 0.05], [0.95, 0.1, 0.08], [0.1, 0.9, 0.1], [0.12, 0.11, 0.93]]])
    ref, _ = oracle.deposit_tets(tet, [1.0], g)
    # rho * h^3 (the FP32 path's global mass rescale is off here; its warp kernels form the
    # deposit in float32, so "exactly" means to float32 rounding there)
    m = gpu_tets(tet, [1.0], g, prec, sched, mass_fixup=False)
    exact_rel = 1e-12 if (prec == pse.PSE_FP64_PLAIN or sched == pse.PSE_THREAD_PER_TET) else 1.2e-7
    assert m[2, 2, 2] == pytest.approx(ref[2, 2, 2], rel=exact_rel)
    m = gpu_tets(tet, [1.0], g, prec, sched)
    e = cell_errors(m, ref, floor_mass=density_floor(tet, [1.0], g))
    assert e["max_rel"] <= tol_for(prec), e


@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_degenerate_tet_centroid_rule(name, prec, sched):
    tet = np.array([[[0.1, 0.1, 0.3], [0.6, 0.1, 0.3], [0.1, 0.6, 0.3], [0.35, 0.35, 0.3]]], dtype=np.float32)
    m, st = gpu_tets(tet, [0.5], 4, prec, sched, stats=True)
    ref, _ = oracle.deposit_tets(tet.astype(np.float64), [0.5], 4)
    np.testing.assert_array_equal(m, ref)
    assert st["degenerate_tets"] == 1


# ------------------------------------------------------------ vs the oracle --
@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_random_dyadic_tets(name, prec, sched):
    tets = f32(random_dyadic_tets(300, seed=5, span=0.45, denom_bits=9, origin=0.05))
    mass = np.random.default_rng(1).uniform(0.5, 2.0, len(tets))
    ref, _ = oracle.deposit_tets(tets, mass, 16)
    m = gpu_tets(tets, mass, 16, prec, sched)
    e = cell_errors(m, ref, floor_mass=density_floor(tets, mass, 16))
    assert e["max_rel"] <= tol_for(prec), explain(tets, mass, 16, prec, sched, e)
    assert e["mass"] <= (1e-13 if prec == pse.PSE_FP64_PLAIN else MASS32), e


@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_large_and_sliver_tets(name, prec, sched):
    rng = np.random.default_rng(17)
    big = rng.uniform(0.2, 0.8, size=(6, 4, 3))                      # spans ~20 cells per axis at g=32
    base = rng.uniform(0.3, 0.7, size=(20, 1, 3))
    sl = base + rng.normal(0, 0.02, size=(20, 4, 3)) * np.array([1, 1, 1e-3])  # flat slivers
    tets = f32(np.concatenate([big, sl]))
    mass = np.ones(len(tets))
    ref, _ = oracle.deposit_tets(tets, mass, 32)
    m = gpu_tets(tets, mass, 32, prec, sched)
    e = cell_errors(m, ref, floor_mass=density_floor(tets, mass, 32))
    assert e["max_rel"] <= tol_for(prec), explain(tets, mass, 32, prec, sched, e)
    assert e["mass"] <= (1e-11 if prec == pse.PSE_FP64_PLAIN else MASS32), e  # FP64 slivers: both sides ~1e-12


@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_config1_full(name, prec, sched):
    """32^3 particles (196,608 tetrahedra), k^-2, rms 0.5 spacings, 64^3 grid: every cell."""
    cfg = CONFIGS[1]
    pos = config_positions(cfg)
    ref, _ = oracle.deposit_lattice(pos, cfg.n, cfg.grid_n)
    m, st = gpu_lattice(pos, cfg.n, cfg.grid_n, prec, sched, stats=True)
    e = cell_errors(m, ref)
    assert e["max_rel"] <= tol_for(prec), e
    assert e["mass"] <= (1e-13 if prec == pse.PSE_FP64_PLAIN else MASS32), e
    assert st["tets"] == cfg.n_tets
    assert abs(st["mass_in"] - 1.0) < 1e-12


@pytest.mark.parametrize("tuning", [None, SPLIT_TUNING, {"split_cells": 64, "chunk_cells": 1000}])
def test_binned_counts_match_warp_cooperative(tuning):
    """The binned schedule visits exactly the pairs of the warp-cooperative one (the counters
    are deterministic), whatever its split thresholds.  The masses agree to FP32 rounding:
    the two kernels are compiled separately and may fuse multiply-adds differently."""
    cfg = CONFIGS[1]
    dpos = dev(config_positions(cfg))
    a, sa = pse.deposit_uniform(dpos, cfg.n, cfg.grid_n, schedule=pse.PSE_WARP_COOPERATIVE, stats=True)
    b, sb = pse.deposit_uniform(dpos, cfg.n, cfg.grid_n, schedule=pse.PSE_BINNED_PERSISTENT, tuning=tuning,
                                stats=True)
    for k in ("tets", "bbox_cells", "inside_cells", "partial_clips", "fp64_redos", "single_cell_tets",
              "bin_counts"):
        assert sa[k] == sb[k], k
    e = cell_errors(b.cpu().numpy(), a.cpu().numpy())
    assert e["max_rel"] <= 2e-6, e
    assert e["mass"] <= 1e-13, e


def test_binned_graph_replay():
    """use_graph: the launch sequence is captured once per argument set and replayed; replays
    read the current contents of the buffers, and other arguments capture a new graph."""
    n, g = 16, 32
    p1 = dev(zeldovich_positions(n, -2.0, 1.5, seed=21))
    p2 = zeldovich_positions(n, -2.0, 1.5, seed=22)
    ws = torch.empty(pse.workspace_size(schedule=pse.PSE_BINNED_PERSISTENT), dtype=torch.uint8, device="cuda")
    tu = dict(SPLIT_TUNING, use_graph=1)
    plain = lambda pos: pse.deposit_uniform(pos, n, g, schedule=pse.PSE_BINNED_PERSISTENT,
                                            tuning=SPLIT_TUNING).cpu().numpy()
    out = torch.empty((g, g, g), dtype=torch.float64, device="cuda")
    ref1 = plain(p1)
    for _ in range(3):
        pse.deposit_uniform(p1, n, g, out=out, workspace=ws, schedule=pse.PSE_BINNED_PERSISTENT, tuning=tu)
        assert cell_errors(out.cpu().numpy(), ref1)["max_rel"] <= 1e-12
    p1.copy_(torch.from_numpy(p2))  # same pointer, new contents
    pse.deposit_uniform(p1, n, g, out=out, workspace=ws, schedule=pse.PSE_BINNED_PERSISTENT, tuning=tu)
    assert cell_errors(out.cpu().numpy(), plain(p1))["max_rel"] <= 1e-12
    out2 = torch.empty_like(out)  # another output buffer: another graph
    pse.deposit_uniform(p1, n, g, out=out2, workspace=ws, schedule=pse.PSE_BINNED_PERSISTENT, tuning=tu)
    assert cell_errors(out2.cpu().numpy(), plain(p1))["max_rel"] <= 1e-12


@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_shell_crossed_small(name, prec, sched):
    """Strong shell crossing (rms 3 spacings, many inverted and sliver tetrahedra), 16^3 particles."""
    n, g = 16, 48
    pos = zeldovich_positions(n, -1.5, 3.0, seed=77)
    ref, _ = oracle.deposit_lattice(pos, n, g)
    m = gpu_lattice(pos, n, g, prec, sched)
    e = cell_errors(m, ref)
    assert e["max_rel"] <= tol_for(prec), e
    assert e["mass"] <= (1e-13 if prec == pse.PSE_FP64_PLAIN else MASS32), e


@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_paper_jitter_input(name, prec, sched):
    n, g = 16, 32
    pos = jitter_positions(n, seed=3, amp=1.0)
    ref, _ = oracle.deposit_lattice(pos, n, g)
    m = gpu_lattice(pos, n, g, prec, sched)
    e = cell_errors(m, ref)
    assert e["max_rel"] <= tol_for(prec), e


@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_ragged_noncubic_lattice_and_grid(name, prec, sched):
    """Row lengths that are not multiples of 32, anisotropic lattice and grid."""
    n = (37, 6, 9)
    rng = np.random.default_rng(4)
    q = np.stack(np.meshgrid(*[np.arange(k) / k for k in n[::-1]], indexing="ij")[::-1], -1).reshape(-1, 3)
    pos = np.mod(q + rng.normal(0, 0.3, q.shape) / np.array(n), 1.0).astype(np.float32)
    g = (40, 12, 10)
    ref, _ = oracle.deposit_lattice(pos, n, g)
    m = gpu_lattice(pos, n, g, prec, sched)
    e = cell_errors(m, ref)
    assert e["max_rel"] <= tol_for(prec), e


@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_open_lattice_and_grid(name, prec, sched):
    n, g = 12, 20
    pos = zeldovich_positions(n, -2.0, 0.8, seed=9)
    ref, rst = oracle.deposit_lattice(pos, n, g, periodic=False)
    m, st = gpu_lattice(pos, n, g, prec, sched, periodic=False, stats=True)
    # cells at the open boundary are partly covered: per-cell density floor
    tets = np.array([oracle.lattice_tet(pos, n, c, s, periodic=False) for c in range((n - 1) ** 3) for s in range(6)])
    e = cell_errors(m, ref, floor_mass=density_floor(tets, np.full(len(tets), 1.0 / (6 * n ** 3)), g))
    assert e["max_rel"] <= tol_for(prec), e
    inner = (slice(3, g - 3),) * 3
    e = cell_errors(m[inner], ref[inner])
    assert e["max_rel"] <= tol_for(prec), e
    assert st["tets"] == 6 * (n - 1) ** 3
    assert st["mass_dropped"] == pytest.approx(rst["lost_mass"], rel=1e-6, abs=1e-15)


@pytest.mark.parametrize("name,prec,sched", PATHS)
def test_cube_subset_and_accumulate(name, prec, sched):
    n, g = 16, 32
    pos = zeldovich_positions(n, -2.0, 1.0, seed=12)
    ids = np.random.default_rng(2).permutation(n ** 3)
    a_ids, b_ids = np.sort(ids[: n ** 3 // 3]), np.sort(ids[n ** 3 // 3:])
    ref_a, _ = oracle.deposit_lattice(pos, n, g, cube_ids=a_ids)
    ref, _ = oracle.deposit_lattice(pos, n, g)
    dpos = dev(pos)
    out = pse.deposit_uniform(dpos, n, g, precision=prec, **sched_kw(sched), cube_ids=dev(a_ids))
    fl = density_floor(subset_tets(pos, n, a_ids), np.full(6 * len(a_ids), 1.0 / (6 * n ** 3)), g)
    e = cell_errors(out.cpu().numpy(), ref_a, floor_mass=fl)
    assert e["max_rel"] <= tol_for(prec), e
    if prec == pse.PSE_FP32_COMPENSATED:  # the float pairs start from a cleared output
        with pytest.raises(pse.PseError):
            pse.deposit_uniform(dpos, n, g, precision=prec, **sched_kw(sched), cube_ids=dev(b_ids), out=out,
                                accumulate=True)
        return
    pse.deposit_uniform(dpos, n, g, precision=prec, **sched_kw(sched), cube_ids=dev(b_ids), out=out,
                        accumulate=True)
    e = cell_errors(out.cpu().numpy(), ref)
    assert e["max_rel"] <= tol_for(prec), e


def test_empty_inputs():
    out = pse.deposit_tets(torch.zeros((0, 4, 3), dtype=torch.float32, device="cuda"),
                           torch.zeros((0,), dtype=torch.float64, device="cuda"), 8)
    assert float(out.abs().sum()) == 0.0
    out = pse.deposit_uniform(dev(lattice_positions(4)), 4, 4, cube_ids=torch.zeros((0,), dtype=torch.int64,
                                                                                      device="cuda"))
    assert float(out.abs().sum()) == 0.0


def test_bad_cube_id_is_reported_not_read():
    pos = dev(lattice_positions(4))
    with pytest.raises(pse.PseError) as ei:
        pse.deposit_uniform(pos, 4, 8, cube_ids=dev(np.array([0, 5, 64, 3], np.int64)), stats=True)
    assert ei.value.code == -7


def test_caller_workspace():
    n, g = 8, 16
    pos = dev(zeldovich_positions(n, -2.0, 1.0, seed=1))
    ws = torch.empty(pse.workspace_size(), dtype=torch.uint8, device="cuda")
    a = pse.deposit_uniform(pos, n, g, workspace=ws)
    b = pse.deposit_uniform(pos, n, g)
    e = cell_errors(a.cpu().numpy(), b.cpu().numpy())
    assert e["max_rel"] <= 1e-12
    with pytest.raises(pse.PseError):
        pse.deposit_uniform(pos, n, g, workspace=ws[:8])


def test_build_tets_matches_tessellation():
    n = 6
    pos = zeldovich_positions(n, -2.0, 1.0, seed=8)
    vidx, vol = pse.build_tets_from_lagrangian_grid(dev(pos), n)
    vidx, vol = vidx.cpu().numpy(), vol.cpu().numpy()
    assert vidx.shape == (6 * n ** 3, 4)
    for t in (0, 1, 5, 17, 6 * n ** 3 - 1):
        tet = oracle.lattice_tet(pos, n, t // 6, t % 6)
        assert abs(vol[t]) == pytest.approx(oracle.tet_volume(tet), rel=1e-5)
        # the vertices are the particles named by vidx, unwrapped to the image nearest vertex 0
        p = pos[vidx[t]].astype(np.float64)
        d = p - p[0]
        d -= np.floor(d + 0.5)
        np.testing.assert_allclose(p[0] + d, tet, atol=1e-7)


# ------------------------------------------------------------ full size ---
def candidate_cubes(pos, n, cells, g, slab=None):
    """Cubes whose (unwrapped) corner bounding box touches any of the given cells
    (z-slabs of `slab` cube layers at a time for large lattices)."""
    if slab is not None and slab < n:
        p = pos.reshape(n, n, n, 3)
        out = []
        for k0 in range(0, n, slab):
            k1 = min(n, k0 + slab)
            rows = np.concatenate([p[k0:k1], p[k1 % n:k1 % n + 1]], 0).astype(np.float64)  # + halo row
            corners = []
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        c = np.roll(rows[dz:dz + (k1 - k0)], shift=(-dy, -dx), axis=(1, 2))
                        d = c - rows[:k1 - k0]
                        d -= np.floor(d + 0.5)
                        corners.append(rows[:k1 - k0] + d)
            cs = np.stack(corners, 0)
            lo = np.floor(cs.min(0) * g).astype(np.int64)
            ext = np.floor(cs.max(0) * g).astype(np.int64) - lo
            sel = np.zeros(lo.shape[:3], bool)
            for c in cells:
                sel |= np.all(np.mod(np.asarray(c) - lo, g) <= ext, axis=-1)
            kk, jj, ii = np.nonzero(sel)
            out.append(ii + n * (jj + n * (kk + k0)))
        return np.sort(np.concatenate(out))
    p = pos.reshape(n, n, n, 3).astype(np.float64)
    corners = []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                c = np.roll(p, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
                d = c - p
                d -= np.floor(d + 0.5)
                corners.append(p + d)
    cs = np.stack(corners, 0)  # [8, n, n, n, 3]
    lo = np.floor(cs.min(0) * g).astype(np.int64)
    ext = np.floor(cs.max(0) * g).astype(np.int64) - lo
    sel = np.zeros((n, n, n), bool)
    for c in cells:
        # periodic containment: (c - lo) mod g <= extent on every axis
        sel |= np.all(np.mod(np.asarray(c) - lo, g) <= ext, axis=-1)
    kk, jj, ii = np.nonzero(sel)
    return np.sort(ii + n * (jj + n * kk))


def test_config2_full_size_sampled_cells():
    """128^3 particles (12.6M tetrahedra) onto 256^3 in the bench's launch configuration;
    64 random cells checked against the oracle run on every cube that can reach them."""
    cfg = CONFIGS[2]
    pos = config_positions(cfg)
    # the launch configurations the bench's autotuner chooses among (128-thread blocks per SM)
    runs = [gpu_lattice(pos, cfg.n, cfg.grid_n, pse.PSE_FP32_FP64ACC, pse.PSE_WARP_COOPERATIVE, stats=True,
                        tuning={"blocks_per_sm": b}) for b in (2, 3, 4)]
    m, st = runs[1]
    assert st["tets"] == cfg.n_tets
    assert abs(m.sum() - 1.0) <= MASS32
    for other, _ in (runs[0], runs[2]):
        assert cell_errors(other, m)["max_rel"] <= 2e-6
    rng = np.random.default_rng(2024)
    g = cfg.grid_n
    cells = [tuple(int(x) for x in rng.integers(0, g, 3)) for _ in range(64)]
    ids = candidate_cubes(pos, cfg.n, cells, g)
    ref, _ = oracle.deposit_lattice(pos, cfg.n, g, cube_ids=ids, nthreads=4)
    got = np.array([m[c[2], c[1], c[0]] for c in cells])
    exp = np.array([ref[c[2], c[1], c[0]] for c in cells])
    den = np.maximum(exp, 1e-3 / g ** 3)
    assert np.max(np.abs(got - exp) / den) <= TOL32


def test_config4_full_size_sampled_cells():
    """512^3 particles (805M tetrahedra, k^-1.5, rms 4 spacings: a fifth of the clips go to the
    FP64 guard) onto 512^3 in the bench's launch configuration: 8 random cells against the
    oracle run on every cube that can reach them; mass and counters of the whole deposit."""
    from pse_inputs import zeldovich_positions_device
    cfg = CONFIGS[4]
    pos = zeldovich_positions_device(cfg.n, cfg.spectral_index, cfg.rms_disp, cfg.seed, device="cuda")
    g = cfg.grid_n
    m, st = pse.deposit_uniform(pos, cfg.n, g, tuning={"blocks_per_sm": 4}, stats=True)
    assert st["tets"] == cfg.n_tets
    m = m.cpu().numpy()
    assert abs(m.sum() - 1.0) <= MASS32
    posh = pos.cpu().numpy()
    del pos
    rng = np.random.default_rng(4096)
    cells = [tuple(int(x) for x in rng.integers(0, g, 3)) for _ in range(8)]
    ids = candidate_cubes(posh, cfg.n, cells, g, slab=64)
    ref, _ = oracle.deposit_lattice(posh, cfg.n, g, cube_ids=ids, nthreads=4)
    got = np.array([m[c[2], c[1], c[0]] for c in cells])
    exp = np.array([ref[c[2], c[1], c[0]] for c in cells])
    assert np.max(np.abs(got - exp) / np.maximum(exp, 1e-3 / g ** 3)) <= TOL32


def test_config2_fp32_vs_fp64_gpu_all_cells():
    """The FP32 warp path against the plain FP64 GPU path on every cell of config 2."""
    cfg = CONFIGS[2]
    dpos = dev(config_positions(cfg))
    a = pse.deposit_uniform(dpos, cfg.n, cfg.grid_n, precision=pse.PSE_FP32_FP64ACC,
                            schedule=pse.PSE_WARP_COOPERATIVE).cpu().numpy()
    b = pse.deposit_uniform(dpos, cfg.n, cfg.grid_n, precision=pse.PSE_FP64_PLAIN,
                            schedule=pse.PSE_THREAD_PER_TET).cpu().numpy()
    e = cell_errors(a, b)
    assert e["max_rel"] <= TOL32, e
    assert e["mass"] <= MASS32, e


def test_compensated_graph_replay_and_binned_split():
    """Compensated accumulation through a captured graph (the pair conversion is part of the
    replayed sequence) and through the binned schedule's split work items."""
    n, g = 16, 32
    pos = zeldovich_positions(n, -2.0, 1.5, seed=23)
    ref, _ = oracle.deposit_lattice(pos, n, g)
    dpos = dev(pos)
    ws = torch.empty(pse.workspace_size(schedule=pse.PSE_BINNED_PERSISTENT), dtype=torch.uint8, device="cuda")
    out = torch.empty((g, g, g), dtype=torch.float64, device="cuda")
    for _ in range(3):
        pse.deposit_uniform(dpos, n, g, out=out, workspace=ws, precision=pse.PSE_FP32_COMPENSATED,
                            schedule=pse.PSE_BINNED_PERSISTENT, tuning=dict(SPLIT_TUNING, use_graph=1))
        e = cell_errors(out.cpu().numpy(), ref)
        assert e["max_rel"] <= TOL32 and e["mass"] <= MASS32, e


@pytest.mark.parametrize("sched", [pse.PSE_THREAD_PER_TET, pse.PSE_WARP_PER_TET])
def test_compensated_accumulation_in_the_baseline_kernels(sched):
    """The thread-per-tetrahedron and warp-per-tetrahedron kernels take the accumulation mode
    at run time; with compensated pairs they match the oracle like the tuned kernels, on a
    uniform grid and (thread per tetrahedron) on an adaptive octree."""
    n, g = 16, 32
    pos = zeldovich_positions(n, -2.0, 1.5, seed=24)
    ref, _ = oracle.deposit_lattice(pos, n, g)
    got = pse.deposit_uniform(dev(pos), n, g, precision=pse.PSE_FP32_COMPENSATED, schedule=sched).cpu().numpy()
    e = cell_errors(got, ref)
    assert e["max_rel"] <= TOL32 and e["mass"] <= MASS32, e
    # without the renormalisation (which forces the total mass by construction), the (hi, lo)
    # pairs must carry the same sums as FP64 reductions of the same FP32 clips: a lost lo word
    # would move cells by ~1e-7
    raw_c = pse.deposit_uniform(dev(pos), n, g, precision=pse.PSE_FP32_COMPENSATED, schedule=sched,
                                mass_fixup=False).cpu().numpy()
    raw_f = pse.deposit_uniform(dev(pos), n, g, precision=pse.PSE_FP32_FP64ACC, schedule=sched,
                                mass_fixup=False).cpu().numpy()
    e = cell_errors(raw_c, raw_f)
    assert e["max_rel"] <= 1e-9 and abs(raw_c.sum() - raw_f.sum()) <= 1e-12, e
    if sched == pse.PSE_THREAD_PER_TET:
        dpos = dev(pos)
        oct_ = pse.build_octree_from_tet_sizes(dpos, n, 4, 3, 2.0)
        o, _ = oracle.deposit_octree(pos, n, oct_.leaves(), 4, 3)
        m = pse.deposit_octree(dpos, n, oct_, precision=pse.PSE_FP32_COMPENSATED, schedule=sched).cpu().numpy()
        e = cell_errors(m, o)
        assert e["max_rel"] <= TOL32 and e["mass"] <= MASS32, e


def test_config2_compensated_fp32_accumulation():
    """Config 2 with compensated FP32 accumulation: the same FP32 clips as the FP64-accumulated
    path, so the two agree far inside the clip tolerance, and both keep the oracle's mass."""
    cfg = CONFIGS[2]
    dpos = dev(config_positions(cfg))
    a, sa = pse.deposit_uniform(dpos, cfg.n, cfg.grid_n, precision=pse.PSE_FP32_FP64ACC, stats=True)
    b, sb = pse.deposit_uniform(dpos, cfg.n, cfg.grid_n, precision=pse.PSE_FP32_COMPENSATED, stats=True)
    for k in ("tets", "bbox_cells", "inside_cells", "partial_clips", "fp64_redos"):
        assert sa[k] == sb[k], k
    e = cell_errors(b.cpu().numpy(), a.cpu().numpy())
    assert e["max_rel"] <= 1e-9 and e["mass"] <= MASS32, e
    raw = pse.deposit_uniform(dpos, cfg.n, cfg.grid_n, precision=pse.PSE_FP32_COMPENSATED, mass_fixup=False)
    assert abs(float(raw.sum()) - 1.0) <= 1e-6


def test_inverted_tetrahedra_are_counted_alike_by_every_schedule():
    """Shell crossing turns tetrahedra inside out; every schedule counts the same ones (an
    undisplaced lattice has none)."""
    n, g = 16, 48
    counts = set()
    for name, prec, sched in PATHS:
        _, st = gpu_lattice(zeldovich_positions(n, -1.5, 3.0, seed=77), n, g, prec, sched, stats=True)
        counts.add(st["inverted_tets"])
    assert len(counts) == 1 and counts.pop() > 0
    _, st = pse.deposit_uniform(dev(lattice_positions(8)), 8, 16, stats=True)
    assert st["inverted_tets"] == 0


def test_slab_partition_sums_to_the_whole_deposit():
    """Option B's partition on the GPU path: the z-slabs of three ranks, each deposited alone
    (cube subsets of the whole lattice), sum to the one-shot deposit (each slab renormalised to
    its own tetrahedra's mass, so the sum keeps the total)."""
    from paper_1612_09491_gb300 import shard
    cfg = CONFIGS[1]
    pos = config_positions(cfg)
    dpos = dev(pos)
    whole = pse.deposit_uniform(dpos, cfg.n, cfg.grid_n).cpu().numpy()
    total = np.zeros_like(whole)
    for r in range(3):
        k0, k1 = shard.slab_bounds(cfg.n, 3, r)
        ids = torch.from_numpy(shard.slab_cube_ids(cfg.n, k0, k1)).cuda()
        total += pse.deposit_uniform(dpos, cfg.n, cfg.grid_n, cube_ids=ids).cpu().numpy()
    e = cell_errors(total, whole)
    assert e["max_rel"] <= 2e-6 and e["mass"] <= MASS32, e


def test_stats_overlapped_cells_and_mass_out():
    """The counters added to pse_deposit_stats: every deposit lands in a cell counted as
    overlapped (at least one per tetrahedron, at most its partial plus inside cells), the
    column runs of the warp schedule serve its partial cells (each run at most 2 cells), and
    mass_out is the mass written into the grid."""
    cfg = CONFIGS[1]
    dpos = dev(config_positions(cfg))
    for prec, sched in ((pse.PSE_FP32_FP64ACC, pse.PSE_WARP_COOPERATIVE), (pse.PSE_FP64_PLAIN, pse.PSE_THREAD_PER_TET)):
        m, st = pse.deposit_uniform(dpos, cfg.n, cfg.grid_n, precision=prec, schedule=sched, stats=True)
        assert st["tets"] <= st["overlapped_cells"] <= st["partial_clips"] + st["inside_cells"] + st["tets"]
        assert abs(st["mass_out"] - float(m.sum())) <= 1e-13
        assert abs(st["mass_out"] - 1.0) <= 1e-12
        if sched == pse.PSE_WARP_COOPERATIVE:
            assert 0 < st["column_runs"] and st["partial_clips"] - st["fp64_redos"] <= 2 * st["column_runs"]
        else:
            assert st["column_runs"] == 0


@pytest.mark.parametrize("grid", ["uniform", "octree", "uniform-streamed", "uniform-subset", "octree-subset"])
def test_guarded_list_and_full_rescan_agree(grid):
    """The guarded pass visits only the tetrahedra the FP32 pass listed, or (list disabled, or
    more guarded tetrahedra than the list holds) scans every tetrahedron again.  The three give
    the same deposit and the same counters, on a shell-crossed lattice where about a quarter of
    the tetrahedra are guarded; the subset cases take a shuffled list of cube ids, whose
    listed ids decode differently from a whole lattice's."""
    n, g = 24, 48
    pos = zeldovich_positions(n, -1.5, 3.0, seed=31)
    dpos = dev(pos)
    ids = np.random.default_rng(3).permutation(n ** 3)[: n ** 3 // 3]
    dids = torch.from_numpy(ids.astype(np.int64)).cuda()
    if grid.startswith("octree"):
        oct_ = pse.build_octree_from_tet_sizes(dpos, n, 8, 3, 2.0)

    def run(cap):
        tu = {"blocks_per_sm": 4, "guard_list_cap": cap}
        if grid == "octree":
            m, st = pse.deposit_octree(dpos, n, oct_, stats=True, tuning=tu, mass_fixup=False)
        elif grid == "octree-subset":
            m, st = pse.deposit_octree(dpos, n, oct_, stats=True, tuning=tu, mass_fixup=False, cube_ids=dids)
        elif grid == "uniform":
            m, st = pse.deposit_uniform(dpos, n, g, stats=True, tuning=tu, mass_fixup=False)
        elif grid == "uniform-subset":
            m, st = pse.deposit_uniform(dpos, n, g, stats=True, tuning=tu, mass_fixup=False, cube_ids=dids)
        else:
            m, st = pse.deposit_uniform_streamed(torch.from_numpy(pos).pin_memory(), n, g, 5, stats=True,
                                                 tuning=tu, mass_fixup=False)
        return m.cpu().numpy(), st

    ref, st_ref = run(0)        # the list (default capacity)
    assert st_ref["fp64_redos"] > 0.1 * st_ref["partial_clips"]
    for cap in (-1, 1000):      # no list; a list too small for this lattice
        m, st = run(cap)
        e = cell_errors(m, ref)
        assert e["max_rel"] <= 1e-12 and e["mass"] <= 1e-13, (cap, e)
        for k in ("tets", "partial_clips", "fp64_redos", "column_runs", "overlapped_cells", "bbox_cells"):
            assert st[k] == st_ref[k], (cap, k, st[k], st_ref[k])
    if grid in ("uniform", "octree"):
        o, _ = (oracle.deposit_octree(pos, n, oct_.leaves(), 8, 3) if grid == "octree"
                else oracle.deposit_lattice(pos, n, g))
        e = cell_errors(ref, o)
        assert e["max_rel"] <= TOL32, e
    elif grid.endswith("subset"):  # the subset's own deposit, against the oracle on the same cubes
        o, _ = (oracle.deposit_octree(pos, n, oct_.leaves(), 8, 3, cube_ids=np.sort(ids)) if grid == "octree-subset"
                else oracle.deposit_lattice(pos, n, g, cube_ids=np.sort(ids)))
        e = cell_errors(ref, o)
        assert e["mass"] <= 1e-6, e  # no renormalisation here: the FP32 clips' own sum
        if grid == "uniform-subset":
            tets = subset_tets(pos, n, np.sort(ids))
            e = cell_errors(ref, o, floor_mass=density_floor(tets, np.full(len(tets), 1.0 / (6 * n ** 3)), g))
            assert e["max_rel"] <= TOL32, e
