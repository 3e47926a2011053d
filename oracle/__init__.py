"""FP64 CPU oracle of the exact tetrahedron deposit -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (``paper_1612_09491_gb300``)
never imports it, and it never imports the product.

``oracle.c`` is a plain C implementation of M[c] = sum_t m_t/|V_t| vol(T_t ∩ C_c)
(Eq. 1 integrated over a cell) by the CPU deposit of Sec. 6.1 and the recursive
tetrahedron split of Sec. 6.3.  ``exact.py`` holds an independent exact-rational
evaluation (Lasserre's recursion) used only to pin the C oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-Wall", "-Wextra",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, stdout=sys.stderr, stderr=sys.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            ip = ctypes.POINTER(ctypes.c_int)
            L.oracle_deposit_lattice.argtypes = [fp, i64p, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                                 i64p, dp, i64p, ctypes.c_int64, ctypes.c_int, dp]
            L.oracle_deposit_lattice.restype = ctypes.c_int
            L.oracle_deposit_tets.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                              i64p, dp, dp]
            L.oracle_deposit_tets.restype = ctypes.c_int
            L.oracle_tet_box_volume.argtypes = [dp, dp, dp]
            L.oracle_tet_box_volume.restype = ctypes.c_double
            L.oracle_tet_halfspaces_volume.argtypes = [dp, ip, ip, dp, ctypes.c_int]
            L.oracle_tet_halfspaces_volume.restype = ctypes.c_double
            L.oracle_lattice_tet.argtypes = [fp, i64p, ctypes.c_double, ctypes.c_int, ctypes.c_int64,
                                             ctypes.c_int, dp]
            L.oracle_lattice_tet.restype = ctypes.c_int
            L.oracle_tet_cells.argtypes = [dp, dp, i64p, dp, ctypes.c_int64]
            L.oracle_tet_cells.restype = ctypes.c_int64
            L.oracle_tet_volume.argtypes = [dp]
            L.oracle_tet_volume.restype = ctypes.c_double
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.oracle_build_octree.argtypes = [fp, i64p, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_double, i32p, ctypes.c_int64, dp, ctypes.c_int64, i64p]
            L.oracle_build_octree.restype = ctypes.c_int64
            L.oracle_deposit_octree.argtypes = [fp, i64p, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int64, dp, i64p,
                                                ctypes.c_int64, ctypes.c_int, dp]
            L.oracle_deposit_octree.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


STAT_KEYS = ("tets", "bbox_cells", "overlapped_cells", "partial_cells", "degenerate_tets",
             "lost_mass", "threads")


def deposit_lattice(pos: np.ndarray, n, grid_n, box: float = 1.0, periodic: bool = True,
                    particle_mass: float | None = None, cube_ids=None, nthreads: int = 0):
    """Cell masses [G2, G1, G0] (x fastest) of the lattice tessellation; returns (mass, stats)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    n = np.ascontiguousarray(np.broadcast_to(np.asarray(n, dtype=np.int64), (3,)))
    g = np.ascontiguousarray(np.broadcast_to(np.asarray(grid_n, dtype=np.int64), (3,)))
    if pos.shape != (int(np.prod(n)), 3):
        raise ValueError("pos must be [n0*n1*n2, 3]")
    if particle_mass is None:
        particle_mass = 1.0 / float(np.prod(n))  # mean density 1 in a unit box
    out = np.zeros(int(np.prod(g)), dtype=np.float64)
    st = np.zeros(7, dtype=np.float64)
    if cube_ids is not None:
        cube_ids = np.ascontiguousarray(cube_ids, dtype=np.int64)
        cptr, ncid = _ptr(cube_ids, ctypes.c_int64), cube_ids.size
    else:
        cptr, ncid = None, 0
    rc = lib().oracle_deposit_lattice(_ptr(pos, ctypes.c_float), _ptr(n, ctypes.c_int64), box,
                                      int(periodic), particle_mass, _ptr(g, ctypes.c_int64),
                                      _ptr(out, ctypes.c_double), cptr, ncid, int(nthreads),
                                      _ptr(st, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle_deposit_lattice failed: {rc}")
    return out.reshape(int(g[2]), int(g[1]), int(g[0])), dict(zip(STAT_KEYS, st.tolist()))


def deposit_tets(verts: np.ndarray, tet_mass, grid_n, box: float = 1.0, periodic: bool = True):
    """Cell masses of explicit tetrahedra verts [T, 4, 3] (box units); returns (mass, stats)."""
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    T = verts.shape[0]
    tm = np.ascontiguousarray(np.broadcast_to(np.asarray(tet_mass, dtype=np.float64), (T,)))
    g = np.ascontiguousarray(np.broadcast_to(np.asarray(grid_n, dtype=np.int64), (3,)))
    out = np.zeros(int(np.prod(g)), dtype=np.float64)
    st = np.zeros(7, dtype=np.float64)
    rc = lib().oracle_deposit_tets(_ptr(verts, ctypes.c_double), _ptr(tm, ctypes.c_double), T, box,
                                   int(periodic), _ptr(g, ctypes.c_int64), _ptr(out, ctypes.c_double),
                                   _ptr(st, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle_deposit_tets failed: {rc}")
    return out.reshape(int(g[2]), int(g[1]), int(g[0])), dict(zip(STAT_KEYS, st.tolist()))


def tet_box_volume(tet, lo, hi) -> float:
    t = np.ascontiguousarray(tet, dtype=np.float64).reshape(12)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    return lib().oracle_tet_box_volume(_ptr(t, ctypes.c_double), _ptr(lo, ctypes.c_double),
                                       _ptr(hi, ctypes.c_double))


def tet_halfspaces_volume(tet, halfspaces) -> float:
    """halfspaces: iterable of (axis, keep_below, s)."""
    t = np.ascontiguousarray(tet, dtype=np.float64).reshape(12)
    hs = list(halfspaces)
    ax = np.array([h[0] for h in hs], dtype=np.intc)
    kb = np.array([int(h[1]) for h in hs], dtype=np.intc)
    s = np.array([h[2] for h in hs], dtype=np.float64)
    return lib().oracle_tet_halfspaces_volume(_ptr(t, ctypes.c_double), _ptr(ax, ctypes.c_int),
                                              _ptr(kb, ctypes.c_int), _ptr(s, ctypes.c_double), len(hs))


def lattice_tet(pos, n, cube: int, s: int, box: float = 1.0, periodic: bool = True) -> np.ndarray:
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    n = np.ascontiguousarray(np.broadcast_to(np.asarray(n, dtype=np.int64), (3,)))
    out = np.zeros(12, dtype=np.float64)
    rc = lib().oracle_lattice_tet(_ptr(pos, ctypes.c_float), _ptr(n, ctypes.c_int64), box, int(periodic),
                                  int(cube), int(s), _ptr(out, ctypes.c_double))
    if rc != 0:
        raise RuntimeError("oracle_lattice_tet failed")
    return out.reshape(4, 3)


def tet_cells(tet, h):
    """All cells (ix, iy, iz) overlapped by one tetrahedron with their overlap volumes (no folding)."""
    t = np.ascontiguousarray(tet, dtype=np.float64).reshape(12)
    hh = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (3,)))
    cap = 4096
    while True:
        cells = np.zeros((cap, 3), dtype=np.int64)
        vols = np.zeros(cap, dtype=np.float64)
        cnt = lib().oracle_tet_cells(_ptr(t, ctypes.c_double), _ptr(hh, ctypes.c_double),
                                     _ptr(cells, ctypes.c_int64), _ptr(vols, ctypes.c_double), cap)
        if cnt < 0:
            raise RuntimeError("oracle_tet_cells failed")
        if cnt <= cap:
            return cells[:cnt].copy(), vols[:cnt].copy()
        cap = int(cnt)


def tet_volume(tet) -> float:
    t = np.ascontiguousarray(tet, dtype=np.float64).reshape(12)
    return lib().oracle_tet_volume(_ptr(t, ctypes.c_double))


def build_octree(pos, n, bc: int, max_level: int, threshold_cells: float = 2.0, box: float = 1.0,
                 periodic: bool = True):
    """Exact-median octree (Sec. 4 structure, tetrahedron-size rule): (leaves [L,4] int32, nodes [K,7])."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    n = np.ascontiguousarray(np.broadcast_to(np.asarray(n, dtype=np.int64), (3,)))
    cap, ncap = 4096, 8192
    while True:
        leaves = np.zeros((cap, 4), dtype=np.int32)
        nodes = np.zeros((ncap, 7), dtype=np.float64)
        nn = ctypes.c_int64(0)
        cnt = lib().oracle_build_octree(_ptr(pos, ctypes.c_float), _ptr(n, ctypes.c_int64), box, int(periodic),
                                        int(bc), int(max_level), float(threshold_cells),
                                        _ptr(leaves, ctypes.c_int32), cap, _ptr(nodes, ctypes.c_double), ncap,
                                        ctypes.byref(nn))
        if cnt < 0:
            raise RuntimeError(f"oracle_build_octree failed: {cnt}")
        if cnt <= cap and nn.value <= ncap:
            return leaves[:cnt].copy(), nodes[:nn.value].copy()
        cap, ncap = max(cap, int(cnt)), max(ncap, int(nn.value))


def deposit_octree(pos, n, leaves, bc: int, max_level: int, box: float = 1.0, periodic: bool = True,
                   particle_mass: float | None = None, cube_ids=None, nthreads: int = 0):
    """Leaf-block masses [n_leaves, bc, bc, bc] (x fastest within a block); returns (mass, stats)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    n = np.ascontiguousarray(np.broadcast_to(np.asarray(n, dtype=np.int64), (3,)))
    leaves = np.ascontiguousarray(leaves, dtype=np.int32)
    if particle_mass is None:
        particle_mass = box ** 3 / float(np.prod(n))
    nl = leaves.shape[0]
    out = np.zeros(nl * bc ** 3, dtype=np.float64)
    st = np.zeros(7, dtype=np.float64)
    if cube_ids is not None:
        cube_ids = np.ascontiguousarray(cube_ids, dtype=np.int64)
        cptr, ncid = _ptr(cube_ids, ctypes.c_int64), cube_ids.size
    else:
        cptr, ncid = None, 0
    rc = lib().oracle_deposit_octree(_ptr(pos, ctypes.c_float), _ptr(n, ctypes.c_int64), box, int(periodic),
                                     particle_mass, int(bc), int(max_level), _ptr(leaves, ctypes.c_int32), nl,
                                     _ptr(out, ctypes.c_double), cptr, ncid, int(nthreads), _ptr(st, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle_deposit_octree failed: {rc}")
    return out.reshape(nl, bc, bc, bc), dict(zip(STAT_KEYS, st.tolist()))


def build_octree_count(pos, n, bc: int, max_level: int, count_threshold: float, subblock: int = 8,
                       box: float = 1.0):
    """The refinement rule of Sec. 4 in plain float64 numpy: subblocks of subblock^3 cubes, the
    bounding box of each subblock's (unwrapped) particles, the estimated tetrahedra per node
    sum_b 6 cubes_b vol(box_b ∩ node) / vol(box_b) over periodic images; refine while the
    estimate exceeds count_threshold and level < max_level.  Returns (leaves [L, 4] depth first,
    {(level, ix, iy, iz): estimate} of every evaluated node)."""
    p = np.asarray(pos, dtype=np.float64).reshape(n, n, n, 3)  # [k, j, i, axis]
    nbl = (n + subblock - 1) // subblock
    boxes = []
    for bz in range(nbl):
        for by in range(nbl):
            for bx in range(nbl):
                i0, j0, k0 = bx * subblock, by * subblock, bz * subblock
                i1, j1, k1 = min(n, i0 + subblock), min(n, j0 + subblock), min(n, k0 + subblock)
                ii = np.arange(i0, i1 + 1) % n
                jj = np.arange(j0, j1 + 1) % n
                kk = np.arange(k0, k1 + 1) % n
                pts = p[np.ix_(kk, jj, ii)].reshape(-1, 3)
                ref = p[k0, j0, i0]
                d = pts - ref
                d -= np.where(d >= 0.5 * box, box, np.where(d < -0.5 * box, -box, 0.0))
                q = ref + d
                boxes.append((q.min(0), q.max(0), 6.0 * (i1 - i0) * (j1 - j0) * (k1 - k0)))

    def overlap(lo, hi, x0, x1):
        return sum(max(min(hi + s * box, x1) - max(lo + s * box, x0), 0.0) for s in (-1, 0, 1))

    est = {}

    def visit(level, ix, iy, iz, leaves):
        refine = False
        if level < max_level:
            size = box / 2 ** level
            x0 = np.array([ix, iy, iz]) * size
            total = 0.0
            for lo, hi, tets in boxes:
                vol = float(np.prod(hi - lo))
                if not vol > 0.0:
                    continue
                ov = 1.0
                for a in range(3):
                    ov *= overlap(lo[a], hi[a], x0[a], x0[a] + size)
                total += tets * ov / vol
            est[(level, ix, iy, iz)] = total
            refine = total > count_threshold
        if not refine:
            leaves.append((level, ix, iy, iz))
            return
        for c in range(8):
            visit(level + 1, 2 * ix + (c & 1), 2 * iy + ((c >> 1) & 1), 2 * iz + (c >> 2), leaves)

    leaves = []
    visit(0, 0, 0, 0, leaves)
    return np.array(leaves, dtype=np.int32), est
