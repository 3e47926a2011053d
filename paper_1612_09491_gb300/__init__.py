"""GB300 (sm_103a) exact tetrahedron deposit of the phase-space-element method.

Thin torch-facing wrappers of the C ABI (include/pse.h); names follow the ABI
without its ``pse_`` prefix.  Tensors must live on the current CUDA device; the
work is enqueued on the current torch stream (or ``stream=``).  Nothing here
computes: every step runs in libpse.so.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import (  # noqa: F401
    PSE_BINNED_PERSISTENT,
    PSE_FP32_COMPENSATED,
    PSE_FP32_FP64ACC,
    PSE_FP64_PLAIN,
    PSE_THREAD_PER_TET,
    PSE_WARP_PER_TET,
    PSE_WARP_COOPERATIVE,
    PseError,
)

__all__ = ["build_tets_from_lagrangian_grid", "deposit_uniform", "deposit_tets", "workspace_size", "last_error",
           "abi_version", "lattice", "opts", "OctreeHandle", "octree_from_leaves", "build_octree_from_tet_sizes",
           "deposit_octree", "deposit_uniform_streamed", "deposit_octree_streamed", "build_octree_streamed"]


_EMPTY_SENTINEL = 16  # non-NULL, never dereferenced (n_cube_ids == 0)


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def lattice(n, box: float = 1.0, periodic: bool = True, particle_mass: float | None = None) -> _lib.Lattice:
    n3 = (n, n, n) if isinstance(n, int) else tuple(int(x) for x in n)
    if particle_mass is None:
        particle_mass = box ** 3 / float(n3[0] * n3[1] * n3[2])  # mean density 1
    lat = _lib.Lattice()
    lat.n[:] = n3
    lat.box = float(box)
    lat.periodic = 1 if periodic else 0
    lat.particle_mass = float(particle_mass)
    return lat


_keep = []  # tuning blocks referenced by option structs during a call


def opts(precision: int = PSE_FP32_FP64ACC, schedule: int = PSE_WARP_COOPERATIVE, guard_eps: float = 0.0,
         accumulate: bool = False, mass_fixup: bool = True, cube_ids=None, tuning=None,
         cost_model=None) -> _lib.DepositOpts:
    """cost_model: a costmodel.CostModel (binned schedule) or None."""
    o = _lib.DepositOpts()
    if cost_model is not None:
        o.cost_model = cost_model.ptr
    if tuning is not None:
        tu = _lib.Tuning()
        tu.blocks_per_sm = int(tuning.get("blocks_per_sm", 0))
        tu.warps_per_block = int(tuning.get("warps_per_block", 0))
        tu.split_cells = int(tuning.get("split_cells", 0))
        tu.chunk_cells = int(tuning.get("chunk_cells", 0))
        tu.use_graph = int(tuning.get("use_graph", 0))
        tu.guard_list_cap = int(tuning.get("guard_list_cap", 0))
        _keep[:] = [tu]
        o.tuning = ctypes.cast(ctypes.pointer(tu), ctypes.c_void_p).value
    o.precision = precision
    o.schedule = schedule
    o.guard_eps = guard_eps
    o.accumulate = 1 if accumulate else 0
    o.mass_fixup = 1 if mass_fixup else 0
    if cube_ids is not None:
        _dev_ptr(cube_ids, _torch().int64, "cube_ids")
        # an empty subset still needs a non-NULL pointer (NULL means "every cube"); it is never read
        o.d_cube_ids = cube_ids.data_ptr() if cube_ids.numel() > 0 else _EMPTY_SENTINEL
        o.n_cube_ids = cube_ids.numel()
    return o


def _grid3(grid_n):
    g = (grid_n,) * 3 if isinstance(grid_n, int) else tuple(int(x) for x in grid_n)
    return (ctypes.c_int64 * 3)(*g), g


def deposit_uniform(pos, n, grid_n, *, box: float = 1.0, periodic: bool = True, particle_mass=None, out=None,
                    precision: int = PSE_FP32_FP64ACC, schedule: int = PSE_WARP_COOPERATIVE, guard_eps: float = 0.0,
                    accumulate: bool = False, mass_fixup: bool = True, cube_ids=None, stats: bool = False,
                    workspace=None, stream=None, tuning=None, cost_model=None):
    """pse_deposit_uniform: cell masses float64 [g2, g1, g0] (x fastest)."""
    torch = _torch()
    L = _lib.load()
    lat = lattice(n, box, periodic, particle_mass)
    g3, g = _grid3(grid_n)
    if out is None:
        out = torch.empty((g[2], g[1], g[0]), dtype=torch.float64, device=pos.device)
    o = opts(precision, schedule, guard_eps, accumulate, mass_fixup, cube_ids, tuning, cost_model)
    st = _lib.DepositStats() if stats else None
    ws_ptr, ws_bytes = (ctypes.c_void_p(None), 0) if workspace is None else \
        (_dev_ptr(workspace, torch.uint8, "workspace"), workspace.numel())
    rc = L.pse_deposit_uniform(_dev_ptr(pos, torch.float32, "pos"), ctypes.byref(lat), g3,
                               _dev_ptr(out, torch.float64, "out"), ctypes.byref(o),
                               ctypes.byref(st) if st is not None else None, ws_ptr, ws_bytes, _stream_ptr(stream))
    _lib.check(rc)
    return (out, st.to_dict()) if stats else out


def deposit_tets(verts, tet_mass, grid_n, *, box: float = 1.0, periodic: bool = True, out=None,
                 precision: int = PSE_FP32_FP64ACC, schedule: int = PSE_WARP_COOPERATIVE, guard_eps: float = 0.0,
                 accumulate: bool = False, mass_fixup: bool = True, stats: bool = False, workspace=None, stream=None,
                 tuning=None):
    """pse_deposit_tets: explicit tetrahedra verts float32 [T, 4, 3] (box units), masses float64 [T]."""
    torch = _torch()
    L = _lib.load()
    g3, g = _grid3(grid_n)
    if out is None:
        out = torch.empty((g[2], g[1], g[0]), dtype=torch.float64, device=verts.device)
    o = opts(precision, schedule, guard_eps, accumulate, mass_fixup, tuning=tuning)
    st = _lib.DepositStats() if stats else None
    ws_ptr, ws_bytes = (ctypes.c_void_p(None), 0) if workspace is None else \
        (_dev_ptr(workspace, torch.uint8, "workspace"), workspace.numel())
    T = verts.shape[0]
    rc = L.pse_deposit_tets(_dev_ptr(verts, torch.float32, "verts"), _dev_ptr(tet_mass, torch.float64, "tet_mass"),
                            T, float(box), 1 if periodic else 0, g3, _dev_ptr(out, torch.float64, "out"),
                            ctypes.byref(o), ctypes.byref(st) if st is not None else None, ws_ptr, ws_bytes,
                            _stream_ptr(stream))
    _lib.check(rc)
    return (out, st.to_dict()) if stats else out


def build_tets_from_lagrangian_grid(pos, n, *, box: float = 1.0, periodic: bool = True, want_vidx: bool = True,
                                    want_vol: bool = True, stream=None):
    """pse_build_tets_from_lagrangian_grid: (vidx int32 [T,4] or None, signed vol float32 [T] or None)."""
    torch = _torch()
    L = _lib.load()
    lat = lattice(n, box, periodic)
    nt = ctypes.c_int64(0)
    _lib.check(L.pse_build_tets_from_lagrangian_grid(_dev_ptr(pos, torch.float32, "pos"), ctypes.byref(lat), None,
                                                     None, ctypes.byref(nt), _stream_ptr(stream)))
    T = nt.value
    vidx = torch.empty((T, 4), dtype=torch.int32, device=pos.device) if want_vidx else None
    vol = torch.empty((T,), dtype=torch.float32, device=pos.device) if want_vol else None
    _lib.check(L.pse_build_tets_from_lagrangian_grid(
        _dev_ptr(pos, torch.float32, "pos"), ctypes.byref(lat),
        _dev_ptr(vidx, torch.int32, "vidx") if vidx is not None else None,
        _dev_ptr(vol, torch.float32, "vol") if vol is not None else None, None, _stream_ptr(stream)))
    return vidx, vol


def workspace_size(op: int = _lib.PSE_OP_DEPOSIT_UNIFORM, lat=None, schedule=None, cost_model=None) -> int:
    """pse_workspace_size; schedule / cost_model: what the deposit will use (the binned schedule
    needs room for its queue, and with a cost model for one bit per tetrahedron of lat)."""
    o = None
    if schedule is not None:
        o = _lib.DepositOpts()
        o.precision = PSE_FP32_FP64ACC
        o.schedule = schedule
        if cost_model is not None:
            o.cost_model = cost_model.ptr
    return int(_lib.load().pse_workspace_size(op, ctypes.byref(lat) if lat is not None else None,
                                              ctypes.cast(ctypes.pointer(o), ctypes.c_void_p) if o is not None else None))


def last_error() -> str:
    return _lib.load().pse_last_error().decode()


def abi_version() -> int:
    return int(_lib.load().pse_abi_version())


class OctreeHandle:
    """Owns a pse_octree; frees it with pse_free_octree when collected."""

    def __init__(self, st: _lib.Octree):
        self.st = st

    @property
    def bc(self) -> int:
        return self.st.bc

    @property
    def max_level(self) -> int:
        return self.st.max_level

    @property
    def n_leaves(self) -> int:
        return self.st.n_leaves

    @property
    def n_cells(self) -> int:
        return self.st.n_cells

    def leaves(self):
        import numpy as np
        buf = (ctypes.c_int32 * (4 * self.st.n_leaves)).from_address(self.st.h_leaves)
        return np.frombuffer(buf, dtype=np.int32).reshape(-1, 4).copy()

    def __del__(self):
        try:
            if self.st.h_leaves:
                _lib.load().pse_free_octree(ctypes.byref(self.st))
        except Exception:
            pass


def octree_from_leaves(leaves, bc: int, max_level: int, box: float = 1.0) -> OctreeHandle:
    """pse_octree_from_leaves: leaves int32 [L, 4] (level, ix, iy, iz) that tile the box."""
    import numpy as np
    lv = np.ascontiguousarray(leaves, dtype=np.int32)
    st = _lib.Octree()
    _lib.check(_lib.load().pse_octree_from_leaves(lv.ctypes.data_as(ctypes.c_void_p), lv.shape[0], bc, max_level,
                                                  float(box), ctypes.byref(st)))
    return OctreeHandle(st)


def build_octree_from_tet_sizes(pos, n, bc: int, max_level: int, threshold_cells: float = 2.0, *,
                                box: float = 1.0, stream=None) -> OctreeHandle:
    """pse_build_octree_from_tet_sizes (periodic lattice)."""
    torch = _torch()
    lat = lattice(n, box, True)
    st = _lib.Octree()
    _lib.check(_lib.load().pse_build_octree_from_tet_sizes(_dev_ptr(pos, torch.float32, "pos"), ctypes.byref(lat),
                                                           bc, max_level, float(threshold_cells), ctypes.byref(st),
                                                           None, 0, _stream_ptr(stream)))
    return OctreeHandle(st)


def deposit_octree(pos, n, octree: OctreeHandle, *, box: float = 1.0, particle_mass=None, out=None,
                   precision: int = PSE_FP32_FP64ACC, schedule: int = PSE_WARP_COOPERATIVE, guard_eps: float = 0.0,
                   accumulate: bool = False, mass_fixup: bool = True, cube_ids=None, stats: bool = False,
                   workspace=None, stream=None, tuning=None):
    """pse_deposit_octree: leaf masses float64 [n_leaves, bc, bc, bc] (x fastest within a block)."""
    torch = _torch()
    L = _lib.load()
    lat = lattice(n, box, True, particle_mass)
    bc = octree.bc
    if out is None:
        out = torch.empty((octree.n_leaves, bc, bc, bc), dtype=torch.float64, device=pos.device)
    o = opts(precision, schedule, guard_eps, accumulate, mass_fixup, cube_ids, tuning)
    st = _lib.DepositStats() if stats else None
    ws_ptr, ws_bytes = (ctypes.c_void_p(None), 0) if workspace is None else \
        (_dev_ptr(workspace, torch.uint8, "workspace"), workspace.numel())
    rc = L.pse_deposit_octree(_dev_ptr(pos, torch.float32, "pos"), ctypes.byref(lat), ctypes.byref(octree.st),
                              _dev_ptr(out, torch.float64, "out"), ctypes.byref(o),
                              ctypes.byref(st) if st is not None else None, ws_ptr, ws_bytes, _stream_ptr(stream))
    _lib.check(rc)
    return (out, st.to_dict()) if stats else out


def _host_ptr(t, name):
    """Pointer of a contiguous float32 CPU tensor or numpy array (host memory)."""
    torch = _torch()
    import numpy as np
    if isinstance(t, torch.Tensor):
        if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float32 CPU tensor")
        return ctypes.c_void_p(t.data_ptr())
    if not isinstance(t, np.ndarray) or t.dtype != np.float32 or not t.flags["C_CONTIGUOUS"]:
        raise TypeError(f"{name} must be a contiguous float32 array")
    return ctypes.c_void_p(t.ctypes.data)


def deposit_uniform_streamed(h_pos, n, grid_n, slab_cubes: int, *, box: float = 1.0, particle_mass=None, out=None,
                             device="cuda", precision: int = PSE_FP32_FP64ACC, schedule: int = PSE_WARP_COOPERATIVE,
                             guard_eps: float = 0.0, accumulate: bool = False, mass_fixup: bool = True,
                             stats: bool = False, workspace=None, stream=None, tuning=None, cost_model=None):
    """pse_deposit_uniform_streamed: positions in host memory (pinned for overlap), z-slabs of slab_cubes."""
    torch = _torch()
    L = _lib.load()
    lat = lattice(n, box, True, particle_mass)
    g3, g = _grid3(grid_n)
    if out is None:
        out = torch.empty((g[2], g[1], g[0]), dtype=torch.float64, device=device)
    o = opts(precision, schedule, guard_eps, accumulate, mass_fixup, None, tuning, cost_model)
    st = _lib.DepositStats() if stats else None
    ws_ptr, ws_bytes = (ctypes.c_void_p(None), 0) if workspace is None else \
        (_dev_ptr(workspace, torch.uint8, "workspace"), workspace.numel())
    _lib.check(L.pse_deposit_uniform_streamed(_host_ptr(h_pos, "h_pos"), ctypes.byref(lat), int(slab_cubes), g3,
                                              _dev_ptr(out, torch.float64, "out"), ctypes.byref(o),
                                              ctypes.byref(st) if st is not None else None, ws_ptr, ws_bytes,
                                              _stream_ptr(stream)))
    return (out, st.to_dict()) if stats else out


def deposit_octree_streamed(h_pos, n, octree: OctreeHandle, slab_cubes: int, *, box: float = 1.0,
                            particle_mass=None, out=None, device="cuda", precision: int = PSE_FP32_FP64ACC,
                            schedule: int = PSE_WARP_COOPERATIVE, guard_eps: float = 0.0, accumulate: bool = False,
                            mass_fixup: bool = True, stats: bool = False, workspace=None, stream=None, tuning=None):
    """pse_deposit_octree_streamed: leaf masses [n_leaves, bc, bc, bc] from host positions in z-slabs."""
    torch = _torch()
    L = _lib.load()
    lat = lattice(n, box, True, particle_mass)
    bc = octree.bc
    if out is None:
        out = torch.empty((octree.n_leaves, bc, bc, bc), dtype=torch.float64, device=device)
    o = opts(precision, schedule, guard_eps, accumulate, mass_fixup, None, tuning)
    st = _lib.DepositStats() if stats else None
    ws_ptr, ws_bytes = (ctypes.c_void_p(None), 0) if workspace is None else \
        (_dev_ptr(workspace, torch.uint8, "workspace"), workspace.numel())
    _lib.check(L.pse_deposit_octree_streamed(_host_ptr(h_pos, "h_pos"), ctypes.byref(lat), int(slab_cubes),
                                             ctypes.byref(octree.st), _dev_ptr(out, torch.float64, "out"),
                                             ctypes.byref(o), ctypes.byref(st) if st is not None else None, ws_ptr,
                                             ws_bytes, _stream_ptr(stream)))
    return (out, st.to_dict()) if stats else out


def build_octree_streamed(h_pos, n, bc: int, max_level: int, slab_cubes: int, threshold_cells: float = 2.0, *,
                          box: float = 1.0, stream=None) -> OctreeHandle:
    """pse_build_octree_streamed: the size-rule octree of a lattice held in host memory."""
    lat = lattice(n, box, True)
    st = _lib.Octree()
    _lib.check(_lib.load().pse_build_octree_streamed(_host_ptr(h_pos, "h_pos"), ctypes.byref(lat), int(slab_cubes),
                                                     bc, max_level, float(threshold_cells), ctypes.byref(st),
                                                     _stream_ptr(stream)))
    return OctreeHandle(st)


def measure_peaks(stream=None, fma_blocks: int = 152 * 8, fma_iters: int = 1 << 16, red_cells: int = 1 << 24,
                  red_blocks: int = 152 * 8, red_per_thread: int = 4096) -> dict:
    """FP32 FMA rate and FP64 global-reduction rate of the current GPU (pse_microbench_*),
    best of 3 timed launches after one warm-up, CUDA events on the stream."""
    torch = _torch()
    L = _lib.load()
    if stream is None:
        stream = torch.cuda.current_stream()
    out = torch.empty(fma_blocks * 256, dtype=torch.float32, device="cuda")
    grid = torch.zeros(red_cells, dtype=torch.float64, device="cuda")

    def best(fn):
        fn()
        ms = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return min(ms)
    sp = ctypes.c_void_p(stream.cuda_stream)
    t_fma = best(lambda: _lib.check(L.pse_microbench_fma(ctypes.c_void_p(out.data_ptr()), fma_blocks, fma_iters, sp)))
    t_red = best(lambda: _lib.check(L.pse_microbench_red(ctypes.c_void_p(grid.data_ptr()), red_cells, red_blocks,
                                                         red_per_thread, sp)))
    flop = 2.0 * 8 * fma_iters * 256 * fma_blocks
    reds = float(red_per_thread) * 256 * red_blocks
    return {"fp32_tflops": flop / (t_fma * 1e-3) / 1e12, "red_f64_per_s": reds / (t_red * 1e-3),
            "fma_ms": t_fma, "red_ms": t_red,
            "how": f"{fma_blocks} x 256 threads x 8 FMA chains x {fma_iters} steps; {red_blocks} x 256 threads x "
                   f"{red_per_thread} FP64 reductions over {red_cells} cells (8-byte, pseudo-random)"}


def octree_restrict(octree: OctreeHandle, leaf_mass, stream=None):
    """pse_octree_restrict: float64 [P, bc, bc, bc] masses of every node of levels 0..max_level-1
    (row of node (l, x, y, z): sum_{k<l} 8^k + x + 2^l (y + 2^l z))."""
    torch = _torch()
    bc, ml = octree.bc, octree.max_level
    rows = sum(8 ** k for k in range(ml))
    out = torch.empty((max(rows, 0), bc, bc, bc), dtype=torch.float64, device=leaf_mass.device)
    if rows == 0:
        return out
    _lib.check(_lib.load().pse_octree_restrict(ctypes.byref(octree.st), _dev_ptr(leaf_mass, torch.float64, "leaf_mass"),
                                               _dev_ptr(out, torch.float64, "out"), _stream_ptr(stream)))
    return out


def build_octree_count(pos, n, bc: int, max_level: int, count_threshold: float, subblock: int = 8, *,
                       box: float = 1.0, stream=None) -> OctreeHandle:
    """pse_build_octree_count: the paper's refinement rule (estimated tetrahedra per node)."""
    torch = _torch()
    lat = lattice(n, box, True)
    st = _lib.Octree()
    _lib.check(_lib.load().pse_build_octree_count(_dev_ptr(pos, torch.float32, "pos"), ctypes.byref(lat), bc,
                                                  max_level, float(count_threshold), int(subblock),
                                                  ctypes.byref(st), _stream_ptr(stream)))
    return OctreeHandle(st)
