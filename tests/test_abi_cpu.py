"""CPU-side checks of the C ABI: the library builds, loads, exports every symbol
include/pse.h declares, its ctypes mirrors match the C layouts, and argument
errors come back as status codes before any device work is attempted."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

from paper_1612_09491_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pse.h")


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.load()


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"PSE_API\s+[\w\s\*]*?\b(pse_\w+)\s*\(", txt)))


def test_header_declares_what_binding_lists():
    assert declared_symbols() == sorted(_lib.EXPORTED)


def test_binding_constants_match_header():
    """Every integer constant the binding mirrors has the header's value."""
    defs = dict(re.findall(r"^#define\s+(PSE_\w+)\s+(-?\d+)\b", open(HEADER).read(), re.M))
    mirrored = [k for k in defs if hasattr(_lib, k)]
    for k in ("PSE_FP64_PLAIN", "PSE_FP32_FP64ACC", "PSE_FP32_COMPENSATED", "PSE_THREAD_PER_TET",
              "PSE_WARP_COOPERATIVE", "PSE_BINNED_PERSISTENT", "PSE_WARP_PER_TET"):
        assert k in mirrored, k
    for k in mirrored:
        assert getattr(_lib, k) == int(defs[k]), k


def test_compensated_accumulation_needs_overwrite(L):
    """The compensated FP32 pairs start from a cleared output: accumulate = 1 is refused
    before any device work."""
    lat = _lib.Lattice()
    lat.n[0] = lat.n[1] = lat.n[2] = 4
    lat.box = 1.0
    lat.periodic = 1
    lat.particle_mass = 1.0 / 64
    o = _lib.DepositOpts()
    o.precision = _lib.PSE_FP32_COMPENSATED
    o.schedule = _lib.PSE_WARP_COOPERATIVE
    o.accumulate = 1
    g = (ctypes.c_int64 * 3)(4, 4, 4)
    rc = L.pse_deposit_uniform(ctypes.c_void_p(16), ctypes.byref(lat), g, ctypes.c_void_p(16), ctypes.byref(o),
                               None, None, 0, None)
    assert rc == _lib.PSE_ERR_UNSUPPORTED
    assert b"compensated" in L.pse_last_error()


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.lib_path()], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\sT\s+(pse_\w+)", out.stdout))
    for s in declared_symbols():
        assert s in exported, s
        assert hasattr(L, s)


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "pse.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(pse_lattice), offsetof(pse_lattice, particle_mass),
         offsetof(pse_lattice, periodic), offsetof(pse_lattice, box));
  printf("%zu %zu %zu %zu\n", sizeof(pse_deposit_opts), offsetof(pse_deposit_opts, guard_eps),
         offsetof(pse_deposit_opts, d_cube_ids), offsetof(pse_deposit_opts, n_cube_ids));
  printf("%zu %zu %zu %zu %zu\n", sizeof(pse_deposit_stats), offsetof(pse_deposit_stats, bin_counts),
         offsetof(pse_deposit_stats, mass_dropped), offsetof(pse_deposit_stats, overlapped_cells),
         offsetof(pse_deposit_stats, mass_out));
  printf("%zu %zu %zu %zu %zu\n", sizeof(pse_tuning), offsetof(pse_tuning, split_cells),
         offsetof(pse_tuning, chunk_cells), offsetof(pse_tuning, use_graph), offsetof(pse_tuning, guard_list_cap));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), "-o", str(exe), str(src)], check=True)
    got = [list(map(int, l.split())) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                              check=True).stdout.split("\n") if l.strip()]
    La, O, S = _lib.Lattice, _lib.DepositOpts, _lib.DepositStats
    assert got[0] == [ctypes.sizeof(La), La.particle_mass.offset, La.periodic.offset, La.box.offset]
    assert got[1] == [ctypes.sizeof(O), O.guard_eps.offset, O.d_cube_ids.offset, O.n_cube_ids.offset]
    assert got[2] == [ctypes.sizeof(S), S.bin_counts.offset, S.mass_dropped.offset, S.overlapped_cells.offset,
                      S.mass_out.offset]
    Tu = _lib.Tuning
    assert got[3] == [ctypes.sizeof(Tu), Tu.split_cells.offset, Tu.chunk_cells.offset, Tu.use_graph.offset,
                      Tu.guard_list_cap.offset]
    assert got[3][0] == 40  # the field took a reserved slot: the struct keeps its size


def test_abi_version(L):
    assert L.pse_abi_version() == 2


def test_invalid_arguments_return_codes(L):
    lat = _lib.Lattice()
    lat.n[:] = (8, 8, 8)
    lat.box = 1.0
    lat.periodic = 1
    lat.particle_mass = 1.0 / 512
    g = (ctypes.c_int64 * 3)(16, 16, 16)
    rc = L.pse_deposit_uniform(None, ctypes.byref(lat), g, None, None, None, None, 0, None)
    assert rc == _lib.PSE_ERR_INVALID_ARG
    assert "non-NULL" in L.pse_last_error().decode()
    bad = (ctypes.c_int64 * 3)(16, 0, 16)
    rc = L.pse_deposit_uniform(ctypes.c_void_p(16), ctypes.byref(lat), bad, ctypes.c_void_p(16), None, None, None, 0,
                               None)
    assert rc == _lib.PSE_ERR_INVALID_ARG and "grid_n[1]" in L.pse_last_error().decode()
    lat.n[1] = 1
    rc = L.pse_deposit_uniform(ctypes.c_void_p(16), ctypes.byref(lat), g, ctypes.c_void_p(16), None, None, None, 0,
                               None)
    assert rc == _lib.PSE_ERR_INVALID_ARG
    lat.n[1] = 8
    o = _lib.DepositOpts()
    o.precision = 7
    rc = L.pse_deposit_uniform(ctypes.c_void_p(16), ctypes.byref(lat), g, ctypes.c_void_p(16), ctypes.byref(o), None,
                               None, 0, None)
    assert rc == _lib.PSE_ERR_INVALID_ARG and "precision" in L.pse_last_error().decode()
    o.precision = _lib.PSE_FP64_PLAIN
    o.schedule = _lib.PSE_WARP_COOPERATIVE
    rc = L.pse_deposit_uniform(ctypes.c_void_p(16), ctypes.byref(lat), g, ctypes.c_void_p(16), ctypes.byref(o), None,
                               None, 0, None)
    assert rc == _lib.PSE_ERR_UNSUPPORTED
    rc = L.pse_deposit_tets(None, None, -1, 1.0, 1, g, ctypes.c_void_p(16), None, None, None, 0, None)
    assert rc == _lib.PSE_ERR_INVALID_ARG


def test_workspace_size(L):
    assert L.pse_workspace_size(_lib.PSE_OP_DEPOSIT_UNIFORM, None, None) >= 64
    assert L.pse_workspace_size(12345, None, None) == 0
    # the binned schedule needs room for its queue of split tetrahedra
    import paper_1612_09491_gb300 as pse
    plain = pse.workspace_size(_lib.PSE_OP_DEPOSIT_UNIFORM, schedule=_lib.PSE_WARP_COOPERATIVE)
    binned = pse.workspace_size(_lib.PSE_OP_DEPOSIT_UNIFORM, schedule=_lib.PSE_BINNED_PERSISTENT)
    assert plain == L.pse_workspace_size(_lib.PSE_OP_DEPOSIT_UNIFORM, None, None)
    assert binned > plain + (1 << 20)
    # the thread-per-tetrahedron kernels need the header only; the warp kernels add one
    # [12][32]-float residual block per warp of their (capped) persistent grid
    thread = pse.workspace_size(_lib.PSE_OP_DEPOSIT_UNIFORM, schedule=_lib.PSE_THREAD_PER_TET)
    assert 64 <= thread < 4096
    assert plain >= thread + 1024 * 4 * 12 * 32 * 4
    oct_warp = pse.workspace_size(_lib.PSE_OP_DEPOSIT_OCTREE)
    oct_thread = pse.workspace_size(_lib.PSE_OP_DEPOSIT_OCTREE, schedule=_lib.PSE_THREAD_PER_TET)
    assert oct_thread == thread and oct_warp == plain


def test_octree_leaf_validation_needs_no_gpu(L):
    import numpy as np
    st = _lib.Octree()
    bad = np.array([[1, 0, 0, 0]], np.int32)  # one octant does not tile the box
    rc = L.pse_octree_from_leaves(bad.ctypes.data_as(ctypes.c_void_p), 1, 4, 1, 1.0, ctypes.byref(st))
    assert rc == _lib.PSE_ERR_INVALID_ARG and "tile" in L.pse_last_error().decode()
    ovl = np.array([[0, 0, 0, 0], [1, 0, 0, 0]], np.int32)
    rc = L.pse_octree_from_leaves(ovl.ctypes.data_as(ctypes.c_void_p), 2, 4, 1, 1.0, ctypes.byref(st))
    assert rc == _lib.PSE_ERR_INVALID_ARG and "overlap" in L.pse_last_error().decode()
    rc = L.pse_octree_from_leaves(bad.ctypes.data_as(ctypes.c_void_p), 1, 0, 1, 1.0, ctypes.byref(st))
    assert rc == _lib.PSE_ERR_INVALID_ARG
