"""ctypes binding of the C ABI in include/pse.h (argument marshalling only).

Every step of the deposit runs in libpse.so's CUDA kernels; this module only
turns torch tensors into device pointers and the current CUDA stream into the
``stream`` argument.  If the library has not been built, importing the functions
raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PSE_OK = 0
PSE_ERR_INVALID_ARG = -1
PSE_ERR_CUDA = -2
PSE_ERR_OOM = -3
PSE_ERR_TIMEOUT = -4
PSE_ERR_UNSUPPORTED = -5
PSE_ERR_WORKSPACE = -6
PSE_ERR_DEVICE = -7

PSE_FP64_PLAIN = 0
PSE_FP32_FP64ACC = 1
PSE_FP32_COMPENSATED = 2
PSE_THREAD_PER_TET = 0
PSE_WARP_COOPERATIVE = 1
PSE_BINNED_PERSISTENT = 2
PSE_WARP_PER_TET = 3

PSE_OP_DEPOSIT_UNIFORM = 1
PSE_OP_DEPOSIT_OCTREE = 2
PSE_OP_BUILD_OCTREE = 3
PSE_OP_DEPOSIT_TETS = 4
PSE_COSTMODEL_NFEAT = 16
PSE_COSTMODEL_NPARAMS = 5410
PSE_TRAIN_FP32 = 1
PSE_TRAIN_GRAD_ONLY = 2

# every symbol include/pse.h declares (checked by the tests)
EXPORTED = (
    "pse_build_tets_from_lagrangian_grid",
    "pse_deposit_uniform",
    "pse_deposit_tets",
    "pse_octree_from_leaves",
    "pse_build_octree_from_tet_sizes",
    "pse_deposit_octree",
    "pse_free_octree",
    "pse_build_octree_leaves_noalloc",
    "pse_build_octree_count",
    "pse_octree_restrict",
    "pse_deposit_uniform_streamed",
    "pse_deposit_octree_streamed",
    "pse_build_octree_streamed",
    "pse_microbench_fma",
    "pse_microbench_red",
    "pse_costmodel_bytes",
    "pse_costmodel_set",
    "pse_costmodel_get",
    "pse_costmodel_features",
    "pse_tet_counts",
    "pse_costmodel_predict",
    "pse_costmodel_train_step",
    "pse_workspace_size",
    "pse_last_error",
    "pse_abi_version",
)


class Lattice(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64 * 3), ("box", ctypes.c_double), ("periodic", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("particle_mass", ctypes.c_double)]


class DepositOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("schedule", ctypes.c_int32), ("cost_model", ctypes.c_void_p),
                ("tuning", ctypes.c_void_p), ("guard_eps", ctypes.c_double), ("spin_limit", ctypes.c_int64),
                ("accumulate", ctypes.c_int32), ("mass_fixup", ctypes.c_int32), ("d_cube_ids", ctypes.c_void_p),
                ("n_cube_ids", ctypes.c_int64)]


class DepositStats(ctypes.Structure):
    _fields_ = [("tets", ctypes.c_uint64), ("bbox_cells", ctypes.c_uint64), ("inside_cells", ctypes.c_uint64),
                ("partial_clips", ctypes.c_uint64), ("fp64_redos", ctypes.c_uint64),
                ("degenerate_tets", ctypes.c_uint64), ("single_cell_tets", ctypes.c_uint64),
                ("bin_counts", ctypes.c_uint64 * 8), ("mass_in", ctypes.c_double), ("mass_dropped", ctypes.c_double),
                ("inverted_tets", ctypes.c_uint64), ("overlapped_cells", ctypes.c_uint64),
                ("column_runs", ctypes.c_uint64), ("mass_out", ctypes.c_double)]

    def to_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "bin_counts"}
        d["bin_counts"] = list(self.bin_counts)
        return d


class Octree(ctypes.Structure):
    _fields_ = [("bc", ctypes.c_int32), ("max_level", ctypes.c_int32), ("n_leaves", ctypes.c_int64),
                ("box", ctypes.c_double), ("d_leaves", ctypes.c_void_p), ("d_fine_map", ctypes.c_void_p),
                ("h_leaves", ctypes.c_void_p), ("n_cells", ctypes.c_int64)]


class Tuning(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("split_cells", ctypes.c_int32), ("chunk_cells", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("guard_list_cap", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class PseError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pse error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """The loaded libpse.so.  Raises if it is missing (build it with build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: the CUDA library has not been built "
                                   "(run paper_1612_09491_gb300.build.build())")
            _build.build()
        L = ctypes.CDLL(path)
        vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
        L.pse_build_tets_from_lagrangian_grid.argtypes = [vp, ctypes.POINTER(Lattice), vp, vp, i64p, vp]
        L.pse_deposit_uniform.argtypes = [vp, ctypes.POINTER(Lattice), i64p, vp, ctypes.POINTER(DepositOpts),
                                          ctypes.POINTER(DepositStats), vp, ctypes.c_size_t, vp]
        L.pse_deposit_tets.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_int32, i64p, vp,
                                       ctypes.POINTER(DepositOpts), ctypes.POINTER(DepositStats), vp, ctypes.c_size_t,
                                       vp]
        OP = ctypes.POINTER(Octree)
        L.pse_octree_from_leaves.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, OP]
        L.pse_build_octree_from_tet_sizes.argtypes = [vp, ctypes.POINTER(Lattice), ctypes.c_int32, ctypes.c_int32,
                                                      ctypes.c_double, OP, vp, ctypes.c_size_t, vp]
        L.pse_deposit_octree.argtypes = [vp, ctypes.POINTER(Lattice), OP, vp, ctypes.POINTER(DepositOpts),
                                         ctypes.POINTER(DepositStats), vp, ctypes.c_size_t, vp]
        L.pse_free_octree.argtypes = [OP]
        L.pse_free_octree.restype = None
        L.pse_build_octree_leaves_noalloc.argtypes = [vp, ctypes.POINTER(Lattice), ctypes.c_int32, ctypes.c_int32,
                                                      ctypes.c_double, vp, ctypes.c_int64, vp, vp]
        L.pse_build_octree_leaves_noalloc.restype = ctypes.c_int
        L.pse_build_octree_count.argtypes = [vp, ctypes.POINTER(Lattice), ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_int32, OP, vp]
        L.pse_build_octree_count.restype = ctypes.c_int
        L.pse_octree_restrict.argtypes = [OP, vp, vp, vp]
        L.pse_octree_restrict.restype = ctypes.c_int
        L.pse_deposit_uniform_streamed.argtypes = [vp, ctypes.POINTER(Lattice), ctypes.c_int64,
                                                   ctypes.POINTER(ctypes.c_int64), vp, ctypes.POINTER(DepositOpts),
                                                   ctypes.POINTER(DepositStats), vp, ctypes.c_size_t, vp]
        L.pse_deposit_uniform_streamed.restype = ctypes.c_int
        L.pse_deposit_octree_streamed.argtypes = [vp, ctypes.POINTER(Lattice), ctypes.c_int64, OP, vp,
                                                  ctypes.POINTER(DepositOpts), ctypes.POINTER(DepositStats), vp,
                                                  ctypes.c_size_t, vp]
        L.pse_deposit_octree_streamed.restype = ctypes.c_int
        L.pse_build_octree_streamed.argtypes = [vp, ctypes.POINTER(Lattice), ctypes.c_int64, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_double, OP, vp]
        L.pse_build_octree_streamed.restype = ctypes.c_int
        L.pse_microbench_fma.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, vp]
        L.pse_microbench_fma.restype = ctypes.c_int
        L.pse_microbench_red.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, vp]
        L.pse_microbench_red.restype = ctypes.c_int
        L.pse_costmodel_bytes.argtypes = []
        L.pse_costmodel_bytes.restype = ctypes.c_size_t
        L.pse_costmodel_set.argtypes = [vp, vp, vp]
        L.pse_costmodel_set.restype = ctypes.c_int
        L.pse_costmodel_get.argtypes = [vp, vp, vp, vp]
        L.pse_costmodel_get.restype = ctypes.c_int
        L.pse_costmodel_features.argtypes = [vp, ctypes.POINTER(Lattice), ctypes.POINTER(ctypes.c_int64), vp, vp]
        L.pse_costmodel_features.restype = ctypes.c_int
        L.pse_tet_counts.argtypes = [vp, ctypes.POINTER(Lattice), ctypes.POINTER(ctypes.c_int64), ctypes.c_double,
                                     vp, vp]
        L.pse_tet_counts.restype = ctypes.c_int
        L.pse_costmodel_predict.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
        L.pse_costmodel_predict.restype = ctypes.c_int
        L.pse_costmodel_train_step.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.c_int32, vp, vp]
        L.pse_costmodel_train_step.restype = ctypes.c_int
        L.pse_workspace_size.argtypes = [ctypes.c_int, ctypes.POINTER(Lattice), vp]
        L.pse_workspace_size.restype = ctypes.c_size_t
        L.pse_last_error.argtypes = []
        L.pse_last_error.restype = ctypes.c_char_p
        L.pse_abi_version.argtypes = []
        for name in ("pse_build_tets_from_lagrangian_grid", "pse_deposit_uniform", "pse_deposit_tets",
                     "pse_octree_from_leaves", "pse_build_octree_from_tet_sizes", "pse_deposit_octree",
                     "pse_abi_version"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return _lib


def check(rc: int):
    if rc != PSE_OK:
        raise PseError(rc, load().pse_last_error().decode())
