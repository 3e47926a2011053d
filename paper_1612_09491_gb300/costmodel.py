"""Torch-facing wrappers of the cost-model entry points (pse_costmodel_*, pse_tet_counts).

Marshalling only: features, labels, predictions and training steps run in libpse.so.
The host side picks minibatch rows (numpy) and the feature standardisation.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from . import _dev_ptr, _grid3, _stream_ptr, _torch, lattice

NFEAT = _lib.PSE_COSTMODEL_NFEAT
NPARAMS = _lib.PSE_COSTMODEL_NPARAMS
_H = 64
# offsets in the flat parameter vector (include/pse.h)
OFF = {"mu": 0, "sigma": 16, "W1": 32, "b1": 32 + _H * 16, "W2": 32 + _H * 16 + _H,
       "b2": 32 + _H * 16 + _H + _H * _H, "W3": 32 + _H * 16 + 2 * _H + _H * _H,
       "b3": 32 + _H * 16 + 2 * _H + _H * _H + 2 * _H}
SHAPES = {"mu": (16,), "sigma": (16,), "W1": (_H, 16), "b1": (_H,), "W2": (_H, _H), "b2": (_H,), "W3": (2, _H),
          "b3": (2,)}


def pack(params: dict) -> np.ndarray:
    """dict of arrays (keys of SHAPES) -> flat float32 parameter vector."""
    v = np.zeros(NPARAMS, np.float32)
    for k, o in OFF.items():
        v[o:o + int(np.prod(SHAPES[k]))] = np.asarray(params[k], np.float32).ravel()
    return v


def unpack(v) -> dict:
    v = np.asarray(v)
    return {k: v[o:o + int(np.prod(SHAPES[k]))].reshape(SHAPES[k]).copy() for k, o in OFF.items()}


def features(pos, n, grid_n, *, box: float = 1.0, periodic: bool = True, stream=None):
    """float32 [T, 16] features of every lattice tetrahedron (pse_costmodel_features)."""
    torch = _torch()
    lat = lattice(n, box, periodic)
    g3, _ = _grid3(grid_n)
    cubes = lat.n[0] * lat.n[1] * lat.n[2] if periodic else (lat.n[0] - 1) * (lat.n[1] - 1) * (lat.n[2] - 1)
    out = torch.empty((6 * cubes, NFEAT), dtype=torch.float32, device=pos.device)
    _lib.check(_lib.load().pse_costmodel_features(_dev_ptr(pos, torch.float32, "pos"), ctypes.byref(lat), g3,
                                                  _dev_ptr(out, torch.float32, "out"), _stream_ptr(stream)))
    return out


def tet_counts(pos, n, grid_n, *, box: float = 1.0, periodic: bool = True, guard_eps: float = 0.0, stream=None):
    """int32 [T, 2] (overlapped cells, partial clips) of every lattice tetrahedron (pse_tet_counts)."""
    torch = _torch()
    lat = lattice(n, box, periodic)
    g3, _ = _grid3(grid_n)
    cubes = lat.n[0] * lat.n[1] * lat.n[2] if periodic else (lat.n[0] - 1) * (lat.n[1] - 1) * (lat.n[2] - 1)
    out = torch.empty((6 * cubes, 2), dtype=torch.int32, device=pos.device)
    _lib.check(_lib.load().pse_tet_counts(_dev_ptr(pos, torch.float32, "pos"), ctypes.byref(lat), g3, guard_eps,
                                          _dev_ptr(out, torch.int32, "out"), _stream_ptr(stream)))
    return out


class CostModel:
    """A device-resident model (pse_costmodel_bytes() bytes of caller memory)."""

    def __init__(self, params=None, device="cuda"):
        torch = _torch()
        L = _lib.load()
        self.buf = torch.zeros(int(L.pse_costmodel_bytes()), dtype=torch.uint8, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        if params is not None:
            self.set(params)

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()

    def set(self, params, stream=None):
        v = pack(params) if isinstance(params, dict) else np.ascontiguousarray(params, np.float32)
        _lib.check(_lib.load().pse_costmodel_set(ctypes.c_void_p(self.ptr), v.ctypes.data_as(ctypes.c_void_p),
                                                 _stream_ptr(stream)))

    def get(self, stream=None):
        """(params, gradient of the last step) as flat float32 vectors."""
        p = np.zeros(NPARAMS, np.float32)
        g = np.zeros(NPARAMS, np.float32)
        _lib.check(_lib.load().pse_costmodel_get(ctypes.c_void_p(self.ptr), p.ctypes.data_as(ctypes.c_void_p),
                                                 g.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
        return p, g

    def predict(self, feat, stream=None):
        torch = _torch()
        out = torch.empty((feat.shape[0], 2), dtype=torch.float32, device=feat.device)
        _lib.check(_lib.load().pse_costmodel_predict(ctypes.c_void_p(self.ptr), _dev_ptr(feat, torch.float32, "feat"),
                                                     feat.shape[0], _dev_ptr(out, torch.float32, "out"),
                                                     _stream_ptr(stream)))
        return out

    def train_step(self, feat, target, lr: float, index=None, batch=None, flags: int = 0, stream=None):
        """One Adam step; returns the device loss tensor (float64 [1], the loss before the update)."""
        torch = _torch()
        b = int(index.shape[0]) if index is not None else int(batch if batch is not None else feat.shape[0])
        _lib.check(_lib.load().pse_costmodel_train_step(
            ctypes.c_void_p(self.ptr), _dev_ptr(feat, torch.float32, "feat"), _dev_ptr(target, torch.float32, "target"),
            _dev_ptr(index, torch.int64, "index") if index is not None else None, b, float(lr), int(flags),
            _dev_ptr(self.loss, torch.float64, "loss"), _stream_ptr(stream)))
        return self.loss


def standardisation(feat_host: np.ndarray):
    """mu, sigma of the features (host numpy); constant features get sigma 1."""
    f = np.asarray(feat_host, np.float64)
    mu = f.mean(0)
    sd = f.std(0)
    sd[sd < 1e-6] = 1.0
    return mu.astype(np.float32), sd.astype(np.float32)


def he_init(seed: int = 0) -> dict:
    rng = np.random.default_rng(seed)
    return {"mu": np.zeros(16), "sigma": np.ones(16),
            "W1": rng.normal(0, np.sqrt(2.0 / 16), (_H, 16)), "b1": np.zeros(_H),
            "W2": rng.normal(0, np.sqrt(2.0 / _H), (_H, _H)), "b2": np.zeros(_H),
            "W3": rng.normal(0, np.sqrt(1.0 / _H), (2, _H)), "b3": np.zeros(2)}


def labels(counts):
    """Training targets from tet_counts: log(1 + overlapped cells), log(1 + partial clips)
    (computed on the host, returned on the counts' device)."""
    torch = _torch()
    t = np.log1p(counts.cpu().numpy().astype(np.float64)).astype(np.float32)
    return torch.from_numpy(t).to(counts.device)


def fit(model: CostModel, feat, target, steps: int, batch: int = 4096, lr: float = 3e-3, seed: int = 0,
        stream=None) -> list:
    """Minibatch Adam on (feat, target); rows drawn on the host.  Returns the loss every 100 steps."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    n = feat.shape[0]
    hist = []
    idx_host = torch.empty(batch, dtype=torch.int64).pin_memory()
    idx = torch.empty(batch, dtype=torch.int64, device=feat.device)
    for s in range(steps):
        idx_host.numpy()[:] = rng.integers(0, n, batch)
        idx.copy_(idx_host, non_blocking=False)
        loss = model.train_step(feat, target, lr, index=idx, stream=stream)
        if s % 100 == 0 or s == steps - 1:
            hist.append(float(loss.item()))
    return hist
