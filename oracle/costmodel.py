"""FP64 reference of the learned cost model -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module.  It restates, in plain numpy float64, what
the CUDA cost-model kernels compute, so that the tests can check them:

* ``features``: the 16 geometric features of one tetrahedron (grid units);
* ``forward`` / ``backward``: the MLP 16 -> 64 -> 64 -> 2 with ReLU, on standardised
  features, and the gradient of the mean squared error;
* ``adam``: one Adam update.

The paper has no cost model.  It motivates load balancing by the spread of work per
tetrahedron (Sec. 5, Sec. 6.2).  The network, its features and its labels (overlapped
cells, partial clips) are this project's design.  The pins are closed-form features
of the Kuhn tetrahedron and central finite differences of the loss; see
tests/test_oracle_costmodel.py.
"""
from __future__ import annotations

import math

import numpy as np

N_FEAT = 16
H = 64
N_OUT = 2

_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
_FACES = ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1))


def features(v) -> np.ndarray:
    """Features of a tetrahedron with vertices v [4, 3] in grid units (cell side 1).

    0-2  bounding-box extent per axis
    3-5  offset of the bounding box's low corner inside its cell (fractional part)
    6    log2 of the bounding-box cell count
    7    log2 of the volume (floored at 1e-30)
    8    log2 of the surface area (floored at 1e-30)
    9-11 longest, shortest and mean edge length
    12   log2 of the conditioning estimate kappa = sum_f |N_f| * L_max / |6V| (at least 1)
    13   volume over bounding-box volume (0 for a flat box)
    14   log2 of longest over shortest edge (shortest floored at 1e-30)
    15   cube root of the volume over the mean edge length
    """
    v = np.asarray(v, dtype=np.float64)
    lo, hi = v.min(0), v.max(0)
    ext = hi - lo
    ncell = float(np.prod(np.floor(hi) - np.floor(lo) + 1.0))
    d6 = abs(float(np.linalg.det(v[1:] - v[0])))
    vol = d6 / 6.0
    nf = [np.cross(v[b] - v[a], v[c] - v[a]) for a, b, c in _FACES]
    area = 0.5 * sum(float(np.linalg.norm(n)) for n in nf)
    el = np.array([np.linalg.norm(v[j] - v[i]) for i, j in _EDGES])
    lmax, lmin, lmean = float(el.max()), float(el.min()), float(el.mean())
    kappa = (2.0 * area) * lmax / d6 if d6 > 0 else math.inf
    f = np.empty(N_FEAT)
    f[0:3] = ext
    f[3:6] = lo - np.floor(lo)
    f[6] = math.log2(ncell)
    f[7] = math.log2(max(vol, 1e-30))
    f[8] = math.log2(max(area, 1e-30))
    f[9], f[10], f[11] = lmax, lmin, lmean
    f[12] = math.log2(max(kappa, 1.0)) if math.isfinite(kappa) else 128.0
    box = float(np.prod(ext))
    f[13] = vol / box if box > 0 else 0.0
    f[14] = math.log2(lmax / max(lmin, 1e-30))
    f[15] = vol ** (1.0 / 3.0) / lmean if lmean > 0 else 0.0
    return f


def init(seed: int = 0):
    """He-style initial parameters (float64 dict)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0, math.sqrt(2.0 / N_FEAT), (H, N_FEAT)), "b1": np.zeros(H),
        "W2": rng.normal(0, math.sqrt(2.0 / H), (H, H)), "b2": np.zeros(H),
        "W3": rng.normal(0, math.sqrt(1.0 / H), (N_OUT, H)), "b3": np.zeros(N_OUT),
    }


def forward(p, z):
    """z: standardised features [B, 16].  Returns (y [B, 2], cache)."""
    a1 = z @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (z, a1, h1, a2, h2)


def loss(p, z, t) -> float:
    """Mean squared error over the batch and both outputs: (1 / (2B)) sum (y - t)^2."""
    y, _ = forward(p, z)
    return float(np.sum((y - t) ** 2) / (2 * len(z)))


def backward(p, z, t):
    """Gradient of loss() with respect to every parameter (float64 dict)."""
    y, (z, a1, h1, a2, h2) = forward(p, z)
    dy = (y - t) / len(z)                     # d loss / d y  (the 1/2 cancels the square's 2)
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dh2 = (dy @ p["W3"]) * (a2 > 0)
    g["W2"], g["b2"] = dh2.T @ h1, dh2.sum(0)
    dh1 = (dh2 @ p["W2"]) * (a1 > 0)
    g["W1"], g["b1"] = dh1.T @ z, dh1.sum(0)
    return g


def adam(p, m, v, g, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update in place (step counts from 1)."""
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] ** 2
        mh = m[k] / (1 - b1 ** step)
        vh = v[k] / (1 - b2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
