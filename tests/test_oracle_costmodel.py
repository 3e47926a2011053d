"""Pins of the FP64 cost-model reference (oracle/costmodel.py) -- no GPU.

* features of the Kuhn tetrahedron (cell side 1) against their closed forms;
* features under integer and fractional translations;
* the analytic gradient against central finite differences of the loss;
* Adam's first step against its closed form (a step of lr against the gradient's sign).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import costmodel as cm

KUHN = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1]], dtype=np.float64)


def test_kuhn_features_closed_form():
    f = cm.features(KUHN + 0.25)
    assert f[0:3] == pytest.approx([1, 1, 1])
    assert f[3:6] == pytest.approx([0.25, 0.25, 0.25])
    assert f[6] == pytest.approx(3.0)                       # 2 x 2 x 2 cells
    assert f[7] == pytest.approx(math.log2(1 / 6))
    area = 1.0 + math.sqrt(2.0)                             # 1/2 + 1/2 + sqrt(2)/2 + sqrt(2)/2
    assert f[8] == pytest.approx(math.log2(area))
    edges = [1, 1, 1, math.sqrt(2), math.sqrt(2), math.sqrt(3)]
    assert f[9] == pytest.approx(math.sqrt(3))
    assert f[10] == pytest.approx(1.0)
    assert f[11] == pytest.approx(sum(edges) / 6)
    assert f[12] == pytest.approx(math.log2(2 * area * math.sqrt(3) / 1.0))
    assert f[13] == pytest.approx(1 / 6)
    assert f[14] == pytest.approx(math.log2(math.sqrt(3)))
    assert f[15] == pytest.approx((1 / 6) ** (1 / 3) / (sum(edges) / 6))


def test_features_translation():
    rng = np.random.default_rng(3)
    v = rng.uniform(0, 3, (4, 3))
    f = cm.features(v)
    g = cm.features(v + np.array([5, -2, 7]))
    np.testing.assert_allclose(f, g, rtol=1e-12, atol=1e-12)
    h = cm.features(v + 0.125)
    np.testing.assert_allclose(np.delete(f, [3, 4, 5, 6]), np.delete(h, [3, 4, 5, 6]), rtol=1e-12)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    p = cm.init(seed=1)
    z = rng.normal(size=(37, cm.N_FEAT))
    t = rng.normal(size=(37, cm.N_OUT))
    g = cm.backward(p, z, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = cm.loss(p, z, t)
            flat[idx] = old - h
            lm = cm.loss(p, z, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (k, idx)


def test_adam_first_step_closed_form():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    cm.adam(p, m, v, g, step=1, lr=0.01)
    # first step: m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    np.testing.assert_allclose(p["w"], np.array([1.0, -2.0, 0.5]) - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8),
                               rtol=1e-14)
