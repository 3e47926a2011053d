"""The collapsed-region input recipe (pse_inputs.collapse_positions), on CPU: a single region
scales offsets from its centre by f inside R, leaves everything beyond R2 in place, is
continuous across both radii (no tetrahedron tears), and is seeded."""
from __future__ import annotations

import numpy as np

from pse_inputs import collapse_positions, lattice_positions


def _one_region(pos, R, R2, f, seed):
    # the centre the generator draws for one region with this seed
    c = np.random.Generator(np.random.PCG64(seed)).random((1, 3))[0]
    return collapse_positions(pos, 1, R, R2, f, seed), c


def test_single_region_recipe():
    n = 48
    pos = lattice_positions(n, offset=0.5)
    R, R2, f = 0.12, 0.2, 0.35
    out, c = _one_region(pos, R, R2, f, seed=5)
    d = pos.astype(np.float64) - c
    d -= np.round(d)
    r = np.linalg.norm(d, axis=1)
    d2 = out.astype(np.float64) - c
    d2 -= np.round(d2)
    r2 = np.linalg.norm(d2, axis=1)
    far = r >= R2
    np.testing.assert_allclose(out[far], pos[far], rtol=0, atol=1e-7)
    core = (r < R) & (r > 0)
    np.testing.assert_allclose(r2[core], f * r[core], rtol=1e-5, atol=1e-7)
    shell = (r >= R) & (r < R2)
    expect = f * R + (r[shell] - R) * (R2 - f * R) / (R2 - R)
    np.testing.assert_allclose(r2[shell], expect, rtol=1e-5, atol=1e-7)
    # radial map: directions are kept
    cosang = np.sum(d[core | shell] * d2[core | shell], axis=1) / (r[core | shell] * r2[core | shell])
    assert np.all(cosang > 1 - 1e-6)


def test_map_is_continuous_and_seeded():
    n = 64
    pos = lattice_positions(n, offset=0.5)
    R, R2, f = 0.1, 0.16, 0.35
    a = collapse_positions(pos, 4, R, R2, f, seed=9)
    np.testing.assert_array_equal(a, collapse_positions(pos, 4, R, R2, f, seed=9))
    # neighbouring particles stay neighbours: one region's map has Lipschitz constant
    # L = max(1, ramp slope (R2 - f R) / (R2 - R)); regions applied in turn multiply it
    L = max(1.0, (R2 - f * R) / (R2 - R))
    for regions, bound in ((1, L), (4, L ** 4)):
        g = collapse_positions(pos, regions, R, R2, f, seed=9).reshape(n, n, n, 3).astype(np.float64)
        for axis in range(3):
            step = np.diff(g, axis=axis)
            step -= np.round(step)
            assert np.linalg.norm(step, axis=-1).max() <= bound * (1 + 1e-5) / n
