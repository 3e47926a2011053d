"""Cell-mass error measures used to state the accuracy of every result.

max_rel: max_c |M[c] - R[c]| / max(R[c], floor * Mbar)   (floor = 1e-3)
l1:      sum_c |M[c] - R[c]| / sum_c R[c]
mass:    |sum M - sum R| / sum R

Mbar is the mean reference mass of the cells that hold mass (for a full lattice
deposit every cell does, and Mbar is the plain mean cell mass).

Sparse deposits (a few tetrahedra, a subset of cubes) leave cells that hold only a
sliver of one tetrahedron; a clip's rounding error scales with the mass of a full
cell at that tetrahedron's density, not with the sliver.  For those, floor_mass
(a scalar or one value per cell) replaces floor * Mbar in the denominator.
"""
from __future__ import annotations

import numpy as np


def cell_errors(m, ref, floor: float = 1e-3, floor_mass=None) -> dict:
    m = np.asarray(m, dtype=np.float64).ravel()
    r = np.asarray(ref, dtype=np.float64).ravel()
    d = np.abs(m - r)
    tot = r.sum()
    occupied = int(np.count_nonzero(r))
    mean = tot / max(occupied, 1)
    if floor_mass is not None:
        fm = np.asarray(floor_mass, dtype=np.float64)
        den = np.maximum(r, fm.ravel() if fm.ndim else float(fm))
        den = np.where(den > 0, den, 1.0)
    else:
        den = np.maximum(r, floor * mean) if mean > 0 else np.ones_like(r)
    return {
        "max_rel": float((d / den).max()) if d.size else 0.0,
        "l1": float(d.sum() / tot) if tot > 0 else float(d.sum()),
        "mass": float(abs(m.sum() - tot) / tot) if tot > 0 else float(abs(m.sum())),
    }
