"""Seeded particle-position generators.

Particles sit on a periodic Lagrangian lattice of ``n^3`` points in a box of side
``box`` (the tracer arrangement of the paper's Sec. 2: tracers start on the
vertices of a regular grid and then move).  The flat particle index is
``p = i + n*(j + n*k)`` (x fastest), which is how the particle IDs order the
data once they have been sorted (Sec. 3).  Positions are returned as float32
``[n^3, 3]`` arrays, wrapped into ``[0, box)``.

Three families of positions:

* ``lattice_positions``: the undisplaced lattice (every tetrahedron has the same
  density, so every deposit cell must receive exactly the same mass).
* ``zeldovich_positions``: a Zel'dovich displacement field of a Gaussian random
  field with a power-law density spectrum P(k) ~ k^index, scaled to a stated rms
  displacement in lattice spacings.  This stands in for the N-body snapshots the
  paper deposits (Dark Sky early data release, Sec. 7), which are not available.
* ``jitter_positions``: the paper's weak-scaling input (Sec. 7.2): lattice plus
  independent uniform offsets of up to one lattice spacing per axis.
* ``collapse_positions``: a Zel'dovich field with collapsed regions added, so that the
  tetrahedra span a wide range of sizes and a tree refined by tetrahedron size is genuinely
  adaptive (the Zel'dovich field alone is quasi-linear: its tetrahedra are too alike in size
  for the octree to stop above the finest level anywhere but everywhere).  Around each of a
  few seeded centres, the offset d from the centre (minimum image) is scaled radially: by f
  inside the Lagrangian radius R (a uniform core f^-3 times denser), then linearly in |d| from
  f R at R to R2 at R2 (an underdense shell), unchanged beyond R2.  The map is continuous,
  so no tetrahedron tears; regions are applied one after another.

Recipe for the Zel'dovich field (the reading used throughout this project):
white noise w ~ N(0,1) on the n^3 lattice (numpy PCG64, the given seed);
delta_k = sqrt(P(|k|)) * FFT(w) with P(k) = |k|^index (k in integer
wavenumbers), delta_0 = 0 and every mode on a Nyquist plane set to 0;
psi_k = i k delta_k / |k|^2; psi = IFFT(psi_k), rescaled so that the rms of the
3-vector |psi| equals ``rms_disp`` lattice spacings; x = q + psi mod box.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class WorkloadConfig:
    """One synthetic workload: lattice, displacement field and deposit grid."""

    index: int
    name: str
    n: int  # particles per side
    spectral_index: float
    rms_disp: float  # rms displacement in lattice spacings
    grid: str  # "uniform" or "octree"
    grid_n: int  # uniform: cells per side; octree: finest equivalent cells per side
    bc: int = 0  # octree: cells per leaf block side
    max_level: int = 0  # octree: deepest refinement level
    collapse: tuple = ()  # (regions, R, R2, f) of collapse_positions, box units; () = none

    @property
    def seed(self) -> int:
        return 1000 + self.index

    @property
    def n_tets(self) -> int:
        return 6 * self.n ** 3


CONFIGS = {
    1: WorkloadConfig(1, "plain-32c-grid64", 32, -2.0, 0.5, "uniform", 64),
    2: WorkloadConfig(2, "precision-128c-grid256", 128, -2.0, 2.0, "uniform", 256),
    3: WorkloadConfig(3, "batching-256c-octree16", 256, -1.5, 4.0, "octree", 256, bc=16, max_level=4),
    4: WorkloadConfig(4, "learned-512c-grid512", 512, -1.5, 4.0, "uniform", 512),
    5: WorkloadConfig(5, "scale-1024c-octree128", 1024, -2.0, 3.0, "octree", 2048, bc=128, max_level=4),
    # the 1024^3 workload's geometry at 1/64 of its size: 2 finest cells per lattice spacing and
    # the same spectrum; with P(k) ~ k^-2 the strain variance at a fixed rms displacement (in
    # spacings) grows as 1/n, so rms 1.5 at 256^3 matches rms 3 at 1024^3.  The case that
    # profilers capture in full.
    6: WorkloadConfig(6, "profile-256c-octree32", 256, -2.0, 1.5, "octree", 512, bc=32, max_level=4),
    # workload 6's field with 8 collapsed regions, on 4 finest cells per lattice spacing: field
    # tetrahedra stop refining at level 3, the collapsed cores refine to level 4
    7: WorkloadConfig(7, "halos-256c-octree64", 256, -2.0, 1.5, "octree", 1024, bc=64, max_level=4,
                      collapse=(8, 0.1, 0.16, 0.35)),
}


def _lagrangian_q(n: int, box: float, offset: float) -> np.ndarray:
    dq = box / n
    ax = (np.arange(n, dtype=np.float64) + offset) * dq
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")  # x fastest in C order
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def _wrap_f32(x: np.ndarray, box: float) -> np.ndarray:
    x = np.mod(x, box)
    out = x.astype(np.float32)
    out[out >= np.float32(box)] = 0.0  # float32 rounding may land exactly on box
    out[out < 0] = 0.0
    return np.ascontiguousarray(out)


def lattice_positions(n: int, box: float = 1.0, offset: float = 0.0) -> np.ndarray:
    """Undisplaced lattice q = (i + offset) * box / n, float32 [n^3, 3]."""
    return _wrap_f32(_lagrangian_q(n, box, offset), box)


def jitter_positions(n: int, seed: int, amp: float = 1.0, box: float = 1.0) -> np.ndarray:
    """Lattice plus independent U(-amp, amp) lattice-spacing offsets per axis (Sec. 7.2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = _lagrangian_q(n, box, 0.0)
    dq = box / n
    return _wrap_f32(q + rng.uniform(-amp, amp, size=q.shape) * dq, box)


def zeldovich_displacement(n: int, spectral_index: float, rms_disp: float, seed: int,
                           box: float = 1.0) -> np.ndarray:
    """Zel'dovich displacement field psi (float64 [n^3, 3], box units), recipe in the module doc."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n, n, n))  # axes (z, y, x), x fastest
    wk = np.fft.rfftn(w)
    del w
    kz = np.fft.fftfreq(n, d=1.0 / n)[:, None, None]
    ky = np.fft.fftfreq(n, d=1.0 / n)[None, :, None]
    kx = np.fft.rfftfreq(n, d=1.0 / n)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = np.power(k2, 0.5 * spectral_index) ** 0.5  # sqrt(P(k)), P = k^index
    nyq = n // 2
    kill = (np.abs(kx) == nyq) | (np.abs(ky) == nyq) | (np.abs(kz) == nyq)
    delta_k = wk * amp
    delta_k[0, 0, 0] = 0.0
    delta_k = np.where(kill, 0.0, delta_k)
    psi = np.empty((n ** 3, 3), dtype=np.float64)
    for a, ka in enumerate((kx, ky, kz)):
        comp = np.fft.irfftn(1j * ka / k2 * delta_k, s=(n, n, n), axes=(0, 1, 2))
        psi[:, a] = comp.ravel()
    rms = np.sqrt(np.mean(np.sum(psi * psi, axis=1)))
    dq = box / n
    if rms > 0:
        psi *= rms_disp * dq / rms
    return psi


def zeldovich_positions(n: int, spectral_index: float, rms_disp: float, seed: int,
                        box: float = 1.0) -> np.ndarray:
    """x = q + psi(q) wrapped into [0, box), float32 [n^3, 3]."""
    psi = zeldovich_displacement(n, spectral_index, rms_disp, seed, box)
    return _wrap_f32(_lagrangian_q(n, box, 0.0) + psi, box)


def collapse_positions(pos: np.ndarray, regions: int, radius: float, radius2: float, factor: float, seed: int,
                       box: float = 1.0) -> np.ndarray:
    """`pos` (float32 [N, 3] in [0, box)) with `regions` collapsed regions at seeded centres (the
    recipe in the module doc; radii in box units), float32 [N, 3] wrapped into [0, box)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = pos.astype(np.float64)
    for c in rng.random((regions, 3)) * box:
        d = x - c
        d -= box * np.round(d / box)
        r = np.linalg.norm(d, axis=1)
        s = np.ones_like(r)
        s[r < radius] = factor
        ramp = (r >= radius) & (r < radius2)
        s[ramp] = (factor * radius + (r[ramp] - radius) * (radius2 - factor * radius) / (radius2 - radius)) / r[ramp]
        x += d * (s - 1.0)[:, None]
    return _wrap_f32(x, box)


def config_positions(cfg: WorkloadConfig | int, box: float = 1.0) -> np.ndarray:
    """Positions of one of the numbered workloads (seed = 1000 + index)."""
    if isinstance(cfg, int):
        cfg = CONFIGS[cfg]
    pos = zeldovich_positions(cfg.n, cfg.spectral_index, cfg.rms_disp, cfg.seed, box)
    if cfg.collapse:
        regions, r1, r2, f = cfg.collapse
        pos = collapse_positions(pos, regions, r1 * box, r2 * box, f, cfg.seed + 1, box)
    return pos


def random_dyadic_tets(count: int, seed: int, span: float = 3.0, denom_bits: int = 6,
                       origin: float = 0.0) -> np.ndarray:
    """Random tetrahedra with dyadic coordinates (exact in float32 and float64).

    Coordinates are multiples of 2^-denom_bits in [origin, origin + span); returned as
    float64 [count, 4, 3].  Degenerate (zero-volume) draws are re-drawn.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    scale = 2.0 ** denom_bits
    out = np.empty((count, 4, 3), dtype=np.float64)
    i = 0
    while i < count:
        v = rng.integers(0, int(span * scale), size=(4, 3)).astype(np.float64) / scale + origin
        e = v[1:] - v[0]
        if abs(np.linalg.det(e)) > 1e-9:
            out[i] = v
            i += 1
    return out


def zeldovich_positions_device(n: int, spectral_index: float, rms_disp: float, seed: int, box: float = 1.0,
                               device="cuda", out=None):
    """The Zel'dovich recipe above for the large lattices (512^3, 1024^3), evaluated on the GPU with
    torch.fft in float32: white noise from torch's generator seeded with `seed` (not numpy's, so the
    field differs from zeldovich_positions at the same seed), one displacement component at a time.
    Returns float32 [n^3, 3] on `device` (or fills `out`, which may live in host memory)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    w = torch.randn((n, n, n), generator=g, device=device, dtype=torch.float32)  # axes (z, y, x)
    wk = torch.fft.rfftn(w)
    del w
    kz = torch.fft.fftfreq(n, d=1.0 / n, device=device).view(n, 1, 1)
    ky = torch.fft.fftfreq(n, d=1.0 / n, device=device).view(1, n, 1)
    kx = torch.fft.rfftfreq(n, d=1.0 / n, device=device).view(1, 1, n // 2 + 1)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = torch.pow(k2, 0.25 * spectral_index)  # sqrt(P(k)), P = k^index
    nyq = n // 2
    kill = (kx.abs() == nyq) | (ky.abs() == nyq) | (kz.abs() == nyq)
    wk *= amp
    wk[0, 0, 0] = 0.0
    wk = torch.where(kill, torch.zeros((), dtype=wk.dtype, device=device), wk)
    del amp, kill
    if out is None:
        out = torch.empty((n ** 3, 3), dtype=torch.float32, device=device)
    ms = 0.0
    q = (torch.arange(n, device=device, dtype=torch.float64) * (box / n))
    comps = []
    for a, ka in enumerate((kx, ky, kz)):
        c = torch.fft.irfftn(wk * (1j * ka / k2), s=(n, n, n))
        ms += float((c.double() ** 2).sum()) / n ** 3
        comps.append(c)
        del c
    scale = (rms_disp * box / n) / max(ms, 1e-300) ** 0.5
    for a in range(3):
        shape = [1, 1, 1]
        shape[2 - a] = n
        x = comps[a].double() * scale + q.view(*shape)
        x = torch.remainder(x, box).float()
        x[x >= box] = 0.0
        out[:, a].copy_(x.reshape(-1))
        comps[a] = None
        del x
    return out
