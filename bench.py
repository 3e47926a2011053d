#!/usr/bin/env python
"""Throughput of the exact tetrahedron deposit on one GB300 (or N replicas).

A step is one pass of the whole hot path over one synthetic lattice: every
tetrahedron of the 6-per-cube tessellation is generated on the fly, classified
against the cells of its bounding box, clipped exactly where partial, and its
mass deposited into the float64 grid (the call overwrites the grid).

Workload (default): 128^3 particles (12,582,912 tetrahedra), Zel'dovich P(k) ~ k^-2
with rms displacement 2 lattice spacings, periodic unit box, uniform 256^3 float64
grid.  Timed arm: FP32 clip with FP64 redo + FP64 accumulation, warp-cooperative
schedule.  Beside it: the plain FP64 one-thread-per-tetrahedron GPU path on the
same GPU, the density error between the two, and the FP64 CPU oracle timed on a
bounded sample of the same workload.

``--impl reference`` times the oracle alone as the reference arm (host cores).
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tetrahedra deposited/sec and tet-cell clips/sec at stated density error vs plain FP64 GPU"
UNIT = "tets/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2

# Algorithmic work per unit for the ALU roofline of the warp-cooperative kernel
# (FP32 floating-point operations, FMA = 2): per tetrahedron the determinant, bounding
# box and face planes (~150); per bounding-box cell one classification against 4 planes
# (~32); per partial clip the intersections and fan integrals of the face polygons
# against the cell's slabs (~620).
FLOP_PER_TET = 150.0
FLOP_PER_BBOX_CELL = 32.0
FLOP_PER_CLIP = 620.0
# From one ncu capture of the tuned deposit kernel (k_warp_coop, 4 blocks of 128 threads
# per SM) on the headline workload: DRAM bytes read + written per launch, and thread
# instructions issued per partial clip (warp instructions x active lanes / partial clips).
# Both go stale when the kernel changes and must be re-taken with it.
DRAM_BYTES_PER_LAUNCH = 300_260_608
THREAD_INST_PER_CLIP = 5182.4
SM_COUNT_GB300 = 152
SM_MAX_MHZ_GB300 = 2070.0  # the part's maximum SM clock
PRECISION = "fp32 clip, fp64 redo of guarded tetrahedra, fp64 accumulation, mass fix-up"
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pse", choices=["pse", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--no-baseline", action="store_true", help="skip the FP64 GPU baseline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


# ---------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.rows = []
        self.proc = None
        self.bus_id = bus_id

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def bus_id_of(dev_index: int):
    import torch
    try:
        p = torch.cuda.get_device_properties(dev_index)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


# ---------------------------------------------------------------- oracle ----
def oracle_rate(pos, cfg, seconds: float, seed: int = 7):
    """Oracle tets/s on a random sample of Lagrangian cubes sized for ~`seconds` of CPU work."""
    import numpy as np

    import oracle
    n = cfg.n
    rng = np.random.default_rng(seed)
    threads = os.cpu_count() or 1
    m = 2048
    while True:  # grow the sample until it takes a quarter of the budget, then extrapolate
        calib = np.sort(rng.choice(n ** 3, size=min(n ** 3, m), replace=False))
        t0 = time.perf_counter()
        oracle.deposit_lattice(pos, n, cfg.grid_n, cube_ids=calib, nthreads=threads)
        dt = time.perf_counter() - t0
        if dt >= 0.25 * seconds or calib.size >= n ** 3:
            break
        m *= 4
    m = int(min(n ** 3, max(calib.size, calib.size * seconds / max(dt, 1e-9))))
    ids = np.sort(rng.choice(n ** 3, size=m, replace=False))
    t0 = time.perf_counter()
    ref, st = oracle.deposit_lattice(pos, n, cfg.grid_n, cube_ids=ids, nthreads=threads)
    dt = time.perf_counter() - t0
    return {"value": 6 * m / dt, "unit": UNIT, "cores": int(st["threads"]), "kind": "oracle",
            "sample": f"{m} random Lagrangian cubes ({6 * m} tetrahedra) of the workload, seed {seed}, "
                      f"{dt:.1f} s"}, ids, ref


def run_reference(args, cfg):
    """The reference arm: the FP64 CPU oracle, each step a bounded sample of the workload."""
    import numpy as np

    import oracle
    from pse_inputs import config_positions
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pos = config_positions(cfg)
    n = cfg.n
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(11)
    calib = np.sort(rng.choice(n ** 3, size=min(n ** 3, 2048), replace=False))
    t0 = time.perf_counter()
    oracle.deposit_lattice(pos, n, cfg.grid_n, cube_ids=calib, nthreads=threads)
    per_cube = (time.perf_counter() - t0) / calib.size
    budget = 150.0 / max(1, args.steps + args.warmup)  # whole run within a few minutes
    m = int(min(n ** 3, max(256, budget / max(per_cube, 1e-9))))
    times = []
    for k in range(args.warmup + args.steps):
        ids = np.sort(rng.choice(n ** 3, size=m, replace=False))
        t0 = time.perf_counter()
        oracle.deposit_lattice(pos, n, cfg.grid_n, cube_ids=ids, nthreads=threads)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = 6 * m / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.name, "particles": f"{n}^3", "grid": f"uniform {cfg.grid_n}^3",
                       "step": f"{m} random Lagrangian cubes per step (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{m} random cubes ({6 * m} tetrahedra) per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- replicas ----
def replica_throughput(step_ms, units_per_rank, dist=None, device="cpu"):
    """Whole-job throughput of N independent replicas: every rank processed units_per_rank
    per step; the step time is the slowest rank's mean (max over ranks).
    Returns (ms_per_step, units per second over all ranks)."""
    import torch
    ms = sum(step_ms) / len(step_ms)
    world = 1
    if dist is not None:
        world = dist.get_world_size()
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms * 1e-3)


# ---------------------------------------------------------- other workloads --
def _timed(step, steps, warmup, flush, stream):
    """CUDA-event times (ms) of `steps` calls of step() after `warmup` untimed ones, L2 flushed between."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def _tet_size_sample(pos, n, g, layers=8):
    """Quantiles of the tetrahedra's mean edge length in cells of a g^3 grid, from the cost-model
    features of `layers` cube layers in the middle of the lattice.  The rows are moved to the
    periodic image nearest their Lagrangian sites and deposited as an open lattice, so no
    tetrahedron of the sample wraps."""
    import numpy as np
    import torch
    k0 = n // 2
    rows = pos[k0 * n * n:(k0 + layers + 1) * n * n].to("cuda", non_blocking=False).view(layers + 1, n, n, 3)
    ax = torch.arange(n, device=rows.device, dtype=torch.float32) / n
    q = torch.stack(torch.broadcast_tensors(ax.view(1, 1, n),
                                            ax.view(1, n, 1),
                                            ((k0 + torch.arange(layers + 1, device=rows.device)) / n)
                                            .float().view(layers + 1, 1, 1)), -1)
    d = rows - q
    d -= torch.round(d)
    x = (q + d).reshape(-1, 3).contiguous()
    from paper_1612_09491_gb300 import costmodel as cm
    e = cm.features(x, (n, n, layers + 1), g, periodic=False)[:, 11]
    e = e[:: max(1, e.numel() // 4_000_000)].cpu().numpy()
    return {"mean_edge_cells_quantiles": dict(zip(("min", "p01", "median", "p99", "max"),
                                                  [float(v) for v in np.quantile(e, [0, .01, .5, .99, 1])])),
            "sample": f"{layers} cube layers in the middle of the lattice, cells of the {g}^3 grid"}


def run_workload(args, cfg):
    """Workloads 3 (octree), 4 (uniform 512^3 with the learned cost model) and 5 (octree over a
    1024^3 lattice streamed from pinned host memory in z-slabs).  One JSON line, like main()."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_09491_gb300 as pse
    from paper_1612_09491_gb300 import autotune
    from paper_1612_09491_gb300 import costmodel as cm
    from paper_1612_09491_gb300.metrics import cell_errors
    from pse_inputs import CONFIGS, config_positions, zeldovich_positions_device

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    prec = pse.PSE_FP32_FP64ACC
    n = cfg.n
    t0 = time.perf_counter()
    if n <= 256:
        pos = torch.from_numpy(config_positions(cfg)).to(dev)
        gen = "numpy PCG64 + FFT on the host"
    else:
        pos = zeldovich_positions_device(n, cfg.spectral_index, cfg.rms_disp, cfg.seed, device=dev)
        gen = "torch generator + torch.fft on the GPU (float32)"
    gen_s = time.perf_counter() - t0
    extra = {"input_generation": f"{gen}, {gen_s:.1f} s"}
    config = {"workload": cfg.name, "particles": f"{n}^3", "tets": cfg.n_tets,
              "spectrum": f"P(k)~k^{cfg.spectral_index}", "rms_disp_spacings": cfg.rms_disp,
              "precision": PRECISION,
              "l2": "512 MB buffer written between timed steps", "parallelism": "replicas x1"}
    base = None
    if cfg.grid == "octree":
        slab = 64
        if cfg.index == 5:
            # the positions live in pinned host memory; the GPU copy is dropped
            h = torch.empty((n ** 3, 3), dtype=torch.float32).pin_memory()
            h.copy_(pos)
            del pos
            torch.cuda.empty_cache()
            t0 = time.perf_counter()
            oct_ = pse.build_octree_streamed(h, n, cfg.bc, cfg.max_level, slab, 2.0)
            extra["octree_build_s"] = time.perf_counter() - t0
            out = torch.empty((oct_.n_leaves, cfg.bc, cfg.bc, cfg.bc), dtype=torch.float64, device=dev)

            def step(stats=False):
                return pse.deposit_octree_streamed(h, n, oct_, slab, out=out, stats=stats, precision=prec,
                                                   tuning={"blocks_per_sm": 4})
            config.update({"grid": f"octree bc={cfg.bc} levels 0-{cfg.max_level} (finest {cfg.grid_n}^3)",
                           "schedule": "warp-cooperative", "streaming": f"z-slabs of {slab} cube layers from "
                                                                        "pinned host memory, double-buffered"})
            h2d = int(h.numel() * 4 * (1 + 1 / slab))
        else:
            t0 = time.perf_counter()
            oct_ = pse.build_octree_from_tet_sizes(pos, n, cfg.bc, cfg.max_level, 2.0)
            torch.cuda.synchronize()
            extra["octree_build_s"] = time.perf_counter() - t0
            out = torch.empty((oct_.n_leaves, cfg.bc, cfg.bc, cfg.bc), dtype=torch.float64, device=dev)
            tuned, tune_ms = autotune.tune(lambda tu: pse.deposit_octree(pos, n, oct_, out=out, tuning=tu,
                                                                         precision=prec),
                                           signature=f"octree:{cfg.name}")
            config["autotune_ms"] = tune_ms

            def step(stats=False):
                return pse.deposit_octree(pos, n, oct_, out=out, stats=stats, tuning=tuned, precision=prec)
            config.update({"grid": f"octree bc={cfg.bc} levels 0-{cfg.max_level} (finest {cfg.grid_n}^3)",
                           "schedule": "warp-cooperative", "tuning": tuned})
            h2d = 0
        config["leaves"] = int(oct_.n_leaves)
        config["leaf_levels"] = {int(l): int(c) for l, c in zip(*np.unique(oct_.leaves()[:, 0], return_counts=True))}
        _, st = step(stats=True)
        grid_cells = oct_.n_cells
    else:
        g = cfg.grid_n
        out = torch.empty((g, g, g), dtype=torch.float64, device=dev)
        ws = torch.empty(pse.workspace_size(pse._lib.PSE_OP_DEPOSIT_UNIFORM, pse.lattice(n),
                                            schedule=pse.PSE_BINNED_PERSISTENT, cost_model=cm.CostModel()),
                         dtype=torch.uint8, device=dev)
        # the cost model, trained on the counts the exact deposit produces on workloads 1 and 2
        t0 = time.perf_counter()
        feats, targs = [], []
        for c in (CONFIGS[1], CONFIGS[2]):
            p = torch.from_numpy(config_positions(c)).to(dev)
            feats.append(cm.features(p, c.n, c.grid_n))
            targs.append(cm.labels(cm.tet_counts(p, c.n, c.grid_n)))
        feat, targ = torch.cat(feats), torch.cat(targs)
        mu, sd = cm.standardisation(feat[:: max(1, feat.shape[0] // 200000)].cpu().numpy())
        model = cm.CostModel(cm.pack({**cm.he_init(0), "mu": mu, "sigma": sd}))
        hist = cm.fit(model, feat, targ, steps=2000, batch=8192, lr=3e-3)
        extra["cost_model"] = {"training_s": time.perf_counter() - t0, "loss_first_last": [hist[0], hist[-1]],
                               "train_rows": int(feat.shape[0])}
        del feat, targ, feats, targs
        arms = {"warp": dict(schedule=pse.PSE_WARP_COOPERATIVE, tuning={"blocks_per_sm": 4}, precision=prec),
                "binned-bbox": dict(schedule=pse.PSE_BINNED_PERSISTENT, precision=prec,
                                    tuning={"blocks_per_sm": 4, "split_cells": 512, "chunk_cells": 512}),
                "binned-model": dict(schedule=pse.PSE_BINNED_PERSISTENT, cost_model=model, precision=prec,
                                     tuning={"blocks_per_sm": 4, "split_cells": 256, "chunk_cells": 512})}
        arm_ms = {}
        for name, kw in arms.items():
            ms_list = _timed(lambda: pse.deposit_uniform(pos, n, g, out=out, workspace=ws, **kw), max(1, args.steps),
                             1, flush, stream)
            arm_ms[name] = sum(ms_list) / len(ms_list)
        extra["arms_ms"] = arm_ms
        chosen = arms["binned-model"]

        def step(stats=False):
            return pse.deposit_uniform(pos, n, g, out=out, workspace=ws, stats=stats, **chosen)
        config.update({"grid": f"uniform {g}^3 float64", "schedule": "binned persistent, cost-model split",
                       "tuning": chosen["tuning"]})
        h2d = 0
        _, st = step(stats=True)
        grid_cells = g ** 3
        # the plain FP64 one-thread-per-tetrahedron path, on a contiguous block of 128 x 128 x 32 cubes
        i, j, k = np.meshgrid(np.arange(128), np.arange(128), np.arange(32), indexing="ij")
        ids = torch.from_numpy(np.sort((i + n * (j + n * (k + n // 2))).ravel())).to(dev)
        bms = _timed(lambda: pse.deposit_uniform(pos, n, g, out=out, precision=pse.PSE_FP64_PLAIN,
                                                 schedule=pse.PSE_THREAD_PER_TET, cube_ids=ids), 1, 1, flush, stream)[0]
        fast = pse.deposit_uniform(pos, n, g, cube_ids=ids, **{k: v for k, v in chosen.items()
                                                               if k != "cost_model"}).cpu().numpy()
        slow = out.cpu().numpy()
        filled = slow >= 0.5 / g ** 3  # cells the block fills (not its sparse fringe)
        base = {"tets_per_s": 6 * ids.numel() / (bms * 1e-3), "sample": "128 x 128 x 32 contiguous cubes",
                "error_of_timed_arm_on_sample": cell_errors(fast, slow, floor_mass=1e-3 / g ** 3),
                "error_floor": "1e-3 of the full deposit's mean cell mass",
                "error_on_filled_cells": cell_errors(fast[filled], slow[filled]), "filled_cells": int(filled.sum()),
                "note": "the block's fringe holds slivers of single tetrahedra; 'filled' = FP64 mass >= half "
                        "the mean cell mass"}

    tet_sizes = _tet_size_sample(h if cfg.index == 5 else pos, n, cfg.grid_n)
    with ClockSampler(bus_id_of(0)) as clk:
        t_wall0 = time.perf_counter()
        step_ms = _timed(step, args.steps, args.warmup, flush, stream)
        t_wall = time.perf_counter() - t_wall0
    ms = sum(step_ms) / len(step_ms)
    value = cfg.n_tets / (ms * 1e-3)
    mass_error = abs(float(out.sum()) - 1.0)
    if base is None and cfg.index == 3:
        fast = out.cpu().numpy()
        bms = _timed(lambda: pse.deposit_octree(pos, n, oct_, out=out, precision=pse.PSE_FP64_PLAIN,
                                                schedule=pse.PSE_THREAD_PER_TET), 1, 1, flush, stream)[0]
        base = {"tets_per_s": cfg.n_tets / (bms * 1e-3), "ms_per_step": bms,
                "error_of_timed_arm": cell_errors(fast, out.cpu().numpy())}
    if base is None and cfg.index == 5:
        # FP32 against the plain FP64 path on a contiguous block of 64 x 64 x 32 cubes, positions
        # back on the GPU for this check; floor 1e-3 of the full deposit's mean cell mass
        pos_d = h.to(dev)
        i, j, k = np.meshgrid(np.arange(64), np.arange(64), np.arange(32), indexing="ij")
        ids = torch.from_numpy(np.sort((i + n * (j + n * (k + n // 2))).ravel())).to(dev)
        pse.deposit_octree(pos_d, n, oct_, out=out, cube_ids=ids, tuning={"blocks_per_sm": 4})
        touched = torch.nonzero(out.view(out.shape[0], -1).abs().sum(1) > 0).ravel()  # leaves the block reaches
        fast = out[touched].cpu().numpy()
        bms = _timed(lambda: pse.deposit_octree(pos_d, n, oct_, out=out, cube_ids=ids, precision=pse.PSE_FP64_PLAIN,
                                                schedule=pse.PSE_THREAD_PER_TET), 1, 1, flush, stream)[0]
        slow = out[touched].cpu().numpy()
        filled = slow >= 0.5 / float(grid_cells)  # cells the block fills (not its sparse fringe)
        base = {"tets_per_s": 6 * ids.numel() / (bms * 1e-3), "sample": "64 x 64 x 32 contiguous cubes",
                "error_of_timed_arm_on_sample": cell_errors(fast, slow, floor_mass=1e-3 / float(grid_cells)),
                "error_floor": "1e-3 of the full deposit's mean cell mass",
                "error_on_filled_cells": cell_errors(fast[filled], slow[filled]),
                "filled_cells": int(filled.sum()), "leaves_compared": int(touched.numel()),
                "note": "the block's fringe holds slivers of single tetrahedra; 'filled' = FP64 mass >= half "
                        "the mean cell mass"}
        del pos_d
    if base is not None:
        base["speedup"] = value / base["tets_per_s"]
    csum = clk.summary()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count or SM_COUNT_GB300
    peaks = pse.measure_peaks(stream)
    peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_GB300 * 1e6 / 1e12
    alg = FLOP_PER_TET * st["tets"] + FLOP_PER_BBOX_CELL * st["bbox_cells"] + FLOP_PER_CLIP * st["partial_clips"]
    achieved = alg / (ms * 1e-3) / 1e12
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config,
        "clips_per_s": st["partial_clips"] / (ms * 1e-3),
        "counters": {k: st[k] for k in ("tets", "bbox_cells", "inside_cells", "partial_clips", "fp64_redos",
                                        "degenerate_tets", "single_cell_tets", "inverted_tets")},
        "tet_sizes": tet_sizes,
        "mass_error": mass_error,
        "fp64_gpu_baseline": base,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "note": "step time (all kernels of the call)",
                     "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 FLOP x "
                                    f"{SM_MAX_MHZ_GB300:.0f} MHz",
                     "measured_fma_tflops": peaks["fp32_tflops"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 0,
                "note": "streamed from pinned host memory inside the step" if h2d else
                        "inputs resident (no host copies in this workload's step)"},
        "grid_cells": int(grid_cells), "clocks": csum, "wall_s_timed": t_wall, **extra,
    }
    print(json.dumps(result), flush=True)


# ---------------------------------------------------------------- ours ------
def main():
    args = parse()
    from pse_inputs import CONFIGS
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        run_reference(args, cfg)
        return
    if args.config >= 3:
        run_workload(args, cfg)
        return

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_09491_gb300 as pse
    from paper_1612_09491_gb300.metrics import cell_errors
    from pse_inputs import config_positions

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    dev = torch.device("cuda", local)
    n, g = cfg.n, cfg.grid_n
    n_tets = cfg.n_tets
    pos_host = config_positions(cfg)
    pos = torch.from_numpy(pos_host).to(dev)
    out = torch.empty((g, g, g), dtype=torch.float64, device=dev)
    ws = torch.empty(pse.workspace_size(schedule=pse.PSE_BINNED_PERSISTENT), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    from paper_1612_09491_gb300 import autotune
    prec = pse.PSE_FP32_FP64ACC

    def call(tu, **kw):
        """One deposit with an autotuner candidate {"schedule": "warp" | "binned", knobs...}."""
        knobs = {k: v for k, v in tu.items() if k != "schedule"}
        sched = pse.PSE_BINNED_PERSISTENT if tu["schedule"] == "binned" else pse.PSE_WARP_COOPERATIVE
        return pse.deposit_uniform(pos, n, g, out=out, workspace=ws, precision=prec, schedule=sched, tuning=knobs,
                                   **kw)

    tuned, tune_ms = autotune.tune(call, signature=f"uniform:{cfg.name}", candidates=autotune.UNIFORM_CANDIDATES)
    peaks = pse.measure_peaks(stream)  # the FP32 and FP64-reduction peaks of this GPU

    def step(accumulate=False):
        call(tuned, accumulate=accumulate)

    # the workload's tetrahedron sizes (mean edge length in cells), from the cost-model features
    from paper_1612_09491_gb300 import costmodel as cm
    edges = cm.features(pos, n, g)[:, 11].cpu().numpy()
    tet_sizes = {"mean_edge_cells_quantiles": dict(zip(("min", "p01", "median", "p99", "max"),
                                                       [float(v) for v in np.quantile(edges, [0, .01, .5, .99, 1])]))}
    del edges
    # kernels of one step: [bin pass, chunk scan,] deposit kernel, mass renormalisation
    launches_per_step = 4 if tuned["schedule"] == "binned" else 2
    # counters of one pass (synchronising call, outside the timed region)
    _, st = call(tuned, stats=True)
    fast_grid = out.cpu().numpy().copy()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(bus_id_of(local)) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)  # evict L2 between steps
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms, value = replica_throughput(step_ms, n_tets, dist, dev)
    clips_per_s = world * st["partial_clips"] / (ms * 1e-3)

    # kernel-only duration (accumulate mode: no output clear), for the roofline
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        kev[k][0].record(stream)
        step(accumulate=True)
        kev[k][1].record(stream)
    torch.cuda.synchronize()
    kern_ms = sum(a.elapsed_time(b) for a, b in kev) / len(kev)

    # end to end through the public API with host buffers
    pos_pin = torch.from_numpy(pos_host).pin_memory()
    out_pin = torch.empty((g, g, g), dtype=torch.float64).pin_memory()
    eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        eev[k][0].record(stream)
        pos.copy_(pos_pin, non_blocking=True)
        step()
        out_pin.copy_(out, non_blocking=True)
        eev[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in eev) / len(eev)

    result = {}
    if rank == 0:
        # plain FP64 GPU baseline on the same GPU, and the density error between the two
        base = None
        if not args.no_baseline:
            bev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            pse.deposit_uniform(pos, n, g, out=out, workspace=ws, precision=pse.PSE_FP64_PLAIN,
                                schedule=pse.PSE_THREAD_PER_TET)  # warm-up
            torch.cuda.synchronize()
            flush.fill_(1)
            bev[0].record(stream)
            pse.deposit_uniform(pos, n, g, out=out, workspace=ws, precision=pse.PSE_FP64_PLAIN,
                                schedule=pse.PSE_THREAD_PER_TET)
            bev[1].record(stream)
            torch.cuda.synchronize()
            bms = bev[0].elapsed_time(bev[1])
            ref64 = out.cpu().numpy()
            err = cell_errors(fast_grid, ref64)
            base = {"tets_per_s": n_tets / (bms * 1e-3), "ms_per_step": bms, "speedup": (n_tets / (ms * 1e-3)) /
                    (n_tets / (bms * 1e-3)), "error_of_timed_arm": err}
            # the paper's GPU design (one warp per tetrahedron, Sec. 6.2) with the same clip
            pms = _timed(lambda: pse.deposit_uniform(pos, n, g, out=out, workspace=ws, precision=prec,
                                                     schedule=pse.PSE_WARP_PER_TET), 3, 1, flush, stream)
            pms = sum(pms) / len(pms)
            base["paper_design_warp_per_tet"] = {"tets_per_s": n_tets / (pms * 1e-3), "ms_per_step": pms,
                                                 "speedup_of_timed_arm": pms / ms}
            # the same clips with compensated FP32 (hi, lo) accumulation instead of FP64 reductions
            knobs = {k: v for k, v in tuned.items() if k != "schedule"}
            csched = pse.PSE_BINNED_PERSISTENT if tuned["schedule"] == "binned" else pse.PSE_WARP_COOPERATIVE
            cms = _timed(lambda: pse.deposit_uniform(pos, n, g, out=out, workspace=ws, tuning=knobs, schedule=csched,
                                                     precision=pse.PSE_FP32_COMPENSATED), 3, 1, flush, stream)
            cms = sum(cms) / len(cms)
            base["fp32_compensated_accumulation"] = {"tets_per_s": n_tets / (cms * 1e-3), "ms_per_step": cms,
                                                     "error_vs_fp64": cell_errors(out.cpu().numpy(), ref64)}
        # roofline of the dominant kernel (FP32 ALU bound)
        alg_flop = (FLOP_PER_TET * st["tets"] + FLOP_PER_BBOX_CELL * st["bbox_cells"] +
                    FLOP_PER_CLIP * st["partial_clips"])
        props = torch.cuda.get_device_properties(dev)
        sms = props.multi_processor_count or SM_COUNT_GB300
        csum = clk.summary()
        peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_GB300 * 1e6 / 1e12
        achieved = alg_flop / (kern_ms * 1e-3) / 1e12
        deposits = st["partial_clips"] + st["inside_cells"]  # FP64 reductions issued (upper bound)
        cpu = None
        oracle_err = None
        if not args.no_cpu:
            cpu, ids, ref = oracle_rate(pos_host, cfg, args.cpu_seconds)
            sub = pse.deposit_uniform(pos, n, g, precision=pse.PSE_FP32_FP64ACC, schedule=pse.PSE_WARP_COOPERATIVE,
                                      cube_ids=torch.from_numpy(ids).to(dev))
            oracle_err = cell_errors(sub.cpu().numpy(), ref)
            oracle_err["sample"] = ("same cube sample as cpu_baseline, deposited alone on both sides (a sparse "
                                    "deposit: cells covered by one tetrahedron's sliver are included)")
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg.name, "particles": f"{n}^3", "tets": n_tets, "grid": f"uniform {g}^3 float64",
                       "spectrum": f"P(k)~k^{cfg.spectral_index}", "rms_disp_spacings": cfg.rms_disp,
                       "precision": PRECISION,
                       "schedule": {"binned": "binned persistent", "warp": "warp-cooperative"}[tuned["schedule"]],
                       "tuning": tuned, "autotune_ms": tune_ms,
                       "l2": "512 MB buffer written between timed steps",
                       "parallelism": f"replicas x{world}"},
            "clips_per_s": clips_per_s,
            "counters": {k: st[k] for k in ("tets", "bbox_cells", "inside_cells", "partial_clips", "fp64_redos",
                                            "degenerate_tets", "single_cell_tets", "inverted_tets", "bin_counts")},
            "tet_sizes": tet_sizes,
            "fp64_gpu_baseline": base,
            "error_vs_oracle": oracle_err,
            "kernel_ms": kern_ms,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": DRAM_BYTES_PER_LAUNCH if tuned == {"blocks_per_sm": 4, "schedule": "warp"}
                         else None, "traffic_unit": "bytes per launch (ncu dram read + write)",
                         "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 FLOP x "
                                        f"{SM_MAX_MHZ_GB300:.0f} MHz",
                         "measured_fma_tflops": peaks["fp32_tflops"],
                         "measured_fma_how": peaks["how"].split(";")[0]},
            "atomics": {"achieved_per_s": deposits / (kern_ms * 1e-3), "peak_per_s": peaks["red_f64_per_s"],
                        "frac": deposits / (kern_ms * 1e-3) / peaks["red_f64_per_s"],
                        "note": "FP64 global reductions of the deposit kernel against a scattered-reduction "
                                "microbenchmark measured in this run"},
            "issue": {"thread_inst_per_clip": THREAD_INST_PER_CLIP,
                      "achieved_tinst_per_s": THREAD_INST_PER_CLIP * st["partial_clips"] / (kern_ms * 1e-3),
                      "peak_tinst_per_s": sms * 4 * 32 * SM_MAX_MHZ_GB300 * 1e6,
                      "frac": THREAD_INST_PER_CLIP * st["partial_clips"] / (kern_ms * 1e-3) /
                              (sms * 4 * 32 * SM_MAX_MHZ_GB300 * 1e6),
                      "note": "instruction issue of the deposit kernel against one warp instruction per "
                              "scheduler per clock (4 per SM), all 32 lanes"},
            "cpu_baseline": cpu,
            "e2e": {"value": world * n_tets / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(pos_host.nbytes),
                    "d2h_bytes_per_step": int(out.numel() * 8), "ms_per_step": e2e_ms},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": csum,
            "wall_s_timed": t_wall,
        }
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
