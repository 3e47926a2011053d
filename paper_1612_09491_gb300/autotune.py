"""Autotuner for the deposit kernels' launch knobs.

Times each candidate tuning on the caller's own workload through the public API
(CUDA events on the current stream, best of a few runs) and returns the fastest.
Results are cached in memory and, if ``cache_path`` is given, in a JSON file keyed
by device name and workload signature.
"""
from __future__ import annotations

import json
import os

# residency: resident 128-thread blocks per SM (2: 255 registers, 3: 170, 4: 128)
CANDIDATES = ({"blocks_per_sm": 2}, {"blocks_per_sm": 3}, {"blocks_per_sm": 4})
# uniform-grid deposits: the warp-cooperative kernel, and the binned persistent schedule
# over its split threshold, split work-item size and residency (launched as a CUDA graph)
UNIFORM_CANDIDATES = tuple([{"schedule": "warp", "blocks_per_sm": b} for b in (2, 3, 4)] +
                           [{"schedule": "binned", "blocks_per_sm": b, "split_cells": sp, "chunk_cells": ch,
                             "use_graph": 1}
                            for b in (2, 3) for sp in (256, 2048) for ch in (256, 1024)])
_mem = {}


def _key(device_name: str, signature: str) -> str:
    return f"{device_name}|{signature}"


def tune(run, signature: str, candidates=CANDIDATES, repeats: int = 3, cache_path: str | None = None):
    """run(tuning_dict) enqueues one deposit; returns (best tuning, {str(tuning): ms})."""
    import torch
    dev = torch.cuda.get_device_name()
    key = _key(dev, signature)
    if key in _mem:
        return _mem[key]
    if cache_path and os.path.exists(cache_path):
        try:
            disk = json.load(open(cache_path))
            if key in disk:
                _mem[key] = (disk[key]["best"], disk[key]["ms"])
                return _mem[key]
        except (OSError, ValueError, KeyError):
            pass
    times = {}
    stream = torch.cuda.current_stream()
    for cand in candidates:
        run(cand)  # warm-up (first launch sets kernel attributes)
        best = float("inf")
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run(cand)
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        times[json.dumps(cand, sort_keys=True)] = best
    best_c = json.loads(min(times, key=times.get))
    _mem[key] = (best_c, times)
    if cache_path:
        try:
            disk = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
            disk[key] = {"best": best_c, "ms": times}
            json.dump(disk, open(cache_path, "w"), indent=1)
        except OSError:
            pass
    return _mem[key]
