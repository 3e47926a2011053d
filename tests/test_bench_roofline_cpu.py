"""bench.py's ALU roofline, on CPU: achieved FLOPs from the counted per-unit model and the
call's counters, the derived peak, and the ncu figures (DRAM traffic per tetrahedron, thread
instructions per clip) used only while the summary's source digest matches the sources."""
from __future__ import annotations

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

ST = {"tets": 1000, "bbox_cells": 30000, "column_runs": 4000, "partial_clips": 5000}
PEAKS = {"fp32_tflops": 77.0}


def test_achieved_and_peak():
    roof, issue = bench.roofline_alu(ST, 2.0, 152, PEAKS, {}, "tet", ST["tets"])
    flop = bench.FLOP_PER_TET * 1000 + bench.FLOP_PER_BBOX_CELL * 30000 + bench.FLOP_PER_RUN * 4000
    assert roof["achieved"] == pytest.approx(flop / 2e-3 / 1e12)
    assert roof["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert roof["traffic"] is None and issue is None  # no summary: no measured figures


def test_profile_figures_apply_only_to_their_sources():
    prof = {"source_digest": bench.source_digest(), "dram_bytes_per_tet": "23.0", "thread_inst_per_clip": "3200"}
    roof, issue = bench.roofline_alu(ST, 2.0, 152, PEAKS, prof, "tet", ST["tets"])
    assert roof["traffic"] == pytest.approx(23.0 * ST["tets"])
    rate = 3200 * ST["partial_clips"] / 2e-3
    assert issue["achieved_tinst_per_s"] == pytest.approx(rate)
    assert issue["frac"] == pytest.approx(rate / (152 * 4 * 32 * 2070e6))
    stale = dict(prof, source_digest="0" * 16)
    roof, issue = bench.roofline_alu(ST, 2.0, 152, PEAKS, stale, "tet", ST["tets"])
    assert roof["traffic"] is None and issue is None


def test_committed_summary_parses():
    prof = bench.profile_figures("k_oct_warp_scale-1024c-octree128")
    assert set(prof) >= {"source_digest", "dram_bytes_per_tet", "thread_inst_per_clip"}
    assert len(prof["source_digest"]) == 16
    assert 0 < float(prof["dram_bytes_per_tet"]) < 100 and 0 < float(prof["thread_inst_per_clip"]) < 1e5
