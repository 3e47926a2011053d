"""The warp kernels' column clip (column_volumes: one x/y clip per face for a run of cells
along the divergence axis, cell volumes as differences of the volume below each level),
compiled for the host from the library's own header and checked against the float64
per-cell clip (overlap_volume_fp64) of the same float32 tetrahedra.

* every cell of every run, random tetrahedra of three sizes (the FP32 path's conditioning
  range, kappa <= 32), vertices on cell planes included: |error| <= 2e-6 of a cell;
* a run that starts inside the tetrahedron's extent (lo_open) gives the same cells as the
  run that starts below it;
* the volumes of all runs of a tetrahedron add up to its volume.

This pins the restructured arithmetic against the plain per-cell clip; the method itself is
pinned by the oracle and the GPU parity tests."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1612_09491_gb300", "csrc")

HARNESS = r'''
#include <algorithm>
#include <cmath>
#include <cstdio>
#include "column.cuh"
using namespace pse;

static float urand(unsigned long long &s)
{
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return (float)((s >> 40) & 0xffffff) / 16777216.0f;
}

template <int KW>
static void run(const TetSetup<float> &ts, int ia, int ib, int w0, int K, float (&vol)[KW], float2 *E)
{
    const int ax = ts.axis, A = (ax + 1) % 3, B = (ax + 2) % 3, C = ax;
    int cell[3];
    cell[A] = ts.lo[A] + ia;
    cell[B] = ts.lo[B] + ib;
    cell[C] = ts.lo[C] + w0;
    P3<float> p[4], na[4];
    for (int q = 0; q < 4; ++q) {
        p[q] = to_axis(mk<float>(ts.v[q].x - cell[0], ts.v[q].y - cell[1], ts.v[q].z - cell[2]), ax);
        na[q] = to_axis(ts.n[q], ax);
    }
    const TetArrays<float> src{p, na};
    column_volumes<KW>(src, ts.lx, ts.ly, K, w0 > 0, vol, E);
}

int main()
{
    unsigned long long seed = 2024;
    float2 E[21 * 32];
    long long ncell = 0;
    double emax = 0.0, esplit = 0.0, esum = 0.0;
    for (int it = 0; it < 12000; ++it) {
        P3<float> v[4];
        const float span = (it % 3 == 0) ? 0.6f : (it % 3 == 1 ? 2.5f : 6.f);
        for (int q = 0; q < 4; ++q)
            v[q] = mk<float>(urand(seed) * span - span * 0.3f, urand(seed) * span - span * 0.3f,
                             urand(seed) * span - span * 0.3f);
        if (it % 7 == 0) { v[1].x = v[0].x; v[2].y = 1.0f; v[3].z = 0.0f; }  // on cell planes
        TetSetup<float> ts;
        tet_setup<float>(v, ts);
        if (ts.vol6 == 0.0 || !(ts.kappa <= 32.f)) continue;
        const int ax = ts.axis, A = (ax + 1) % 3, B = (ax + 2) % 3, C = ax;
        double tot = 0.0;
        for (int ia = 0; ia < ts.dim[A]; ++ia)
            for (int ib = 0; ib < ts.dim[B]; ++ib)
                for (int w0 = 0; w0 < ts.dim[C]; w0 += 2) {
                    const int K = std::min(2, ts.dim[C] - w0);
                    float vol[2];
                    run<2>(ts, ia, ib, w0, K, vol, E);
                    for (int j = 0; j < K; ++j) {
                        int cc[3];
                        cc[A] = ts.lo[A] + ia;
                        cc[B] = ts.lo[B] + ib;
                        cc[C] = ts.lo[C] + w0 + j;
                        P3<double> pd[4];
                        for (int q = 0; q < 4; ++q)
                            pd[q] = mk<double>((double)ts.v[q].x - cc[0], (double)ts.v[q].y - cc[1],
                                               (double)ts.v[q].z - cc[2]);
                        emax = std::max(emax, std::fabs((double)vol[j] - overlap_volume_fp64(pd)));
                        tot += vol[j];
                        ++ncell;
                        // the same cell as the first of a run that starts at it (lo_open when j > 0)
                        if (j == 1) {
                            float v1[1];
                            run<1>(ts, ia, ib, w0 + 1, 1, v1, E);
                            esplit = std::max(esplit, std::fabs((double)v1[0] - (double)vol[1]));
                        }
                    }
                }
        esum = std::max(esum, std::fabs(tot - ts.vol6 / 6.0) / std::max(1.0, ts.vol6 / 6.0));
    }
    std::printf("%lld %.6g %.6g %.6g\n", ncell, emax, esplit, esum);
    return 0;
}
'''


def _cuda_include():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return os.path.join(c, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


def test_column_clip_matches_fp64_cell_clip(tmp_path):
    inc = _cuda_include()
    cxx = shutil.which("g++")
    if inc is None or cxx is None:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "column.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "column"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-I", inc, "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    n, emax, esplit, esum = int(out[0]), float(out[1]), float(out[2]), float(out[3])
    assert n > 200_000
    assert emax <= 2e-6, emax        # per cell, in cell volumes
    assert esplit <= 2e-6, esplit    # a run split at a cell gives that cell again
    assert esum <= 5e-6, esum        # all cells of a tetrahedron: its volume
