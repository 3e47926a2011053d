"""The guarded pass's column clip in float64 (column_volumes<2, double>), compiled for the host
from the library's own header and checked against the float64 per-cell clip
(overlap_volume_fp64) of the same exact tetrahedra.

Flattened tetrahedra (slivers 0.1, 1e-3 and 1e-6 cells thick, vertices given as a float32
value plus its rounding residual, as the kernels store them) and ill-conditioned random ones
(kappa > 32, the ones the FP32 guard sends to this pass): every cell of every run within
1e-12 of a cell of the per-cell clip, and the runs of a tetrahedron add up to its volume.
The tetrahedra are oriented by their exact vertices: with the float32-rounded ones some
1e-6 slivers come out inverted (the harness counts them, and the test asserts that the case
occurs), and the clip of an inverted tetrahedron is wrong by its whole volume.

The method itself is pinned by the oracle and the GPU parity tests; this pins the
restructured float64 arithmetic and the exact-orientation rule against the plain clip."""
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

static double urand(unsigned long long &s)
{
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return (double)((s >> 11) & ((1ull << 53) - 1)) / 9007199254740992.0;
}

int main()
{
    unsigned long long seed = 4242;
    static double2 E[21 * 32];
    for (int mode = 0; mode < 4; ++mode) {
        // modes 0-2: slivers of the given thickness; mode 3: random, kept when kappa > 32
        const double thick = mode == 0 ? 1e-1 : (mode == 1 ? 1e-3 : (mode == 2 ? 1e-6 : 0.0));
        double emax = 0.0, esum = 0.0;
        long ncell = 0, ntet = 0, nflip = 0;
        for (int it = 0; it < 2500; ++it) {
            double x[4][3];
            const double span = 1.0 + 3.0 * urand(seed);
            for (int q = 0; q < 4; ++q)
                for (int a = 0; a < 3; ++a) x[q][a] = urand(seed) * span - 0.3 * span;
            if (mode < 3) {  // project onto two parallel planes `thick` apart
                double d[3] = {urand(seed) - 0.5, urand(seed) - 0.5, urand(seed) - 0.5};
                const double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                for (double &c : d) c /= dn;
                for (int q = 0; q < 4; ++q) {
                    const double h = x[q][0] * d[0] + x[q][1] * d[1] + x[q][2] * d[2];
                    const double t = (q & 1 ? 0.5 : -0.5) * thick - h;
                    for (int a = 0; a < 3; ++a) x[q][a] += t * d[a];
                }
            }
            // the kernels' form: float32 vertex plus float32 residual
            P3<float> v[4], r[4];
            for (int q = 0; q < 4; ++q) {
                v[q] = mk<float>((float)x[q][0], (float)x[q][1], (float)x[q][2]);
                r[q] = mk<float>((float)(x[q][0] - (double)v[q].x), (float)(x[q][1] - (double)v[q].y),
                                 (float)(x[q][2] - (double)v[q].z));
            }
            TetSetup<float> ts;  // axis, box and reference slopes from the float32 set, as on the device
            if (tet_setup<float>(v, ts)) std::swap(r[1], r[2]);
            if (ts.vol6 == 0.0) continue;
            if (mode == 3 && ts.kappa <= 32.f) continue;
            ++ntet;
            P3<double> ve[4];
            for (int q = 0; q < 4; ++q)
                ve[q] = mk<double>((double)ts.v[q].x + r[q].x, (double)ts.v[q].y + r[q].y,
                                   (double)ts.v[q].z + r[q].z);
            if (det6(ve) < 0.0) {  // orient by the exact vertices
                std::swap(ve[1], ve[2]);
                ++nflip;           // the float32 set (oriented by tet_setup) has the other sign
            }
            const double V = std::fabs(det6(ve)) / 6.0;
            const int ax = ts.axis, A = (ax + 1) % 3, B = (ax + 2) % 3, C = ax;
            double tot = 0.0;
            for (int ia = 0; ia < ts.dim[A]; ++ia)
                for (int ib = 0; ib < ts.dim[B]; ++ib)
                    for (int w0 = 0; w0 < ts.dim[C]; w0 += 2) {
                        const int K = std::min(2, ts.dim[C] - w0);
                        int cell[3];
                        cell[A] = ts.lo[A] + ia;
                        cell[B] = ts.lo[B] + ib;
                        cell[C] = ts.lo[C] + w0;
                        P3<double> p[4], n[4];
                        for (int q = 0; q < 4; ++q)
                            p[q] = to_axis(mk<double>(ve[q].x - cell[0], ve[q].y - cell[1], ve[q].z - cell[2]), ax);
                        for (int f = 0; f < 4; ++f) {
                            int a, b, c;
                            face_vertices(f, a, b, c);
                            n[f] = cross(sub(p[b], p[a]), sub(p[c], p[a]));
                        }
                        double vol[2];
                        const TetArrays<double> src{p, n};
                        column_volumes<2>(src, (double)ts.lx, (double)ts.ly, K, w0 > 0, vol, E);
                        for (int j = 0; j < K; ++j) {
                            int cc[3] = {cell[0], cell[1], cell[2]};
                            cc[C] += j;
                            P3<double> pd[4];
                            for (int q = 0; q < 4; ++q)
                                pd[q] = mk<double>(ve[q].x - cc[0], ve[q].y - cc[1], ve[q].z - cc[2]);
                            emax = std::max(emax, std::fabs(vol[j] - overlap_volume_fp64(pd)));
                            tot += vol[j];
                            ++ncell;
                        }
                    }
            esum = std::max(esum, std::fabs(tot - V));
        }
        std::printf("mode %d %ld %ld %ld %.6g %.6g\n", mode, ntet, ncell, nflip, emax, esum);
    }
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


def test_fp64_column_clip_matches_fp64_cell_clip(tmp_path):
    inc = _cuda_include()
    cxx = shutil.which("g++")
    if inc is None or cxx is None:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "column_fp64.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "column_fp64"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-I", inc, "-o", str(exe), str(src)], check=True, capture_output=True)
    lines = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    assert len(lines) == 4
    for line in lines:
        _, mode, ntet, ncell, nflip, emax, esum = line.split()
        assert int(ntet) >= (300 if mode == "3" else 2000), line
        assert int(ncell) > 5 * int(ntet), line
        assert float(emax) <= 1e-12, line        # per cell, in cell volumes
        assert float(esum) <= 1e-12, line        # all runs of a tetrahedron: its volume
        if mode == "2":
            assert int(nflip) > 0, line          # rounded 1e-6 slivers do come out inverted
