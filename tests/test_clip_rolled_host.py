"""The warp kernels' FP32 clip (overlap_volume_rolled: edge slots in memory, rolled loops, one
loop body per slab axis) against the register clip (overlap_volume_ax<float>), both compiled
for the host from the library's own header: same arithmetic in the same order, so the two
must agree bit for bit, on random tetrahedra of three sizes against a 4^3 block of cells,
including vertices placed exactly on cell planes.  This pins the restructuring, not the
method: the method is pinned by the oracle and the GPU parity tests."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1612_09491_gb300", "csrc")

HARNESS = r'''
#include <cmath>
#include <math.h>
#include <cstdio>
#include <cstring>
#include "geom.cuh"
using namespace pse;

static float urand(unsigned long long &s)
{
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return (float)((s >> 40) & 0xffffff) / 16777216.0f;
}

int main()
{
    unsigned long long seed = 12345;
    float2 E[21 * 32];
    long long n = 0, mism = 0;
    for (int it = 0; it < 20000; ++it) {
        P3<float> v[4];
        const float span = (it % 3 == 0) ? 0.6f : (it % 3 == 1 ? 2.5f : 6.f);
        for (int q = 0; q < 4; ++q)
            v[q] = mk<float>(urand(seed) * span - span * 0.3f, urand(seed) * span - span * 0.3f,
                             urand(seed) * span - span * 0.3f);
        if (it % 7 == 0) { v[1].x = v[0].x; v[2].y = 1.0f; v[3].z = 0.0f; }  // on cell planes
        TetSetup<float> ts;
        tet_setup<float>(v, ts);
        if (ts.vol6 == 0.0) continue;
        for (int cx = -1; cx <= 2; ++cx)
            for (int cy = -1; cy <= 2; ++cy)
                for (int cz = -1; cz <= 2; ++cz) {
                    P3<float> p[4], pa[4], na[4];
                    for (int q = 0; q < 4; ++q) p[q] = mk<float>(ts.v[q].x - cx, ts.v[q].y - cy, ts.v[q].z - cz);
                    float e1, e2;
                    const float r1 = overlap_volume_ax<float>(p, ts.n, ts.axis, ts.lx, ts.ly, e1);
                    for (int q = 0; q < 4; ++q) {
                        pa[q] = to_axis(p[q], ts.axis);
                        na[q] = to_axis(ts.n[q], ts.axis);
                    }
                    const float r2 = overlap_volume_rolled(pa, na, ts.lx, ts.ly, e2, E);
                    ++n;
                    if (std::memcmp(&r1, &r2, 4) || std::memcmp(&e1, &e2, 4)) ++mism;
                }
    }
    std::printf("%lld %lld\n", n, mism);
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


def test_rolled_clip_equals_register_clip(tmp_path):
    inc = _cuda_include()
    cxx = shutil.which("g++")
    if inc is None or cxx is None:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "rolled.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "rolled"
    # no contraction: both versions must round every operation the same way
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-I", inc, "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    n, mism = int(out[0]), int(out[1])
    assert n > 1_000_000
    assert mism == 0, f"{mism} of {n} clips differ"
