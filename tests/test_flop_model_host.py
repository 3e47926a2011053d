"""The FLOP model behind the deposit kernels' ALU roofline, counted: the kernels' own
templates (tet_setup, classify_cell, column_volumes) are compiled for the host with a float
scalar that tallies every add, subtract, multiply, divide and square root (FMA = 2; min,
max, compares and floor are not counted), and run on Zel'dovich tetrahedra of the deposit
workloads' spectrum (P(k) ~ k^-2, the strain of the 1024^3 lattice at 3 spacings rms) at
three cell scales (1, 2 and 4 cells per lattice spacing).  The per-unit figures bench.py
reports against (per tetrahedron, per bounding-box cell, per clipped run of up to two cells)
must lie within 12% of the counts at every scale."""
from __future__ import annotations

import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from pse_inputs.lattice import zeldovich_positions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1612_09491_gb300", "csrc")

HARNESS = r'''
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "column.cuh"

// A float that counts the floating-point operations done on it.
namespace cnt {
struct Tally { long long add = 0, mul = 0, fma = 0, div = 0, sqrt = 0; };
static Tally g;
struct CF {
    float v;
    int pad;  // 8 bytes: the generic (non-float) branches of the templates
    CF() = default;
    constexpr CF(float x) : v(x), pad(0) {}
    explicit CF(int x) : v((float)x), pad(0) {}
    explicit CF(double x) : v((float)x), pad(0) {}
    explicit operator double() const { return v; }
    explicit operator float() const { return v; }
    explicit operator int() const { return (int)v; }
};
inline CF operator-(CF a) { return CF(-a.v); }
inline CF operator+(CF a, CF b) { ++g.add; return CF(a.v + b.v); }
inline CF operator-(CF a, CF b) { ++g.add; return CF(a.v - b.v); }
inline CF operator*(CF a, CF b) { ++g.mul; return CF(a.v * b.v); }
inline CF operator/(CF a, CF b) { ++g.div; return CF(a.v / b.v); }
inline CF &operator+=(CF &a, CF b) { return a = a + b; }
inline CF &operator-=(CF &a, CF b) { return a = a - b; }
inline bool operator<(CF a, CF b) { return a.v < b.v; }
inline bool operator>(CF a, CF b) { return a.v > b.v; }
inline bool operator<=(CF a, CF b) { return a.v <= b.v; }
inline bool operator>=(CF a, CF b) { return a.v >= b.v; }
inline bool operator==(CF a, CF b) { return a.v == b.v; }
inline bool operator!=(CF a, CF b) { return a.v != b.v; }
inline CF fdiv(CF a, CF b) { return a / b; }
inline CF fmaT(CF a, CF b, CF c) { ++g.fma; return CF(std::fma(a.v, b.v, c.v)); }
inline CF mul_rn(CF a, CF b) { return a * b; }
inline CF fabs(CF a) { return CF(std::fabs(a.v)); }
inline CF fmin(CF a, CF b) { return CF(std::fmin(a.v, b.v)); }
inline CF fmax(CF a, CF b) { return CF(std::fmax(a.v, b.v)); }
inline CF floor(CF a) { return CF(std::floor(a.v)); }
inline CF ceil(CF a) { return CF(std::ceil(a.v)); }
inline CF sqrt(CF a) { ++g.sqrt; return CF(std::sqrt(a.v)); }
inline CF sat01(CF x) { return CF(x.v > 0.f ? (x.v < 1.f ? x.v : 1.f) : 0.f); }
}  // namespace cnt
namespace pse {
template <> inline cnt::CF roundoff<cnt::CF>() { return cnt::CF(1.1920928955078125e-07f); }
}
using namespace pse;
using cnt::CF;
static double flops() { return (double)cnt::g.add + cnt::g.mul + 2.0 * cnt::g.fma + cnt::g.div + cnt::g.sqrt; }

int main(int argc, char **argv)
{
    FILE *f = std::fopen(argv[1], "rb");
    std::vector<float> buf;
    float x;
    while (std::fread(&x, 4, 1, f) == 1) buf.push_back(x);
    std::fclose(f);
    const long ntet = (long)buf.size() / 12;
    double f_tet = 0, f_cls = 0, f_run = 0;
    long n_bbox = 0, n_partial = 0, n_runs = 0, n_used = 0;
    CF E0[21 * 32 * 2];
    auto *E = reinterpret_cast<slot2_t<CF> *>(E0);
    for (long t = 0; t < ntet; ++t) {
        P3<CF> v[4];
        for (int q = 0; q < 4; ++q) v[q] = mk<CF>(CF(buf[12 * t + 3 * q]), CF(buf[12 * t + 3 * q + 1]), CF(buf[12 * t + 3 * q + 2]));
        // the vertices relative to their base cell, as the kernels hold them
        const int bx = (int)std::floor(buf[12 * t]), by = (int)std::floor(buf[12 * t + 1]), bz = (int)std::floor(buf[12 * t + 2]);
        for (int q = 0; q < 4; ++q) v[q] = mk<CF>(CF(v[q].x.v - bx), CF(v[q].y.v - by), CF(v[q].z.v - bz));
        double f0 = flops();
        TetSetup<CF> ts;
        tet_setup<CF>(v, ts);
        f_tet += flops() - f0;
        if (ts.vol6 == 0.0 || !(ts.kappa <= 32.f)) continue;  // the FP32 pass's records
        ++n_used;
        const int ax = ts.axis, A = (ax + 1) % 3, B = (ax + 2) % 3, C = ax;
        P3<CF> na[4];
        for (int q = 0; q < 4; ++q) na[q] = to_axis(ts.n[q], ax);
        for (int ia = 0; ia < ts.dim[A]; ++ia)
            for (int ib = 0; ib < ts.dim[B]; ++ib)
                for (int w0 = 0; w0 < ts.dim[C]; w0 += 2) {
                    const int K = std::min(2, ts.dim[C] - w0);
                    int cell[3];
                    cell[A] = ts.lo[A] + ia;
                    cell[B] = ts.lo[B] + ib;
                    cell[C] = ts.lo[C] + w0;
                    int np = 0, nin = 0;
                    for (int j = 0; j < K; ++j) {
                        int cc[3] = {cell[0], cell[1], cell[2]};
                        cc[C] += j;
                        f0 = flops();
                        const int cls = classify_cell<CF>(ts.n, ts.e, ts.pos, ts.neg, CF(cc[0]), CF(cc[1]), CF(cc[2]));
                        f_cls += flops() - f0;
                        ++n_bbox;
                        np += cls == CELL_PARTIAL;
                        nin += cls == CELL_INSIDE;
                    }
                    if (np == 0) continue;  // no partial cell: the run is not clipped
                    n_partial += np;
                    ++n_runs;
                    P3<CF> p[4];
                    for (int q = 0; q < 4; ++q)
                        p[q] = to_axis(mk<CF>(CF(ts.v[q].x.v - cell[0]), CF(ts.v[q].y.v - cell[1]), CF(ts.v[q].z.v - cell[2])), ax);
                    const TetArrays<CF> src{p, na};
                    CF vol[2];
                    f0 = flops();
                    column_volumes<2>(src, ts.lx, ts.ly, K, w0 > 0, vol, E);
                    f_run += flops() - f0;
                }
    }
    std::printf("tets %ld used %ld bbox %ld runs %ld partial %ld ", ntet, n_used, n_bbox, n_runs, n_partial);
    std::printf("per_tet %.1f per_bbox_cell %.1f per_partial_clip %.1f per_run %.1f\n", f_tet / ntet, f_cls / n_bbox,
                f_run / n_partial, f_run / n_runs);
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


def _bench_constants():
    text = open(os.path.join(ROOT, "bench.py")).read()
    return {k: float(re.search(rf"^{k} = ([0-9.]+)", text, re.M).group(1))
            for k in ("FLOP_PER_TET", "FLOP_PER_BBOX_CELL", "FLOP_PER_RUN")}


def test_flop_model_matches_counted_operations(tmp_path):
    inc = _cuda_include()
    cxx = shutil.which("g++")
    if inc is None or cxx is None:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "flops.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "flops"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-I", inc, "-o", str(exe), str(src)], check=True, capture_output=True)
    n = 32
    # the 1024^3 workload's strain at this lattice size (strain variance ~ rms^2 / n for k^-2)
    pos = zeldovich_positions(n, -2.0, 3.0 * np.sqrt(n / 1024), seed=1005)
    ids = np.random.default_rng(0).choice(6 * n ** 3, 6000, replace=False)
    tets = np.array([oracle.lattice_tet(pos, n, int(t // 6), int(t % 6)) for t in ids])
    model = _bench_constants()
    for cells_per_spacing in (1, 2, 4):
        f = tmp_path / f"tets{cells_per_spacing}.bin"
        (tets * (cells_per_spacing * n)).astype(np.float32).tofile(f)
        out = subprocess.run([str(exe), str(f)], check=True, capture_output=True, text=True).stdout.split()
        got = dict(zip(out[0::2], out[1::2]))
        assert int(got["runs"]) > 10_000, got
        for key, name in (("per_tet", "FLOP_PER_TET"), ("per_bbox_cell", "FLOP_PER_BBOX_CELL"),
                          ("per_run", "FLOP_PER_RUN")):
            counted = float(got[key])
            assert abs(model[name] / counted - 1.0) <= 0.12, (cells_per_spacing, key, counted, model[name])
