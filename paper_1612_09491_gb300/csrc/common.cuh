// common.cuh -- device building blocks shared by the uniform-grid (deposit.cu) and
// octree (octree.cu) deposit kernels: tetrahedron sources, cell deposits, counters
// and the warp-cooperative (tetrahedron, cell) pair machinery.
#pragma once

#include "column.cuh"
#include "internal.h"

namespace pse {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void kuhn_offsets(int s, int (&o1)[3], int (&o2)[3])
{
    // axis permutations (a, b, c): xyz, xzy, yxz, yzx, zxy, zyx
    const int a = (s < 2) ? 0 : (s < 4) ? 1 : 2;
    const int b = (s == 0) ? 1 : (s == 1) ? 2 : (s == 2) ? 0 : (s == 3) ? 2 : (s == 4) ? 0 : 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o1[k] = (k == a) ? 1 : 0;
        o2[k] = (k == a || k == b) ? 1 : 0;
    }
}

// The Lagrangian orientation of Kuhn tetrahedron s is the parity of its axis permutation:
// xzy, yxz and zyx are odd, so those tetrahedra start with a negative signed volume.  A
// tetrahedron is inverted (turned inside out by shell crossing) when its signed volume
// now has the other sign.
__device__ __forceinline__ bool kuhn_negative(int s) { return s == 1 || s == 2 || s == 5; }

// floor to int for coordinates in grid units; non-finite or out-of-range values map to
// kBadCoord, which tet_ok() rejects before anything is indexed with them.
constexpr int kBadCoord = -(1 << 30);

__device__ __forceinline__ int safe_floor(double x)
{
    return (x > -1073741824.0 && x < 1073741824.0) ? (int)floor(x) : kBadCoord;
}

// A tetrahedron is processed only if its base cell and bounding box are sane.
template <class T>
__device__ __forceinline__ bool tet_ok(const int (&base)[3], const TetSetup<T> &ts)
{
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ok = ok && base[a] != kBadCoord && ts.dim[a] >= 1 && ts.dim[a] <= (1 << 24) &&
             ts.lo[a] > -(1 << 24) && ts.lo[a] < (1 << 24);
    }
    return ok;
}

__device__ __forceinline__ int64_t wrap_idx(int64_t i, int64_t n)
{
    if (i >= n) i -= n;
    if (i < 0) i += n;
    return i;
}

// Vertices of tetrahedron s of Lagrangian cube (ci, cj, ck), in grid units relative to
// the base cell (the cell holding corner 000).  Periodic unwrap: corner v is moved by
// -box when v - v0 >= box/2 and by +box when v - v0 < -box/2 (nearest image), decided
// in float64 on the float32 inputs.
template <class T>
__device__ __forceinline__ void lattice_tet(const DepositParams &P, int64_t ci, int64_t cj, int64_t ck, int s,
                                            P3<T> (&v)[4], int (&base)[3], P3<float> *res = nullptr)
{
    int o1[3], o2[3];
    kuhn_offsets(s, o1, o2);
    float x[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int64_t i = ci, j = cj, k = ck;
        if (q == 1) { i += o1[0]; j += o1[1]; k += o1[2]; }
        if (q == 2) { i += o2[0]; j += o2[1]; k += o2[2]; }
        if (q == 3) { i += 1; j += 1; k += 1; }
        if (P.periodic) {
            i = wrap_idx(i, P.n[0]);
            j = wrap_idx(j, P.n[1]);
            if (!P.slab) k = wrap_idx(k, P.n[2]);
        }
        const float *p = P.pos + 3 * (i + P.n[0] * (j + P.n[1] * k));
        x[q][0] = __ldg(p);
        x[q][1] = __ldg(p + 1);
        x[q][2] = __ldg(p + 2);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) base[a] = safe_floor((double)x[0][a] * P.scale_d[a]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        T c[3];
        float rr[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int shift = 0;
            if (P.periodic && q > 0) {
                const double d = (double)x[q][a] - (double)x[0][a];
                shift = (d >= 0.5 * P.box) ? -1 : ((d < -0.5 * P.box) ? 1 : 0);
            }
            const long long off = (long long)shift * P.g[a] - base[a];
            if constexpr (sizeof(T) == 4) {
                c[a] = fmaf(x[q][a], P.scale_f[a], (float)off);
                if (res) rr[a] = (float)(fma((double)x[q][a], P.scale_d[a], (double)off) - (double)c[a]);
            } else {
                c[a] = fma((double)x[q][a], P.scale_d[a], (double)off);
            }
        }
        v[q] = mk<T>(c[0], c[1], c[2]);
        if (sizeof(T) == 4 && res) res[q] = mk<float>(rr[0], rr[1], rr[2]);
    }
}

template <class T>
__device__ __forceinline__ void explicit_tet(const DepositParams &P, int64_t t, P3<T> (&v)[4], int (&base)[3],
                                             P3<float> *res = nullptr)
{
    const float *p = P.verts + 12 * t;
    float x[4][3];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int a = 0; a < 3; ++a) x[q][a] = __ldg(p + 3 * q + a);
#pragma unroll
    for (int a = 0; a < 3; ++a) base[a] = safe_floor((double)x[0][a] * P.scale_d[a]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        T c[3];
        float rr[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if constexpr (sizeof(T) == 4) {
                c[a] = fmaf(x[q][a], P.scale_f[a], (float)(-base[a]));
                if (res) rr[a] = (float)(fma((double)x[q][a], P.scale_d[a], (double)(-base[a])) - (double)c[a]);
            } else {
                c[a] = fma((double)x[q][a], P.scale_d[a], (double)(-base[a]));
            }
        }
        v[q] = mk<T>(c[0], c[1], c[2]);
        if (sizeof(T) == 4 && res) res[q] = mk<float>(rr[0], rr[1], rr[2]);
    }
}

// The float32 vertices of the FP32 path are rounded; res holds the rounding residuals
// (exact value = (double)v + (double)res, both terms exact in float64), so that the
// guarded float64 clips and volume use the exact tetrahedron.
__device__ __forceinline__ void swap12(P3<float> (&r)[4])
{
    const P3<float> t = r[1];
    r[1] = r[2];
    r[2] = t;
}

// exact vertices in the frame of cell (cx, cy, cz) of the base frame
__device__ __forceinline__ void exact_vertices(const P3<float> (&v)[4], const P3<float> (&r)[4], int cx, int cy,
                                               int cz, P3<double> (&pd)[4])
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        pd[q] = mk<double>(((double)v[q].x + (double)r[q].x) - (double)cx, ((double)v[q].y + (double)r[q].y) - (double)cy,
                           ((double)v[q].z + (double)r[q].z) - (double)cz);
}

// |6V| of the exact tetrahedron (falls back to the float32 one if that is 0); flip is set
// when the exact tetrahedron's orientation is the opposite of the float32 one's (a sliver
// thinner than float32 rounding can turn over when rounded)
__device__ __forceinline__ double exact_vol6(const P3<float> (&v)[4], const P3<float> (&r)[4], double vol6_f32,
                                             bool *flip = nullptr)
{
    P3<double> pd[4];
    exact_vertices(v, r, 0, 0, 0, pd);
    const double s = det6(pd);
    if (flip) *flip = s < 0.0;
    const double d = fabs(s);
    return d > 0.0 ? d : vol6_f32;
}

// Lagrangian cube of work unit u; false (and nothing read) for an out-of-range cube id.
__device__ __forceinline__ bool cube_of_unit(const DepositParams &P, int64_t u, int64_t &i, int64_t &j, int64_t &k)
{
    const int64_t c = (P.src == SRC_CUBE_LIST) ? P.cube_ids[u] : u;
    if (c < 0 || c >= P.nc[0] * P.nc[1] * P.nc[2]) return false;
    i = c % P.nc[0];
    j = (c / P.nc[0]) % P.nc[1];
    k = c / (P.nc[0] * P.nc[1]);
    return true;
}

__device__ __forceinline__ int64_t fold_cell(int64_t c, int64_t g)
{
    if (c >= -g && c < 2 * g) {
        if (c < 0) c += g;
        if (c >= g) c -= g;
        return c;
    }
    c %= g;
    return c < 0 ? c + g : c;
}

// How a kernel adds to the output cells (compile-time, so that the FP64 kernels carry
// no trace of the other mode):
//  * F64: one global FP64 reduction per addend.
//  * COMP: compensated FP32 accumulation.  Until the end of the call each cell holds an
//    FP32 pair (hi at the lower 4 bytes, lo at the upper 4).  hi takes m rounded to float
//    with an atomic add that returns the previous value; the exact rounding error of that
//    add (Knuth's two-sum, exact under round-to-nearest) and the error of rounding m to
//    float go to lo.  hi + lo then carries the cell's sum to about 2^-48 relative per addend.
//  * RUNTIME: either, from P.comp (the baseline kernels).
enum class Acc : int { F64 = 0, COMP = 1, RUNTIME = 2 };

__device__ __forceinline__ void cell_add_compensated(double *addr, double m)
{
    float *hl = reinterpret_cast<float *>(addr);
    const float v = __double2float_rn(m);
    const float r = __double2float_rn(m - (double)v);
    const float old = atomicAdd(hl, v);
    const float s = __fadd_rn(old, v);
    const float bv = __fsub_rn(s, old);
    const float e = __fadd_rn(__fsub_rn(old, __fsub_rn(s, bv)), __fsub_rn(v, bv));
    const float c = __fadd_rn(e, r);
    if (c != 0.f) atomicAdd(hl + 1, c);
}

template <Acc A = Acc::RUNTIME>
__device__ __forceinline__ void cell_add(const DepositParams &P, double *addr, double m)
{
    if constexpr (A == Acc::F64) {
        atomicAdd(addr, m);
    } else if constexpr (A == Acc::COMP) {
        cell_add_compensated(addr, m);
    } else {
        if (P.comp) cell_add_compensated(addr, m);
        else atomicAdd(addr, m);
    }
}

// Add m to cell (cx, cy, cz) (unfolded grid indices); returns false if the cell is
// outside an open grid (then the mass is dropped).
template <Acc A = Acc::RUNTIME>
__device__ __forceinline__ bool deposit_cell(const DepositParams &P, int64_t cx, int64_t cy, int64_t cz, double m)
{
    if (P.periodic) {
        cx = fold_cell(cx, P.g[0]);
        cy = fold_cell(cy, P.g[1]);
        cz = fold_cell(cz, P.g[2]);
    } else if (cx < 0 || cy < 0 || cz < 0 || cx >= P.g[0] || cy >= P.g[1] || cz >= P.g[2]) {
        return false;
    }
    cell_add<A>(P, P.out + (cx + P.g[0] * (cy + P.g[1] * cz)), m);
    return true;
}

template <class T>
__device__ __forceinline__ void centroid_cell(const P3<T> (&v)[4], int (&c)[3])
{
    c[0] = (int)floor(((double)v[0].x + (double)v[1].x + (double)v[2].x + (double)v[3].x) * 0.25);
    c[1] = (int)floor(((double)v[0].y + (double)v[1].y + (double)v[2].y + (double)v[3].y) * 0.25);
    c[2] = (int)floor(((double)v[0].z + (double)v[1].z + (double)v[2].z + (double)v[3].z) * 0.25);
}

__device__ __forceinline__ int size_bin(int64_t cells)
{
    int b = 0;
    int64_t edge = 1;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        b += (cells > edge) ? 1 : 0;
        edge *= 8;
    }
    return b;
}

// Mass sums for the FP32 renormalisation, always kept: the target sum of m_t and the sum
// of every computed deposit.  A persistent lane adds up to ~10^6 terms, so plain running
// sums would drift by up to n x 2^-53 (the same mass added repeatedly rounds the same way):
// equal lattice masses are counted as an integer (times m_t at the end) and deposits are
// summed with Kahan's compensation.
struct Counters {
    unsigned long long u[ST_NUM_U64];
    double mass_in, dropped;
    double tgt;            // explicit tetrahedra: sum of m_t
    unsigned ntgt;         // lattice tetrahedra (each P.m_tet)
    double dep, dep_c;     // Kahan sum of deposits and its compensation
    double dep_b;          // plain sum of the deposits since the last fold (a few dozen)
    __device__ void zero()
    {
#pragma unroll
        for (int i = 0; i < ST_NUM_U64; ++i) u[i] = 0;
        mass_in = 0.0;
        dropped = 0.0;
    }
    __device__ void zero_mass()
    {
        tgt = 0.0;
        ntgt = 0;
        dep = 0.0;
        dep_c = 0.0;
        dep_b = 0.0;
    }
    __device__ __forceinline__ void add_tgt(const DepositParams &P, double m_t)
    {
        if (P.src == SRC_TETS) tgt += m_t;
        else ++ntgt;
    }
    __device__ __forceinline__ void add_dep(double m) { dep_b += m; }
    // fold the batch into the Kahan sum (after every round of pairs, every tetrahedron of
    // the thread kernels, and before the flush)
    __device__ __forceinline__ void fold_dep()
    {
        const double y = dep_b - dep_c;
        const double t = dep + y;
        dep_c = (t - dep) - y;
        dep = t;
        dep_b = 0.0;
    }
    __device__ void flush_mass(const DepositParams &P, Workspace *ws)
    {
        fold_dep();
        double a = fma((double)ntgt, P.m_tet, tgt), b = dep - dep_c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(kFull, a, o);
            b += __shfl_down_sync(kFull, b, o);
        }
        if ((threadIdx.x & 31) == 0 && (a != 0.0 || b != 0.0)) {
            atomicAdd(&ws->mass_target, a);
            atomicAdd(&ws->mass_deposited, b);
        }
    }
    __device__ void flush(Workspace *ws)
    {
        // warp-aggregate, then one atomic per warp and counter
#pragma unroll
        for (int i = 0; i < ST_NUM_U64; ++i) {
            unsigned long long x = u[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
            if ((threadIdx.x & 31) == 0 && x) atomicAdd(&ws->stats[i], x);
        }
        double a = mass_in, b = dropped;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(kFull, a, o);
            b += __shfl_down_sync(kFull, b, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&ws->mass_in, a);
            if (b != 0.0) atomicAdd(&ws->mass_dropped, b);
        }
    }
};

__device__ __forceinline__ void set_error(Workspace *ws, int code, int detail)
{
    if (atomicCAS(&ws->error_code, 0, code) == 0) ws->error_detail = detail;
}

struct WarpSmem {
    float v[12][32];      // base-frame vertices (x0 y0 z0 x1 ...), positively oriented
    float n[12][32];      // outward face normals
    float e[4][32];
    float pos[4][32];
    float neg[4][32];
    float lx[32], ly[32];  // reference-plane slopes (in the clip's frame)
    int axis[32];          // the clip's divergence axis (to_axis)
    int lo[3][32];
    int dim[3][32];
    int base[3][32];
    int leaf[32];         // octree: leaf of this (tetrahedron, leaf) pair
    int org[3][32];       // octree: the leaf's first cell, base-cell frame
    float rho[32];        // 6 m_t / |6V| (deposit = rho * overlap volume, formed in float32)
    int start[32];        // exclusive prefix of the pair counts
    int skip[32];         // first pair of this record (split tetrahedra; else 0)
    int guard[32];        // bit 0: a guarded tetrahedron (clipped in float64);
                          // kGuardFlip: its exact vertices are oriented the other way round
    int cut[32];          // octree: 1 if the record's cell range starts above the tetrahedron's
                          // own first layer along its divergence axis (a leaf block cuts it)
    float *vres;          // this warp's residual block in global memory: [12][32] floats, the
                          // rounding residuals of guarded records (exact vertex = v + vres)
    unsigned long long q[64];  // queued partial pairs: t | ix << 5 | iy << 24 | iz << 43
    unsigned long long gq[64]; // queued partial pairs of guarded tetrahedra (float64 clips)
    double2 *dpoly;            // the guarded pass's float64 edge slots: [21][32], this warp's
    float2 poly[21][32];       // FP32 clip: each lane's 7 edge slots, 3 float2 each:
                               // (a.x, a.y), (a.z, b.x), (b.y, b.z)
};

constexpr int kQBits = 19;  // per-axis cell offset bits in a queue entry
constexpr int kGuardFlip = 2;
constexpr unsigned long long kQMask = (1ull << kQBits) - 1;

__device__ __forceinline__ unsigned long long q_pack(int t, int ix, int iy, int iz)
{
    return (unsigned long long)t | ((unsigned long long)ix << 5) | ((unsigned long long)iy << (5 + kQBits)) |
           ((unsigned long long)iz << (5 + 2 * kQBits));
}

__device__ __forceinline__ void decompose(int local, int dx, int dy, int &ix, int &iy, int &iz)
{
    const int dxy = dx * dy;
    iz = local / dxy;
    const int r = local - iz * dxy;
    iy = r / dx;
    ix = r - iy * dx;
}

// The float64 clip of guarded record t against cell (cx, cy, cz) in the cell-by-cell
// schedule (the warp-per-tetrahedron baseline), kept out of line so that the FP32 hot loop
// stays small; it rebuilds the exact vertices from the float32 vertices and their residuals.
__device__ __noinline__ double redo_fp64(const WarpSmem *S, int t, int cx, int cy, int cz)
{
    P3<float> v[4], r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = mk<float>(S->v[3 * q][t], S->v[3 * q + 1][t], S->v[3 * q + 2][t]);
        r[q] = mk<float>(S->vres[(3 * q) * 32 + t], S->vres[(3 * q + 1) * 32 + t], S->vres[(3 * q + 2) * 32 + t]);
    }
    P3<double> pd[4];
    exact_vertices(v, r, cx, cy, cz, pd);
    return overlap_volume_fp64(pd);
}

// Record a guarded tetrahedron's residuals for redo_fp64.
__device__ __forceinline__ void store_residuals(WarpSmem *S, int lane, const P3<float> (&r)[4])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        S->vres[(3 * q) * 32 + lane] = r[q].x;
        S->vres[(3 * q + 1) * 32 + lane] = r[q].y;
        S->vres[(3 * q + 2) * 32 + lane] = r[q].z;
    }
}

// Record lane's tetrahedron (uniform grid) for the pair machinery.
__device__ __forceinline__ void store_record(WarpSmem *S, int lane, const TetSetup<float> &ts,
                                             const P3<float> (&res)[4], const int (&base)[3], double m_t,
                                             float kappa_max, int skip)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        S->v[3 * q][lane] = ts.v[q].x;
        S->v[3 * q + 1][lane] = ts.v[q].y;
        S->v[3 * q + 2][lane] = ts.v[q].z;
        S->n[3 * q][lane] = ts.n[q].x;
        S->n[3 * q + 1][lane] = ts.n[q].y;
        S->n[3 * q + 2][lane] = ts.n[q].z;
        S->e[q][lane] = ts.e[q];
        S->pos[q][lane] = ts.pos[q];
        S->neg[q][lane] = ts.neg[q];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        S->lo[a][lane] = ts.lo[a];
        S->dim[a][lane] = ts.dim[a];
        S->base[a][lane] = base[a];
    }
    const int guard = (ts.kappa <= kappa_max) ? 0 : 1;
    bool flip = false;
    S->rho[lane] = guard ? (float)(6.0 * m_t / exact_vol6(ts.v, res, ts.vol6, &flip))
                         : __fdiv_rn((float)(6.0 * m_t), (float)ts.vol6);
    S->lx[lane] = ts.lx;
    S->ly[lane] = ts.ly;
    S->axis[lane] = ts.axis;
    S->guard[lane] = guard | (flip ? kGuardFlip : 0);
    S->skip[lane] = skip;
    S->cut[lane] = 0;
    if (guard) store_residuals(S, lane, res);
}

// ---------------------------------------------------------------------------
// Column runs.  A tetrahedron below the FP32 guard is enumerated by runs of up to kRun
// cells along its divergence axis C (to_axis: A = C + 1, B = C + 2 mod 3): pair index
// ia + dA (ib + dB w) is the run of cells (A, B) = (lo_A + ia, lo_B + ib) and C in
// [lo_C + kRun w, lo_C + kRun w + kw).  One column clip (column_volumes) serves the run.
// ---------------------------------------------------------------------------
constexpr int kRun = 2;  // longer runs lose accuracy: the level terms grow with the run's height

__device__ __forceinline__ int axis_a(int C) { return C == 2 ? 0 : C + 1; }
__device__ __forceinline__ int axis_b(int C) { return C == 0 ? 2 : C - 1; }

// pairs of an unguarded record: its runs
__device__ __forceinline__ int64_t run_count(const int (&dim)[3], int C)
{
    const int dC = C == 0 ? dim[0] : (C == 1 ? dim[1] : dim[2]);
    const int dA = C == 2 ? dim[0] : (C == 0 ? dim[1] : dim[2]);
    const int dB = C == 0 ? dim[2] : (C == 1 ? dim[0] : dim[1]);
    return (int64_t)dA * dB * ((dC + kRun - 1) / kRun);
}

// Run (ia, ib, w) of record t: base-frame first cell (cx, cy, cz) and length kw.
// (la, lb, lc: the same first cell along the axes A, B and C.)
__device__ __forceinline__ void run_cells(const WarpSmem *S, int t, int ia, int ib, int w, int &cx, int &cy, int &cz,
                                          int &kw, int &la, int &lb, int &lc)
{
    const int C = S->axis[t], A = axis_a(C), B = axis_b(C);
    kw = min(kRun, S->dim[C][t] - w * kRun);
    la = S->lo[A][t] + ia;
    lb = S->lo[B][t] + ib;
    lc = S->lo[C][t] + w * kRun;
    cx = C == 0 ? lc : (C == 1 ? lb : la);
    cy = C == 1 ? lc : (C == 2 ? lb : la);
    cz = C == 2 ? lc : (C == 0 ? lb : la);
}
__device__ __forceinline__ void run_cells(const WarpSmem *S, int t, int ia, int ib, int w, int &cx, int &cy, int &cz,
                                          int &kw)
{
    int la, lb, lc;
    run_cells(S, t, ia, ib, w, cx, cy, cz, kw, la, lb, lc);
}

// Run number `local` of record t (ia fastest, then ib, then w).
__device__ __forceinline__ void run_of(const WarpSmem *S, int t, int local, int &ia, int &ib, int &w, int &cx,
                                       int &cy, int &cz, int &kw)
{
    const int C = S->axis[t];
    const int dA = S->dim[axis_a(C)][t], dB = S->dim[axis_b(C)][t];
    ia = local % dA;
    const int r = local / dA;
    ib = r % dB;
    w = r / dB;
    run_cells(S, t, ia, ib, w, cx, cy, cz, kw);
}

// A record's cell offsets must fit the kQBits-bit fields of a queue entry.
__device__ __forceinline__ bool dims_fit_queue(const int (&dim)[3])
{
    return dim[0] < (1 << 19) && dim[1] < (1 << 19) && dim[2] < (1 << 19);
}

// Unguarded record t as the column clip reads it: vertices relative to the run's first cell
// and relabelled so that axis C is z (to_axis), face normals likewise.  The relabelling is
// bound once per run as three row pointers, (C+1)%3, (C+2)%3 and C, into the record arrays
// (vertex or face i is 3 rows = 96 floats further on; the normals follow the vertices at
// 12 rows = 384 floats), so a fetch is three loads at fixed offsets and no selects.
struct RecordRun {
    const float *va, *vb, *vc;  // &S->v[row][t] for the three rows
    float fa, fb, fc;           // the run's first cell along the same three axes
    __device__ __forceinline__ P3<float> vtx(int i) const
    {
        return mk<float>(va[96 * i] - fa, vb[96 * i] - fb, vc[96 * i] - fc);
    }
    __device__ __forceinline__ P3<float> nrm(int f) const
    {
        return mk<float>(va[384 + 96 * f], vb[384 + 96 * f], vc[384 + 96 * f]);
    }
};
static_assert(offsetof(WarpSmem, n) == offsetof(WarpSmem, v) + 384 * sizeof(float), "RecordRun reads n after v");

// Guarded record t as the guarded pass's column clip reads it: the exact vertices (float32
// vertex plus its rounding residual) in float64, in the exact tetrahedron's positive
// orientation, relative to the run's first cell and relabelled so that axis C is z; the
// outward face normals are formed from them when asked for.  (v - f is exact: both are
// float32 values a few cells apart.)
struct RecordRun64 {
    const WarpSmem *S;
    int t, C;
    float fx, fy, fz;
    bool flip;
    __device__ __forceinline__ double co(int row, float f) const
    {
        return ((double)S->v[row][t] - (double)f) + (double)S->vres[row * 32 + t];
    }
    __device__ __forceinline__ P3<double> vtx(int i) const
    {
        const int k = flip ? (i == 1 ? 2 : (i == 2 ? 1 : i)) : i;
        return to_axis(mk<double>(co(3 * k, fx), co(3 * k + 1, fy), co(3 * k + 2, fz)), C);
    }
    __device__ __forceinline__ P3<double> nrm(int f) const
    {
        int a, b, c;
        face_vertices(f, a, b, c);
        const P3<double> pa = vtx(a);
        return cross(sub(vtx(b), pa), sub(vtx(c), pa));
    }
};

// Classify the box of kw cells from cell (cx, cy, cz) along axis C against record t's
// face planes (classify_cell for kw = 1).
__device__ __forceinline__ int classify_run(const WarpSmem *S, int t, int C, float cx, float cy, float cz, int kw)
{
    bool inside = true, outside = false;
    const float ext = (float)(kw - 1);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const float nx = S->n[3 * f][t], ny = S->n[3 * f + 1][t], nz = S->n[3 * f + 2][t];
        const float nc = C == 0 ? nx : (C == 1 ? ny : nz);
        const float s = fmaf(nx, cx, fmaf(ny, cy, fmaf(nz, cz, -S->e[f][t])));
        inside = inside && (s + fmaf(ext, fmaxf(nc, 0.f), S->pos[f][t]) <= 0.f);
        outside = outside || (s + fmaf(ext, fminf(nc, 0.f), S->neg[f][t]) >= 0.f);
    }
    return outside ? CELL_OUTSIDE : (inside ? CELL_INSIDE : CELL_PARTIAL);
}

// Add m to cell (cx, cy, cz) (base-cell frame) of virtual tetrahedron t: the uniform
// grid (folded / dropped as deposit_cell does) or t's octree leaf block.
template <bool OCT, Acc A>
__device__ __forceinline__ bool deposit_pair(const DepositParams &P, const WarpSmem *S, int t, int cx, int cy, int cz,
                                             double m)
{
    if constexpr (OCT) {
        const int64_t bc = P.bc;
        const int64_t lx = cx - S->org[0][t], ly = cy - S->org[1][t], lz = cz - S->org[2][t];
        cell_add<A>(P, P.out + (int64_t)S->leaf[t] * bc * bc * bc + lx + bc * (ly + bc * lz), m);
        return true;
    } else {
        return deposit_cell<A>(P, (int64_t)S->base[0][t] + cx, (int64_t)S->base[1][t] + cy, (int64_t)S->base[2][t] + cz,
                            m);
    }
}

// Decode queue entry `ent` of record t: the cell (base-cell frame).
__device__ __forceinline__ void q_cell(const WarpSmem *S, unsigned long long ent, int &t, int &cx, int &cy, int &cz)
{
    t = (int)(ent & 31u);
    cx = S->lo[0][t] + (int)((ent >> 5) & kQMask);
    cy = S->lo[1][t] + (int)((ent >> (5 + kQBits)) & kQMask);
    cz = S->lo[2][t] + (int)((ent >> (5 + 2 * kQBits)) & kQMask);
}

template <bool STATS, bool OCT, Acc A>
__device__ __forceinline__ void deposit_clip(const DepositParams &P, const WarpSmem *S, int t, int cx, int cy, int cz,
                                             double vol, Counters &cnt)
{
    if (STATS) cnt.u[ST_PARTIAL_CLIPS]++;
    if (vol > 0.0) {
        if (STATS) cnt.u[ST_OVERLAPPED]++;
        const double m = (double)(S->rho[t] * (float)vol);
        cnt.add_dep(m);
        if (!deposit_pair<OCT, A>(P, S, t, cx, cy, cz, m) && STATS) cnt.dropped += m;
    }
}

// FP32 clips of the first `count` entries of S->q (tetrahedra below the guard).
template <bool STATS, bool OCT, Acc A>
__device__ __forceinline__ void clip_round(const DepositParams &P, WarpSmem *S, int count, int lane, Counters &cnt)
{
    if (lane < count) {
        int t, cx, cy, cz;
        q_cell(S, S->q[lane], t, cx, cy, cz);
        const float fx = (float)cx, fy = (float)cy, fz = (float)cz;
        P3<float> p[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            p[q] = mk<float>(S->v[3 * q][t] - fx, S->v[3 * q + 1][t] - fy, S->v[3 * q + 2][t] - fz);
        P3<float> n[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) n[f] = mk<float>(S->n[3 * f][t], S->n[3 * f + 1][t], S->n[3 * f + 2][t]);
        P3<float> pa[4], na[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            pa[q] = to_axis(p[q], S->axis[t]);
            na[q] = to_axis(n[q], S->axis[t]);
        }
        float err;
        const double vol = (double)overlap_volume_rolled(pa, na, S->lx[t], S->ly[t], err, &S->poly[0][lane]);
        deposit_clip<STATS, OCT, A>(P, S, t, cx, cy, cz, vol, cnt);
    }
    __syncwarp();
}

// Column clips of the first `count` entries of S->q, one run per lane: in float32 (T = float,
// the records below the guard) or in float64 from the exact vertices (T = double, the
// guarded records).  (Dealing the (run, face) jobs and the level fans out over the warp
// raised the active lanes but cost more in shuffles and reloads than it saved: 12% slower.)
template <bool STATS, bool OCT, Acc A, class T>
__device__ __forceinline__ void run_round(const DepositParams &P, WarpSmem *S, int count, int lane, Counters &cnt)
{
    if (lane < count) {
        const unsigned long long ent = S->q[lane];
        const int t = (int)(ent & 31u);
        const int w = (int)((ent >> (5 + 2 * kQBits)) & kQMask);
        const int C = S->axis[t];
        int cx, cy, cz, kw, la, lb, lc;
        run_cells(S, t, (int)((ent >> 5) & kQMask), (int)((ent >> (5 + kQBits)) & kQMask), w, cx, cy, cz, kw, la, lb,
                  lc);
        if (STATS) cnt.u[ST_RUNS]++;
        const bool lo_open = w > 0 || S->cut[t] != 0;
        double vol[kRun];
        if constexpr (sizeof(T) == sizeof(float)) {
            // rows (C+1)%3 = A, (C+2)%3 = B and C, and the run's first cell along them
            const RecordRun src{&S->v[axis_a(C)][t], &S->v[axis_b(C)][t], &S->v[C][t], (float)la, (float)lb, (float)lc};
            float v32[kRun];
            column_volumes<kRun>(src, S->lx[t], S->ly[t], kw, lo_open, v32, &S->poly[0][lane]);
#pragma unroll
            for (int j = 0; j < kRun; ++j) vol[j] = v32[j];
        } else {
            const RecordRun64 src{S, t, C, (float)cx, (float)cy, (float)cz, (S->guard[t] & kGuardFlip) != 0};
            column_volumes<kRun>(src, (double)S->lx[t], (double)S->ly[t], kw, lo_open, vol, S->dpoly + lane);
        }
        const float rho = S->rho[t];
#pragma unroll
        for (int j = 0; j < kRun; ++j) {
            const int ex = cx + (C == 0 ? j : 0), ey = cy + (C == 1 ? j : 0), ez = cz + (C == 2 ? j : 0);
            if (STATS && j < kw) {
                // the same per-cell classification as the cell schedules, for the counters
                P3<float> n[4];
                float e[4], ps[4], ng[4];
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    n[f] = mk<float>(S->n[3 * f][t], S->n[3 * f + 1][t], S->n[3 * f + 2][t]);
                    e[f] = S->e[f][t];
                    ps[f] = S->pos[f][t];
                    ng[f] = S->neg[f][t];
                }
                const int cls = classify_cell<float>(n, e, ps, ng, (float)ex, (float)ey, (float)ez);
                if (cls == CELL_PARTIAL) {
                    cnt.u[ST_PARTIAL_CLIPS]++;
                    if (sizeof(T) != sizeof(float)) cnt.u[ST_FP64_REDOS]++;
                } else if (cls == CELL_INSIDE) {
                    cnt.u[ST_INSIDE_CELLS]++;
                }
            }
            if (j < kw && vol[j] > 0.0) {
                if (STATS) cnt.u[ST_OVERLAPPED]++;
                const double m = (sizeof(T) == sizeof(float)) ? (double)(rho * (float)vol[j]) : (double)rho * vol[j];
                cnt.add_dep(m);
                if (!deposit_pair<OCT, A>(P, S, t, ex, ey, ez, m) && STATS) cnt.dropped += m;
            }
        }
    }
    __syncwarp();
}

// Float64 clips (exact vertices) of the first `count` entries of S->gq.  Guarded pairs
// are queued apart so that these rounds run with full warps.
template <bool STATS, bool OCT, Acc A>
__device__ __forceinline__ void redo_round(const DepositParams &P, WarpSmem *S, int count, int lane, Counters &cnt)
{
    if (lane < count) {
        int t, cx, cy, cz;
        q_cell(S, S->gq[lane], t, cx, cy, cz);
        const double vol = redo_fp64(S, t, cx, cy, cz);
        if (STATS) cnt.u[ST_FP64_REDOS]++;
        deposit_clip<STATS, OCT, A>(P, S, t, cx, cy, cz, vol, cnt);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// The guarded-tetrahedron list.  The FP32 pass already sets up every tetrahedron; it lists
// the guarded multi-cell ones so that the guarded pass visits only those instead of
// generating and setting up every tetrahedron again (on a lattice with few guarded
// tetrahedra that second scan was most of the guarded pass).
// ---------------------------------------------------------------------------
// Append the id of this lane's guarded tetrahedron (want) with one atomic per warp.  Ids past
// the capacity are not stored, but the count still grows, which sends the guarded pass back
// to a full scan.  Called by all 32 lanes.
__device__ __forceinline__ void list_guarded(const DepositParams &P, bool want, int64_t id, int lane)
{
    const unsigned m = __ballot_sync(kFull, want);
    if (m == 0u || P.guard_cap == 0) return;
    unsigned long long first = 0;
    if (lane == 0) first = atomicAdd(&P.ws->guard_count, (unsigned long long)__popc(m));
    first = __shfl_sync(kFull, first, 0);
    if (want) {
        const unsigned long long k = first + (unsigned long long)__popc(m & ((1u << lane) - 1u));
        if (k < (unsigned long long)P.guard_cap) P.guard_list[k] = id;
    }
}

// The guarded pass: the number of listed tetrahedra when the FP32 pass listed all of them,
// else -1 (scan every tetrahedron).
__device__ __forceinline__ int64_t listed_guarded(const DepositParams &P)
{
    if (P.guard_cap == 0) return -1;
    const unsigned long long c = *reinterpret_cast<const volatile unsigned long long *>(&P.ws->guard_count);
    return c > (unsigned long long)P.guard_cap ? -1 : (int64_t)c;
}

// Which records a kernel holds, and so which clips it carries:
//  * kPassAll: records on both sides of the guard, enumerated by cells; FP32 clips and FP64
//    clips in the same kernel (the warp-per-tetrahedron baseline);
//  * kPassFp32: records below the guard only, enumerated by column runs (FP32 column clips);
//  * kPassGuard: guarded records only, enumerated by column runs (FP64 column clips from
//    the exact vertices).
// The warp-cooperative and octree schedules run kPassFp32 and then kPassGuard over the same
// tetrahedra, so neither kernel carries the other's clip code or registers.
enum { kPassAll = 0, kPassFp32 = 1, kPassGuard = 2 };

// Enumerate every (virtual tetrahedron, cell or run) pair of the 32 records in S (npairs:
// this lane's pair count), 32 pairs per round: classify; deposit "cell inside" pairs; queue
// partial pairs and clip them 32 at a time.
template <bool STATS, bool OCT, Acc A, int PASS>
__device__ __forceinline__ void coop_pairs(const DepositParams &P, WarpSmem *S, int lane, int npairs, Counters &cnt)
{
    constexpr bool COL = PASS != kPassAll;  // both passes of the warp schedules clip column runs
    constexpr bool HAS_Q = true;
    constexpr bool HAS_GQ = PASS == kPassAll;
    const unsigned lt_mask = (1u << lane) - 1u;
    int incl = npairs;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    S->start[lane] = incl - npairs;
    __syncwarp();
    // one clip_round call site, so that the clip is inlined once (instruction-cache footprint)
    int qn = 0, gn = 0;
    for (int b0 = 0;; b0 += 32) {
        if (b0 < total) {
            const int idx = b0 + lane;
            bool partial = false, gpartial = false;
            unsigned long long ent = 0;
            if (idx < total) {
                int t = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1)
                    if (S->start[t + step] <= idx && t + step < 32) t += step;
                const int local = idx - S->start[t] + S->skip[t];
                if constexpr (COL) {
                    int ia, ib, w, cx, cy, cz, kw;
                    run_of(S, t, local, ia, ib, w, cx, cy, cz, kw);
                    const int C = S->axis[t];
                    const int cls = classify_run(S, t, C, (float)cx, (float)cy, (float)cz, kw);
                    if (cls == CELL_INSIDE) {
                        const double m = (double)S->rho[t];
                        for (int j = 0; j < kw; ++j) {
                            cnt.add_dep(m);
                            if (!deposit_pair<OCT, A>(P, S, t, cx + (C == 0 ? j : 0), cy + (C == 1 ? j : 0),
                                                      cz + (C == 2 ? j : 0), m) && STATS)
                                cnt.dropped += m;
                        }
                        if (STATS) { cnt.u[ST_INSIDE_CELLS] += kw; cnt.u[ST_OVERLAPPED] += kw; }
                    } else if (cls == CELL_PARTIAL) {
                        ent = q_pack(t, ia, ib, w);
                        partial = true;
                    }
                } else {
                    int ix, iy, iz;
                    decompose(local, S->dim[0][t], S->dim[1][t], ix, iy, iz);
                    const float cx = (float)(S->lo[0][t] + ix), cy = (float)(S->lo[1][t] + iy),
                                cz = (float)(S->lo[2][t] + iz);
                    P3<float> n[4];
                    float e[4], ps[4], ng[4];
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        n[f] = mk<float>(S->n[3 * f][t], S->n[3 * f + 1][t], S->n[3 * f + 2][t]);
                        e[f] = S->e[f][t];
                        ps[f] = S->pos[f][t];
                        ng[f] = S->neg[f][t];
                    }
                    const int cls = classify_cell<float>(n, e, ps, ng, cx, cy, cz);
                    if (cls == CELL_INSIDE) {
                        const double m = (double)S->rho[t];
                        cnt.add_dep(m);
                        if (!deposit_pair<OCT, A>(P, S, t, S->lo[0][t] + ix, S->lo[1][t] + iy, S->lo[2][t] + iz, m) &&
                            STATS)
                            cnt.dropped += m;
                        if (STATS) { cnt.u[ST_INSIDE_CELLS]++; cnt.u[ST_OVERLAPPED]++; }
                    } else if (cls == CELL_PARTIAL) {
                        ent = q_pack(t, ix, iy, iz);
                        if (PASS == kPassGuard || (PASS == kPassAll && S->guard[t])) gpartial = true;
                        else partial = true;
                    }
                }
            }
            if constexpr (HAS_Q) {
                const unsigned bal = __ballot_sync(kFull, partial);
                if (partial) S->q[qn + __popc(bal & lt_mask)] = ent;
                qn += __popc(bal);
            }
            if constexpr (HAS_GQ) {
                const unsigned gbal = __ballot_sync(kFull, gpartial);
                if (gpartial) S->gq[gn + __popc(gbal & lt_mask)] = ent;
                gn += __popc(gbal);
            }
            __syncwarp();
        }
        const bool last = b0 + 32 >= total;
        if constexpr (HAS_Q) {
            if (qn >= 32 || (last && qn > 0)) {
                const int take = qn >= 32 ? 32 : qn;
                if constexpr (PASS == kPassFp32) run_round<STATS, OCT, A, float>(P, S, take, lane, cnt);
                else if constexpr (PASS == kPassGuard) run_round<STATS, OCT, A, double>(P, S, take, lane, cnt);
                else clip_round<STATS, OCT, A>(P, S, take, lane, cnt);
                if (lane < qn - take) S->q[lane] = S->q[take + lane];
                qn -= take;
                __syncwarp();
            }
        }
        if constexpr (HAS_GQ) {
            if (gn >= 32 || (last && gn > 0)) {
                const int take = gn >= 32 ? 32 : gn;
                redo_round<STATS, OCT, A>(P, S, take, lane, cnt);
                if (lane < gn - take) S->gq[lane] = S->gq[take + lane];
                gn -= take;
                __syncwarp();
            }
        }
        if (last && qn == 0 && gn == 0) break;
    }
    cnt.fold_dep();
}


// Each warp's shared memory is a WarpSmem, except in the guarded pass: there the float64
// edge slots ([21][32] double2) take the place of the FP32 ones (poly, the struct's last
// member, which that pass never touches) and run past the struct's end, so a warp needs
// 19 KB instead of 24 and three 4-warp blocks fit an SM.
constexpr size_t kGuardWarpBytes = offsetof(WarpSmem, poly) + sizeof(double2) * 21 * 32;
static_assert(offsetof(WarpSmem, poly) % 16 == 0 && kGuardWarpBytes % 16 == 0 && sizeof(WarpSmem) % 16 == 0,
              "warp blocks of shared memory must keep 16-byte alignment");
PSE_HD constexpr size_t warp_stride(bool guard_slots) { return guard_slots ? kGuardWarpBytes : sizeof(WarpSmem); }

// this warp's block of dynamic shared memory
__device__ __forceinline__ WarpSmem *warp_smem(bool guard_slots)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return reinterpret_cast<WarpSmem *>(smem_raw + (threadIdx.x >> 5) * warp_stride(guard_slots));
}

// Point S->vres at this warp's residual block and, in the guarded pass, S->dpoly at its
// float64 edge slots (every lane writes the same values).
__device__ __forceinline__ void bind_residuals(const DepositParams &P, WarpSmem *S, bool guard_slots = false)
{
    S->vres = P.vres + ((size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (12 * 32);
    if (guard_slots) S->dpoly = reinterpret_cast<double2 *>(&S->poly[0][0]);
    __syncwarp();
}

// dynamic shared memory of a warp kernel with `warps` warps
inline size_t warp_smem_bytes(int warps, bool guard_slots) { return warp_stride(guard_slots) * warps; }

inline int persistent_blocks(const void *kernel, int threads, size_t smem)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

}  // namespace
}  // namespace pse
