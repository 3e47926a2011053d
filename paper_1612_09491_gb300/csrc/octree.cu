// octree.cu -- the adaptive deposit grid (Sec. 4): tetrahedron-size histograms for
// the octree build, and the deposit onto leaf blocks.
//
// Tree: the root is the periodic box; a node at level l has side box/2^l; every leaf
// carries a block of bc^3 cells of side h_l = box/(bc 2^l) (Sec. 4: every leaf patch
// has the same number of cells).  Finest-level nodes (2^max_level per axis) map to
// the leaf that contains them (fine_map), so the leaves a tetrahedron touches are
// found from the finest nodes its bounding box covers.
//
// A tetrahedron overlapping k leaves is deposited as k "virtual" tetrahedra: the
// same tetrahedron expressed in the cell units of that leaf's level, with its cell
// range clipped to the leaf's block.  Each virtual tetrahedron runs through the same
// classification and clip as the uniform grid (common.cuh).
#include "common.cuh"

namespace pse {
namespace {

// Lagrangian tetrahedron as float32 positions plus integer periodic shifts
// (vertex q sits at x[q] + k[q] * box), nearest image to vertex 0.
__device__ __forceinline__ void lattice_tet_raw(const DepositParams &P, int64_t ci, int64_t cj, int64_t ck, int s,
                                                float (&x)[4][3], int (&k)[4][3])
{
    int o1[3], o2[3];
    kuhn_offsets(s, o1, o2);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int64_t i = ci, j = cj, kk = ck;
        if (q == 1) { i += o1[0]; j += o1[1]; kk += o1[2]; }
        if (q == 2) { i += o2[0]; j += o2[1]; kk += o2[2]; }
        if (q == 3) { i += 1; j += 1; kk += 1; }
        if (P.periodic) {
            i = wrap_idx(i, P.n[0]);
            j = wrap_idx(j, P.n[1]);
            if (!P.slab) kk = wrap_idx(kk, P.n[2]);
        }
        const float *p = P.pos + 3 * (i + P.n[0] * (j + P.n[1] * kk));
        x[q][0] = __ldg(p);
        x[q][1] = __ldg(p + 1);
        x[q][2] = __ldg(p + 2);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int sh = 0;
            if (P.periodic && q > 0) {
                const double d = (double)x[q][a] - (double)x[0][a];
                sh = (d >= 0.5 * P.box) ? -1 : ((d < -0.5 * P.box) ? 1 : 0);
            }
            k[q][a] = sh;
        }
}

// The tetrahedron in the cell units of a grid with g cells per side over the box,
// relative to its base cell (the cell of vertex 0).
template <class T>
__device__ __forceinline__ void to_grid(const DepositParams &P, const float (&x)[4][3], const int (&k)[4][3],
                                        int64_t g, P3<T> (&v)[4], int (&base)[3], P3<float> *res = nullptr)
{
    const double sd = (double)g / P.box;
    const float sf = (float)sd;
#pragma unroll
    for (int a = 0; a < 3; ++a) base[a] = safe_floor((double)x[0][a] * sd);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        T c[3];
        float rr[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const long long off = (long long)k[q][a] * g - base[a];
            if constexpr (sizeof(T) == 4) {
                c[a] = fmaf(x[q][a], sf, (float)off);
                if (res) rr[a] = (float)(fma((double)x[q][a], sd, (double)off) - (double)c[a]);
            } else {
                c[a] = fma((double)x[q][a], sd, (double)off);
            }
        }
        v[q] = mk<T>(c[0], c[1], c[2]);
        if (sizeof(T) == 4 && res) res[q] = mk<float>(rr[0], rr[1], rr[2]);
    }
}

__device__ __forceinline__ double unwrapped(const DepositParams &P, const float (&x)[4][3], const int (&k)[4][3],
                                            int q, int a)
{
    return (double)x[q][a] + (double)k[q][a] * P.box;
}

// Range of finest-level nodes covered by the tetrahedron's bounding box (unfolded).
__device__ __forceinline__ void fine_range(const DepositParams &P, const float (&x)[4][3], const int (&k)[4][3],
                                           int64_t (&f0)[3], int64_t (&f1)[3])
{
    const double s = (double)P.fine / P.box;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double mn = unwrapped(P, x, k, 0, a), mx = mn;
#pragma unroll
        for (int q = 1; q < 4; ++q) {
            mn = fmin(mn, unwrapped(P, x, k, q, a));
            mx = fmax(mx, unwrapped(P, x, k, q, a));
        }
        f0[a] = (int64_t)floor(mn * s);
        f1[a] = (int64_t)floor(mx * s);
    }
}

struct LeafHit {
    int leaf;
    int level;
    int64_t org[3];  // the leaf's first cell at its level, unfolded (periodic image of the tetrahedron)
};

// Advance `cursor` over the finest nodes of [f0, f1] until a node that is the first
// node of its (leaf, periodic image) within the range; fills `hit`.  False when done.
__device__ __forceinline__ bool next_leaf(const DepositParams &P, const int64_t (&f0)[3], const int64_t (&f1)[3],
                                          int64_t &cursor, LeafHit &hit)
{
    const int64_t nx = f1[0] - f0[0] + 1, ny = f1[1] - f0[1] + 1, nz = f1[2] - f0[2] + 1;
    const int64_t total = nx * ny * nz;
    const int64_t F = P.fine;
    while (cursor < total) {
        const int64_t c = cursor++;
        const int64_t f[3] = {f0[0] + c % nx, f0[1] + (c / nx) % ny, f0[2] + c / (nx * ny)};
        int64_t g[3];
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            g[a] = P.periodic ? fold_cell(f[a], F) : f[a];
            inside = inside && g[a] >= 0 && g[a] < F;
        }
        if (!inside) continue;
        const int leaf = __ldg(P.fine_map + g[0] + F * (g[1] + F * g[2]));
        const int level = __ldg(P.leaves + 4 * leaf);
        const int64_t span = (int64_t)1 << (P.max_level - level);
        bool first = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int64_t lo = (int64_t)__ldg(P.leaves + 4 * leaf + 1 + a) * span + (f[a] - g[a]);
            first = first && (f[a] == (lo > f0[a] ? lo : f0[a]));
        }
        if (!first) continue;
        hit.leaf = leaf;
        hit.level = level;
        const int64_t gl = (int64_t)P.bc << level;  // cells per side at the leaf's level
#pragma unroll
        for (int a = 0; a < 3; ++a)
            hit.org[a] = (int64_t)__ldg(P.leaves + 4 * leaf + 1 + a) * P.bc + ((f[a] - g[a]) / F) * gl;
        return true;
    }
    return false;
}

// The leaf cell (index into the leaf-mass array) that holds the unwrapped point c.
__device__ __forceinline__ int64_t point_cell(const DepositParams &P, const double (&c)[3], bool &ok)
{
    const int64_t F = P.fine;
    int64_t g[3], img[3];
    ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int64_t f = (int64_t)floor(c[a] * (double)F / P.box);
        g[a] = P.periodic ? fold_cell(f, F) : f;
        img[a] = f - g[a];
        ok = ok && g[a] >= 0 && g[a] < F;
    }
    if (!ok) return 0;
    const int leaf = __ldg(P.fine_map + g[0] + F * (g[1] + F * g[2]));
    const int level = __ldg(P.leaves + 4 * leaf);
    const int64_t bc = P.bc, gl = bc << level;
    int64_t idx = (int64_t)leaf * bc * bc * bc, stride = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double u = c[a] * (double)gl / P.box;
        int64_t cc = (int64_t)floor(u) - ((int64_t)__ldg(P.leaves + 4 * leaf + 1 + a) * bc + (img[a] / F) * gl);
        cc = cc < 0 ? 0 : (cc >= bc ? bc - 1 : cc);
        idx += cc * stride;
        stride *= bc;
    }
    return idx;
}

__device__ __forceinline__ void tet_centroid(const DepositParams &P, const float (&x)[4][3], const int (&k)[4][3],
                                             double (&c)[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
        c[a] = 0.25 * (unwrapped(P, x, k, 0, a) + unwrapped(P, x, k, 1, a) + unwrapped(P, x, k, 2, a) +
                       unwrapped(P, x, k, 3, a));
}

__device__ __forceinline__ double det6_box(const DepositParams &P, const float (&x)[4][3], const int (&k)[4][3])
{
    double e[3][3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int a = 0; a < 3; ++a) e[q][a] = unwrapped(P, x, k, q + 1, a) - unwrapped(P, x, k, 0, a);
    return e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
}

template <Acc A = Acc::RUNTIME>
__device__ __forceinline__ void add_mass(const DepositParams &P, const double (&c)[3], double m, Counters &cnt,
                                         bool stats)
{
    bool ok;
    const int64_t idx = point_cell(P, c, ok);
    if (ok) cell_add<A>(P, P.out + idx, m);
    else if (stats) cnt.dropped += m;
}

// ---------------------------------------------------------------------------
// thread per tetrahedron (T = double: the plain FP64 octree path)
// ---------------------------------------------------------------------------
template <class T, bool STATS>
__global__ void __launch_bounds__(128) k_oct_thread(const DepositParams P)
{
    Counters cnt;
    if (STATS) cnt.zero();
    cnt.zero_mass();
    const int64_t n_tets = 6 * P.n_units;
    const int64_t bc = P.bc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tets;
         t += (int64_t)gridDim.x * blockDim.x) {
        cnt.fold_dep();  // the previous tetrahedron's deposits
        int64_t ci, cj, ck;
        if (!cube_of_unit(P, t / 6, ci, cj, ck)) {
            set_error(P.ws, 3, (int)((t / 6) & 0x7fffffff));
            continue;
        }
        float x[4][3];
        int k[4][3];
        lattice_tet_raw(P, ci, cj, ck, (int)(t % 6), x, k);
        const double m_t = P.m_tet;
        if (STATS) {
            cnt.u[ST_TETS]++;
            cnt.mass_in += m_t;
            cnt.u[ST_INVERTED] += ((det6_box(P, x, k) < 0.0) != kuhn_negative((int)(t % 6))) ? 1 : 0;
        }
        cnt.add_tgt(P, m_t);
        double cen[3];
        tet_centroid(P, x, k, cen);
        if (det6_box(P, x, k) == 0.0) {
            add_mass(P, cen, m_t, cnt, STATS);
            cnt.add_dep(m_t);
            if (STATS) { cnt.u[ST_DEGENERATE]++; cnt.u[ST_OVERLAPPED]++; }
            continue;
        }
        int64_t f0[3], f1[3];
        fine_range(P, x, k, f0, f1);
        int64_t cursor = 0;
        LeafHit hit;
        while (next_leaf(P, f0, f1, cursor, hit)) {
            P3<T> v[4];
            P3<float> res[4];
            int base[3];
            to_grid<T>(P, x, k, bc << hit.level, v, base, res);
            TetSetup<T> ts;
            if (tet_setup<T>(v, ts)) swap12(res);
            if (!tet_ok(base, ts)) {
                set_error(P.ws, 4, (int)(t & 0x7fffffff));
                break;
            }
            // cell range of the tetrahedron clipped to this leaf's block (base-cell frame)
            int lo[3], hi[3], org[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                org[a] = (int)(hit.org[a] - base[a]);
                lo[a] = ts.lo[a] > org[a] ? ts.lo[a] : org[a];
                hi[a] = ts.lo[a] + ts.dim[a] - 1 < org[a] + (int)bc - 1 ? ts.lo[a] + ts.dim[a] - 1 : org[a] + (int)bc - 1;
            }
            const bool single = ts.dim[0] == 1 && ts.dim[1] == 1 && ts.dim[2] == 1;
            const bool g64 = (sizeof(T) == 4) && !(ts.kappa <= P.kappa_max) && !single;
            double rho = 6.0 * m_t / ts.vol6;
            if constexpr (sizeof(T) == 4) {
                if (g64) rho = 6.0 * m_t / exact_vol6(ts.v, res, ts.vol6);
            }
            double* blk = P.out + (int64_t)hit.leaf * bc * bc * bc;
            for (int cz = lo[2]; cz <= hi[2]; ++cz)
                for (int cy = lo[1]; cy <= hi[1]; ++cy)
                    for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                        if (STATS) cnt.u[ST_BBOX_CELLS]++;
                        double vol = 0.0;
                        if (single) {
                            vol = ts.vol6 / 6.0;
                            if (STATS) { cnt.u[ST_SINGLE_CELL]++; cnt.u[ST_OVERLAPPED]++; }
                        } else {
                            const int cls = classify_cell<T>(ts.n, ts.e, ts.pos, ts.neg, (T)cx, (T)cy, (T)cz);
                            if (cls == CELL_INSIDE) {
                                vol = 1.0;
                                if (STATS) cnt.u[ST_INSIDE_CELLS]++;
                            } else if (cls == CELL_PARTIAL) {
                                P3<T> p[4];
#pragma unroll
                                for (int q = 0; q < 4; ++q)
                                    p[q] = mk<T>(ts.v[q].x - (T)cx, ts.v[q].y - (T)cy, ts.v[q].z - (T)cz);
                                if constexpr (sizeof(T) == 4) {
                                    if (g64) {
                                        P3<double> pd[4];
                                        exact_vertices(ts.v, res, cx, cy, cz, pd);
                                        vol = overlap_volume_fp64(pd);
                                        if (STATS) cnt.u[ST_FP64_REDOS]++;
                                    } else {
                                        T err;
                                        vol = (double)overlap_volume_ax<T>(p, ts.n, ts.axis, ts.lx, ts.ly, err);
                                    }
                                } else {
                                    T err;
                                    vol = (double)overlap_volume_ax<T>(p, ts.n, ts.axis, ts.lx, ts.ly, err);
                                }
                                if (STATS) cnt.u[ST_PARTIAL_CLIPS]++;
                            }
                        }
                        if (vol > 0.0) {
                            if (STATS) cnt.u[ST_OVERLAPPED]++;
                            const double m = rho * vol;
                            cnt.add_dep(m);
                            cell_add(P, blk + (cx - org[0]) + bc * ((cy - org[1]) + bc * (cz - org[2])), m);
                        }
                    }
        }
    }
    if (STATS) cnt.flush(P.ws);
    if (P.fixup || STATS) cnt.flush_mass(P, P.ws);
}

// ---------------------------------------------------------------------------
// warp-cooperative FP32 path: per sub-batch, rounds of (tetrahedron, leaf) pairs
// ---------------------------------------------------------------------------
// PASS kPassFp32 visits every (tetrahedron, leaf) pair: it counts the tetrahedra, deposits
// degenerate ones and those inside one cell of a leaf, and clips the pairs below the guard by
// column runs.  PASS kPassGuard visits the pairs again and clips only the guarded ones, by
// column runs in FP64.
template <bool STATS, int MINB, Acc A, int PASS>
__global__ void __launch_bounds__(128, MINB) k_oct_warp(const DepositParams P)
{
    constexpr bool FIRST = PASS == kPassFp32;
    WarpSmem *S = warp_smem(!FIRST);
    bind_residuals(P, S, !FIRST);
    const int lane = threadIdx.x & 31;
    Counters cnt;
    if (STATS) cnt.zero();
    cnt.zero_mass();
    const int64_t bc = P.bc;
    // the guarded pass: the tetrahedra the FP32 pass listed, 32 per item, when it listed all
    const int64_t listed = FIRST ? -1 : listed_guarded(P);
    const bool LIST = listed >= 0;
    const int64_t n_items = LIST ? (listed + 31) / 32 : P.n_items;

    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(FIRST ? &P.ws->work_counter : &P.ws->work_counter2, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if ((int64_t)item >= n_items) break;
        int64_t ci = 0, cj = 0, ck = 0;
        int s_listed = 0;
        bool have = false;
        if (LIST) {
            const int64_t k = (int64_t)item * 32 + lane;
            if (k < listed) {  // id = 6 (ci + nc0 (cj + nc1 ck)) + s, whatever the source
                const int64_t id = P.guard_list[k];
                const int64_t c = id / 6;
                s_listed = (int)(id % 6);
                ci = c % P.nc[0];
                cj = (c / P.nc[0]) % P.nc[1];
                ck = c / (P.nc[0] * P.nc[1]);
                have = true;
            }
        } else if (P.src == SRC_LATTICE) {
            const int64_t segs = (P.nc[0] + 31) / 32;
            const int64_t row = (int64_t)item / segs, seg = (int64_t)item % segs;
            const int64_t i = seg * 32 + lane;
            if (i < P.nc[0]) {
                ci = i;
                cj = row % P.nc[1];
                ck = row / P.nc[1];
                have = true;
            }
        } else {
            const int64_t u = (int64_t)item * 32 + lane;
            if (u < P.n_units) {
                have = cube_of_unit(P, u, ci, cj, ck);
                if (!have) set_error(P.ws, 3, (int)(u & 0x7fffffff));
            }
        }
        for (int si = 0; si < (LIST ? 1 : 6); ++si) {
            const int s = LIST ? s_listed : si;
            bool to_list = false;  // the FP32 pass: a pair of this tetrahedron is guarded
            float x[4][3];
            int k[4][3];
            double cen[3] = {0.0, 0.0, 0.0};
            const double m_t = P.m_tet;
            bool live = false;
            int64_t f0[3] = {0, 0, 0}, f1[3] = {-1, -1, -1}, cursor = 0;
            if (have) {
                lattice_tet_raw(P, ci, cj, ck, s, x, k);
                if (STATS && FIRST) {
                    cnt.u[ST_TETS]++;
                    cnt.mass_in += m_t;
                    cnt.u[ST_INVERTED] += ((det6_box(P, x, k) < 0.0) != kuhn_negative(s)) ? 1 : 0;
                }
                if (FIRST) cnt.add_tgt(P, m_t);
                if (det6_box(P, x, k) == 0.0) {
                    if (FIRST) {
                        tet_centroid(P, x, k, cen);
                        add_mass<A>(P, cen, m_t, cnt, STATS);
                        cnt.add_dep(m_t);
                        if (STATS) { cnt.u[ST_DEGENERATE]++; cnt.u[ST_OVERLAPPED]++; }
                    }
                } else {
                    fine_range(P, x, k, f0, f1);
                    live = true;
                }
            }
            bool more = live;
            while (__any_sync(kFull, more)) {
                int npairs = 0;
                if (more) {
                    LeafHit hit;
                    more = next_leaf(P, f0, f1, cursor, hit);
                    if (more) {
                        P3<float> v[4], res[4];
                        int base[3];
                        to_grid<float>(P, x, k, bc << hit.level, v, base);
                        TetSetup<float> ts;
                        const bool swapped = tet_setup<float>(v, ts);
                        const bool guard = !(ts.kappa <= P.kappa_max);
#pragma unroll
                        for (int q = 0; q < 4; ++q) res[q] = mk<float>(0.f, 0.f, 0.f);
                        if (!FIRST && guard) {  // rounding residuals for the guarded clip
                            P3<float> v2[4];
                            int b2[3];
                            to_grid<float>(P, x, k, bc << hit.level, v2, b2, res);
                            if (swapped) swap12(res);
                        }
                        const bool single = ts.dim[0] == 1 && ts.dim[1] == 1 && ts.dim[2] == 1;
                        if (!tet_ok(base, ts)) {
                            set_error(P.ws, 4, lane);
                            more = false;
                        } else {
                            int lo[3], dim[3];
#pragma unroll
                            for (int a = 0; a < 3; ++a) {
                                const int org = (int)(hit.org[a] - base[a]);
                                lo[a] = ts.lo[a] > org ? ts.lo[a] : org;
                                const int hi = ts.lo[a] + ts.dim[a] - 1 < org + (int)bc - 1 ? ts.lo[a] + ts.dim[a] - 1
                                                                                            : org + (int)bc - 1;
                                dim[a] = hi - lo[a] + 1;
                                S->org[a][lane] = org;
                            }
                            const int64_t ncell = (int64_t)dim[0] * dim[1] * dim[2];
                            if (!FIRST && (single || !guard)) {
                                // the guarded pass: nothing to do for this pair
                            } else if (single) {
                                // whole tetrahedron inside one cell of this leaf
                                cell_add<A>(P, P.out + (int64_t)hit.leaf * bc * bc * bc + (lo[0] - S->org[0][lane]) +
                                              bc * ((lo[1] - S->org[1][lane]) + bc * (lo[2] - S->org[2][lane])),
                                          m_t);
                                cnt.add_dep(m_t);
                                if (STATS) { cnt.u[ST_SINGLE_CELL]++; cnt.u[ST_BBOX_CELLS]++; cnt.u[ST_OVERLAPPED]++; }
                            } else if (ncell > (int64_t)(1 << 25) || !dims_fit_queue(dim)) {
                                set_error(P.ws, 2, lane);
                            } else if (FIRST && guard) {
                                // left to the guarded pass; counted here
                                to_list = true;
                                if (STATS) { cnt.u[ST_BBOX_CELLS] += ncell; cnt.u[ST_BIN0 + size_bin(ncell)]++; }
                            } else if (ncell > 0) {
                                npairs = (int)run_count(dim, ts.axis);
                                if (STATS && FIRST) {
                                    cnt.u[ST_BBOX_CELLS] += ncell;
                                    cnt.u[ST_BIN0 + size_bin(ncell)]++;
                                }
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
                                    S->lo[a][lane] = lo[a];
                                    S->dim[a][lane] = dim[a];
                                    S->base[a][lane] = base[a];
                                }
                                S->leaf[lane] = hit.leaf;
                                bool flip = false;
                                S->rho[lane] = guard ? (float)(6.0 * m_t / exact_vol6(ts.v, res, ts.vol6, &flip))
                                                     : __fdiv_rn((float)(6.0 * m_t), (float)ts.vol6);
                                S->lx[lane] = ts.lx;
                                S->ly[lane] = ts.ly;
                                S->axis[lane] = ts.axis;
                                S->guard[lane] = guard ? (1 | (flip ? kGuardFlip : 0)) : 0;
                                S->skip[lane] = 0;
                                {
                                    const int C = ts.axis;
                                    S->cut[lane] = (C == 0 ? lo[0] > ts.lo[0] : (C == 1 ? lo[1] > ts.lo[1] : lo[2] > ts.lo[2]))
                                                       ? 1 : 0;
                                }
                                if (guard) store_residuals(S, lane, res);
                            }
                        }
                    }
                }
                coop_pairs<STATS, true, A, PASS>(P, S, lane, npairs, cnt);
                __syncwarp();
            }
            __syncwarp();
            if (FIRST) list_guarded(P, to_list, 6 * (ci + P.nc[0] * (cj + P.nc[1] * ck)) + s, lane);
        }
    }
    if (STATS) cnt.flush(P.ws);
    if (P.fixup || STATS) cnt.flush_mass(P, P.ws);
}

// ---------------------------------------------------------------------------
// octree build: per-level histograms of the tetrahedra's mean edge length
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t hist_offset(int level) { return (int64_t)64 * ((((int64_t)1) << (3 * level)) - 1) / 7; }

// One pass over the tetrahedra: per level 0 .. max_level-1, the node that holds the
// tetrahedron's vertex centroid and the 64-bin log10 histogram bin of its mean edge length
// in that level's cells.  A lane takes one Lagrangian cube (a warp: 32 neighbouring cubes of a
// row) and its 6 Kuhn tetrahedra, which all start at corner 000: the 7 other corners are
// loaded once, unwrapped once (offsets from corner 000 formed in float64 and rounded to
// float32; a bin is 24% wide), and the 19 distinct edges serve all 6 tetrahedra.  The
// centroid is summed in float64 from the same offsets, and the nodes of the coarser levels
// are the finest level's node coordinates shifted (scaling by 2^l commutes with rounding).
// Equal (node, bin) keys are merged in the warp before one atomic per key.
__global__ void __launch_bounds__(256) k_tet_size_hist(const DepositParams P, unsigned *__restrict__ hist)
{
    __shared__ unsigned sh[64 + 512];  // levels 0 and 1 aggregated per block
    for (int i = threadIdx.x; i < 576; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int levels = P.max_level;  // decisions are made for levels 0 .. max_level-1
    const double inv_box = 1.0 / P.box;
    const float h0 = (float)(P.box / (double)P.bc);
    const bool rows = P.src == SRC_LATTICE;
    const int64_t segs = (P.nc[0] + 31) / 32;
    const int64_t n_items = rows ? segs * P.nc[1] * P.nc[2] : (P.n_units + 31) / 32;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int top = levels > 0 ? levels - 1 : 0;  // the finest decision level
    const double top_scale = (double)((int64_t)1 << top);
    // whole warps iterate together (the merge below needs every lane)
    for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < n_items; item += warps) {
        int64_t ci = 0, cj = 0, ck = 0;
        bool ok = false;
        if (rows) {
            const int64_t row = item / segs, i = (item % segs) * 32 + lane;
            if (i < P.nc[0]) {
                ci = i;
                cj = row % P.nc[1];
                ck = row / P.nc[1];
                ok = true;
            }
        } else {
            const int64_t u = item * 32 + lane;
            ok = u < P.n_units && cube_of_unit(P, u, ci, cj, ck);
        }
        // corner c = (bit 0: +x, bit 1: +y, bit 2: +z): offsets from corner 000
        float x0[3] = {0.f, 0.f, 0.f}, r[8][3];
        double d[8][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) { r[0][a] = 0.f; d[0][a] = 0.0; }
        if (ok) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                int64_t i = ci + (c & 1), j = cj + ((c >> 1) & 1), kk = ck + ((c >> 2) & 1);
                if (P.periodic) {
                    i = wrap_idx(i, P.n[0]);
                    j = wrap_idx(j, P.n[1]);
                    if (!P.slab) kk = wrap_idx(kk, P.n[2]);
                }
                const float *pp = P.pos + 3 * (i + P.n[0] * (j + P.n[1] * kk));
                float x[3] = {__ldg(pp), __ldg(pp + 1), __ldg(pp + 2)};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (c == 0) {
                        x0[a] = x[a];
                    } else {
                        const double raw = (double)x[a] - (double)x0[a];
                        const int sh = P.periodic ? ((raw >= 0.5 * P.box) ? -1 : ((raw < -0.5 * P.box) ? 1 : 0)) : 0;
                        d[c][a] = raw + (double)sh * P.box;
                        r[c][a] = (float)d[c][a];
                    }
                }
            }
        }
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            int o1[3], o2[3];
            kuhn_offsets(s, o1, o2);
            const int c1 = o1[0] | (o1[1] << 1) | (o1[2] << 2), c2 = o2[0] | (o2[1] << 1) | (o2[2] << 2);
            const int cq[4] = {0, c1, c2, 7};
            float me = 0.f;  // mean edge length in level-0 cells
            int64_t top_c[3] = {0, 0, 0};
            if (ok) {
                float es = 0.f;
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = a + 1; b < 4; ++b) {
                        const float dx = r[cq[b]][0] - r[cq[a]][0], dy = r[cq[b]][1] - r[cq[a]][1],
                                    dz = r[cq[b]][2] - r[cq[a]][2];
                        es += sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    }
                me = es * (1.f / 6.f) / h0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    double cen = (double)x0[a] + 0.25 * ((d[c1][a] + d[c2][a]) + d[7][a]);
                    cen -= P.box * floor(cen * inv_box);
                    if (!(cen < P.box) || !(cen >= 0.0)) cen = 0.0;
                    int64_t c = (int64_t)floor(cen * top_scale * inv_box);
                    const int64_t nn = (int64_t)1 << top;
                    top_c[a] = c < 0 ? 0 : (c >= nn ? nn - 1 : c);
                }
            }
            for (int l = 0; l < levels; ++l) {
                unsigned long long key = ~0ull - (unsigned long long)lane;  // lanes without a cube match nothing
                int bin = 0;
                int64_t node = 0;
                if (ok) {
                    const int sh = top - l;
                    node = (top_c[0] >> sh) + ((top_c[1] >> sh) << l) + ((top_c[2] >> sh) << (2 * l));
                    // a level-l cell is 2^-l of a level-0 cell (an exact float scaling)
                    bin = (int)floorf((log10f(ldexpf(me, l)) + 3.0f) * (64.0f / 6.0f));
                    bin = bin < 0 ? 0 : (bin > 63 ? 63 : bin);
                    key = (unsigned long long)node * 64 + (unsigned long long)bin;
                }
                const unsigned peers = __match_any_sync(kFull, key);
                if (ok && lane == __ffs(peers) - 1) {
                    const unsigned cnt = (unsigned)__popc(peers);
                    if (l == 0) atomicAdd(&sh[bin], cnt);
                    else if (l == 1) atomicAdd(&sh[64 + node * 64 + bin], cnt);
                    else atomicAdd(&hist[hist_offset(l) + node * 64 + bin], cnt);
                }
            }
        }
    }
    __syncthreads();
    const int agg = levels >= 2 ? 576 : (levels == 1 ? 64 : 0);
    for (int i = threadIdx.x; i < agg; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

}  // namespace

namespace {
// ---------------------------------------------------------------------------
// Restriction up the tree: the masses of every node of levels 0 .. max_level-1 on its
// own bc^3 block (leaves: their block; internal nodes: each cell the sum of the 8 cells
// of the level below that it covers; nodes below a leaf: 0).  One launch per level,
// finest first, so that an internal node's children are complete when it is summed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t level_offset(int l)
{
    int64_t o = 0;
    for (int k = 0; k < l; ++k) o += (int64_t)1 << (3 * k);
    return o;
}

// leaf record of the finest node below node (l, x, y, z), and its level
__device__ __forceinline__ int leaf_below(const int32_t *fine_map, const int32_t *leaves, int max_level, int l,
                                          int64_t x, int64_t y, int64_t z, int &leaf_level)
{
    const int64_t F = (int64_t)1 << max_level, s = (int64_t)1 << (max_level - l);
    const int leaf = fine_map[x * s + F * (y * s + F * (z * s))];
    leaf_level = leaves[4 * leaf];
    return leaf;
}

__global__ void __launch_bounds__(256) k_restrict_level(const int32_t *__restrict__ fine_map,
                                                        const int32_t *__restrict__ leaves, int max_level, int bc,
                                                        int l, const double *__restrict__ leaf_mass,
                                                        double *__restrict__ pyramid)
{
    const int64_t nn = (int64_t)1 << l, bc3 = (int64_t)bc * bc * bc;
    const int64_t total = nn * nn * nn * bc3;
    const int64_t row0 = level_offset(l), row1 = level_offset(l + 1);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = idx / bc3, cell = idx % bc3;
        const int64_t nx = node % nn, ny = (node / nn) % nn, nz = node / (nn * nn);
        const int ci = (int)(cell % bc), cj = (int)((cell / bc) % bc), ck = (int)(cell / ((int64_t)bc * bc));
        int ll;
        const int leaf = leaf_below(fine_map, leaves, max_level, l, nx, ny, nz, ll);
        double v = 0.0;
        if (ll == l) {
            v = leaf_mass[(int64_t)leaf * bc3 + cell];
        } else if (ll > l) {
            for (int d = 0; d < 8; ++d) {
                const int fx = 2 * ci + (d & 1), fy = 2 * cj + ((d >> 1) & 1), fz = 2 * ck + (d >> 2);
                const int64_t cx = 2 * nx + fx / bc, cy = 2 * ny + fy / bc, cz = 2 * nz + fz / bc;
                const int64_t lc = (fx % bc) + (int64_t)bc * ((fy % bc) + (int64_t)bc * (fz % bc));
                int cl;
                const int cleaf = leaf_below(fine_map, leaves, max_level, l + 1, cx, cy, cz, cl);
                if (cl == l + 1) {
                    v += leaf_mass[(int64_t)cleaf * bc3 + lc];
                } else {
                    const int64_t cn = 2 * nn;
                    v += pyramid[(row1 + cx + cn * (cy + cn * cz)) * bc3 + lc];
                }
            }
        }
        pyramid[(row0 + node) * bc3 + cell] = v;
    }
}
}  // namespace

cudaError_t launch_octree_restrict(const int32_t *fine_map, const int32_t *leaves, int max_level, int bc,
                                   const double *leaf_mass, double *pyramid, cudaStream_t st)
{
    for (int l = max_level - 1; l >= 0; --l) {
        const int64_t total = ((int64_t)1 << (3 * l)) * (int64_t)bc * bc * bc;
        int64_t blocks = (total + 255) / 256;
        if (blocks > 152 * 64) blocks = 152 * 64;
        if (blocks < 1) blocks = 1;
        k_restrict_level<<<(unsigned)blocks, 256, 0, st>>>(fine_map, leaves, max_level, bc, l, leaf_mass, pyramid);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {
// ---------------------------------------------------------------------------
// The paper's refinement criterion (Sec. 4): the Lagrangian lattice is cut into
// subblocks of S^3 cubes; the axis-aligned bounding box of each subblock's particles
// (unwrapped around its first particle) stands for its 6 S^3 tetrahedra, spread evenly.
// A node's estimated tetrahedron count is the sum over subblocks of 6 * cubes *
// vol(box ∩ node) / vol(box), periodic images included.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_subblock_boxes(const float *__restrict__ pos, int64_t n0, int64_t n1,
                                                        int64_t n2, int s, double box, double *__restrict__ boxes)
{
    const int64_t b0 = (n0 + s - 1) / s, b1 = (n1 + s - 1) / s, b2 = (n2 + s - 1) / s;
    const int64_t nb = b0 * b1 * b2;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bx = b % b0, by = (b / b0) % b1, bz = b / (b0 * b1);
        const int64_t i0 = bx * s, j0 = by * s, k0 = bz * s;
        const int64_t i1 = min(n0, i0 + s), j1 = min(n1, j0 + s), k1 = min(n2, k0 + s);  // cubes [i0, i1)
        const float *r = pos + 3 * (i0 + n0 * (j0 + n1 * k0));
        const double rx = r[0], ry = r[1], rz = r[2];
        double lo[3] = {rx, ry, rz}, hi[3] = {rx, ry, rz};
        for (int64_t k = k0; k <= k1; ++k)
            for (int64_t j = j0; j <= j1; ++j)
                for (int64_t i = i0; i <= i1; ++i) {
                    const int64_t ii = i % n0, jj = j % n1, kk = k % n2;
                    const float *p = pos + 3 * (ii + n0 * (jj + n1 * kk));
                    const double ref[3] = {rx, ry, rz};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        double d = (double)p[a] - ref[a];
                        d -= (d >= 0.5 * box) ? box : ((d < -0.5 * box) ? -box : 0.0);
                        lo[a] = fmin(lo[a], ref[a] + d);
                        hi[a] = fmax(hi[a], ref[a] + d);
                    }
                }
        double *o = boxes + 7 * b;
        for (int a = 0; a < 3; ++a) {
            o[a] = lo[a];
            o[3 + a] = hi[a];
        }
        o[6] = 6.0 * (double)((i1 - i0) * (j1 - j0) * (k1 - k0));  // tetrahedra of the subblock
    }
}

// overlap length of [lo, hi] with [x0, x1] over the periodic images of the interval
__device__ __forceinline__ double overlap_1d(double lo, double hi, double x0, double x1, double box)
{
    double len = 0.0;
#pragma unroll
    for (int sgn = -1; sgn <= 1; ++sgn) {
        const double a = fmax(lo + sgn * box, x0), b = fmin(hi + sgn * box, x1);
        len += fmax(b - a, 0.0);
    }
    return len;
}

// one block per node of `nodes` (level, ix, iy, iz): estimated tetrahedra overlapping it
__global__ void __launch_bounds__(256) k_node_counts(const double *__restrict__ boxes, int64_t nb,
                                                     const int32_t *__restrict__ nodes, double box,
                                                     double *__restrict__ counts)
{
    __shared__ double part[256];
    const int32_t *nd = nodes + 4 * blockIdx.x;
    const double size = box / (double)(1 << nd[0]);
    const double x0 = nd[1] * size, y0 = nd[2] * size, z0 = nd[3] * size;
    double sum = 0.0;
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
        const double *o = boxes + 7 * b;
        const double vx = o[3] - o[0], vy = o[4] - o[1], vz = o[5] - o[2];
        const double vol = vx * vy * vz;
        if (!(vol > 0.0)) continue;
        const double ov = overlap_1d(o[0], o[3], x0, x0 + size, box) * overlap_1d(o[1], o[4], y0, y0 + size, box) *
                          overlap_1d(o[2], o[5], z0, z0 + size, box);
        sum += o[6] * ov / vol;
    }
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[blockIdx.x] = part[0];
}
}  // namespace

cudaError_t launch_subblock_boxes(const float *pos, const int64_t n[3], int s, double box, double *boxes,
                                  cudaStream_t st)
{
    const int64_t nb = ((n[0] + s - 1) / s) * ((n[1] + s - 1) / s) * ((n[2] + s - 1) / s);
    int64_t blocks = (nb + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_subblock_boxes<<<(unsigned)blocks, 256, 0, st>>>(pos, n[0], n[1], n[2], s, box, boxes);
    return cudaGetLastError();
}

cudaError_t launch_node_counts(const double *boxes, int64_t nb, const int32_t *nodes, int64_t n_nodes, double box,
                               double *counts, cudaStream_t st)
{
    if (n_nodes < 1) return cudaSuccess;
    k_node_counts<<<(unsigned)n_nodes, 256, 0, st>>>(boxes, nb, nodes, box, counts);
    return cudaGetLastError();
}

cudaError_t launch_octree_hist(const DepositParams &p, unsigned *hist, cudaStream_t st)
{
    const int threads = 256;
    const int64_t n = p.n_units;  // one lane per cube
    int64_t blocks = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)persistent_blocks((const void *)k_tet_size_hist, threads, 0) * 4;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_tet_size_hist<<<(unsigned)blocks, threads, 0, st>>>(p, hist);
    return cudaGetLastError();
}

namespace {
template <int PASS>
cudaError_t launch_oct_pass(const DepositParams &p, bool stats, int blocks_per_sm, cudaStream_t st)
{
    // blocks_per_sm resident blocks of 128 threads: 2 (255 registers), 3 (170) or 4 (128);
    // the counting variant (stats) is built for 2 only
    const int threads = 128;
    constexpr bool GUARD = PASS == kPassGuard;
    const size_t smem = warp_smem_bytes(threads / 32, GUARD);
    // the guarded pass runs 2 blocks per SM (190 registers): its FP64 pipe is already the
    // bottleneck there (84% busy), so more residency would not help
    const int minb = (stats || GUARD) ? 2 : (blocks_per_sm >= 4 ? 4 : (blocks_per_sm == 3 ? 3 : 2));
    const void *k;
    if constexpr (GUARD) {
        k = p.comp ? (stats ? (const void *)k_oct_warp<true, 2, Acc::COMP, PASS> : (const void *)k_oct_warp<false, 2, Acc::COMP, PASS>)
                   : (stats ? (const void *)k_oct_warp<true, 2, Acc::F64, PASS> : (const void *)k_oct_warp<false, 2, Acc::F64, PASS>);
    } else {
        k = p.comp ? (stats ? (const void *)k_oct_warp<true, 2, Acc::COMP, PASS>
                      : minb == 4 ? (const void *)k_oct_warp<false, 4, Acc::COMP, PASS>
                      : minb == 3 ? (const void *)k_oct_warp<false, 3, Acc::COMP, PASS>
                                  : (const void *)k_oct_warp<false, 2, Acc::COMP, PASS>)
            : (stats ? (const void *)k_oct_warp<true, 2, Acc::F64, PASS>
               : minb == 4 ? (const void *)k_oct_warp<false, 4, Acc::F64, PASS>
               : minb == 3 ? (const void *)k_oct_warp<false, 3, Acc::F64, PASS>
                           : (const void *)k_oct_warp<false, 2, Acc::F64, PASS>);
    }
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int blocks = persistent_blocks(k, threads, smem);
    if (blocks > kMaxWarpBlocks) blocks = kMaxWarpBlocks;
    const int64_t need = (p.n_items + 3) / 4;
    if (need < blocks) blocks = (int)(need < 1 ? 1 : need);
    void *args[] = {const_cast<DepositParams *>(&p)};
    return cudaLaunchKernel(k, dim3(blocks), dim3(threads), args, smem, st);
}
}  // namespace

cudaError_t launch_octree_deposit(const DepositParams &p, bool fp64, bool thread_per_tet, bool stats,
                                  int blocks_per_sm, cudaStream_t st)
{
    if (thread_per_tet) {
        const int threads = 128;
        const void *k = fp64 ? (stats ? (const void *)k_oct_thread<double, true> : (const void *)k_oct_thread<double, false>)
                             : (stats ? (const void *)k_oct_thread<float, true> : (const void *)k_oct_thread<float, false>);
        int64_t blocks = (6 * p.n_units + threads - 1) / threads;
        const int64_t cap = (int64_t)persistent_blocks(k, threads, 0) * 8;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        void *args[] = {const_cast<DepositParams *>(&p)};
        return cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(threads), args, 0, st);
    }
    // the FP32 pass, then the guarded pass over the same pairs
    cudaError_t err = launch_oct_pass<kPassFp32>(p, stats, blocks_per_sm, st);
    if (err != cudaSuccess) return err;
    return launch_oct_pass<kPassGuard>(p, stats, blocks_per_sm, st);
}

}  // namespace pse
