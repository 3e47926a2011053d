// deposit.cu -- tetrahedron deposit kernels for sm_103a.
//
//  * k_thread_per_tet<T>: one thread per tetrahedron walks its bounding-box cells,
//    classifies each, clips the partial ones and adds m_t V_ov/|V_t| with a global
//    float64 atomic.  With T = double this is the plain FP64 baseline.
//  * k_warp_coop: one warp takes a batch of 32 tetrahedra (32 Lagrangian cubes x
//    one Kuhn permutation), enumerates all their (tetrahedron, cell) pairs 32 at a
//    time, classifies them in lock-step, deposits "cell inside tetrahedron" pairs
//    at once and compacts the partial pairs into a per-warp queue; whenever 32 are
//    queued every lane clips one (FP32, in registers).  Tetrahedra whose conditioning
//    estimate exceeds the guard are clipped in FP64.  This is the role of the paper's
//    warp-per-tetrahedron kernel with its shared-memory buffer of partial cells
//    (Sec. 6.2), generalised to batches of tetrahedra so that small tetrahedra fill
//    the warp too.  Each tetrahedron's FP64 sum of deposits is tracked so that the
//    rounding residual m_t - sum can be added to the cell of its centroid.
//  * k_build_tets: particle indices and signed volumes of every tetrahedron.
#include "geom.cuh"
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
                                            P3<T> (&v)[4], int (&base)[3])
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
        if (P.periodic) { i = wrap_idx(i, P.n[0]); j = wrap_idx(j, P.n[1]); k = wrap_idx(k, P.n[2]); }
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
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int shift = 0;
            if (P.periodic && q > 0) {
                const double d = (double)x[q][a] - (double)x[0][a];
                shift = (d >= 0.5 * P.box) ? -1 : ((d < -0.5 * P.box) ? 1 : 0);
            }
            const long long off = (long long)shift * P.g[a] - base[a];
            if constexpr (sizeof(T) == 4)
                c[a] = fmaf(x[q][a], P.scale_f[a], (float)off);
            else
                c[a] = fma((double)x[q][a], P.scale_d[a], (double)off);
        }
        v[q] = mk<T>(c[0], c[1], c[2]);
    }
}

template <class T>
__device__ __forceinline__ void explicit_tet(const DepositParams &P, int64_t t, P3<T> (&v)[4], int (&base)[3])
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
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if constexpr (sizeof(T) == 4)
                c[a] = fmaf(x[q][a], P.scale_f[a], (float)(-base[a]));
            else
                c[a] = fma((double)x[q][a], P.scale_d[a], (double)(-base[a]));
        }
        v[q] = mk<T>(c[0], c[1], c[2]);
    }
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

// Add m to cell (cx, cy, cz) (unfolded grid indices); returns false if the cell is
// outside an open grid (then the mass is dropped).
__device__ __forceinline__ bool deposit_cell(const DepositParams &P, int64_t cx, int64_t cy, int64_t cz, double m)
{
    if (P.periodic) {
        cx = fold_cell(cx, P.g[0]);
        cy = fold_cell(cy, P.g[1]);
        cz = fold_cell(cz, P.g[2]);
    } else if (cx < 0 || cy < 0 || cz < 0 || cx >= P.g[0] || cy >= P.g[1] || cz >= P.g[2]) {
        return false;
    }
    atomicAdd(P.out + (cx + P.g[0] * (cy + P.g[1] * cz)), m);
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

struct Counters {
    unsigned long long u[ST_NUM_U64];
    double mass_in, dropped;
    __device__ void zero()
    {
#pragma unroll
        for (int i = 0; i < ST_NUM_U64; ++i) u[i] = 0;
        mass_in = 0.0;
        dropped = 0.0;
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

// ---------------------------------------------------------------------------
// thread per tetrahedron
// ---------------------------------------------------------------------------
template <class T, bool STATS>
__global__ void __launch_bounds__(128) k_thread_per_tet(const DepositParams P)
{
    Counters cnt;
    if (STATS) cnt.zero();
    const int64_t n_tets = (P.src == SRC_TETS) ? P.n_units : 6 * P.n_units;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tets;
         t += (int64_t)gridDim.x * blockDim.x) {
        P3<T> v[4];
        int base[3];
        double m_t;
        if (P.src == SRC_TETS) {
            explicit_tet<T>(P, t, v, base);
            m_t = P.tet_mass[t];
        } else {
            int64_t i, j, k;
            if (!cube_of_unit(P, t / 6, i, j, k)) {
                set_error(P.ws, 3, (int)((t / 6) & 0x7fffffff));
                continue;
            }
            lattice_tet<T>(P, i, j, k, (int)(t % 6), v, base);
            m_t = P.m_tet;
        }
        TetSetup<T> ts;
        tet_setup<T>(v, ts);
        if (STATS) { cnt.u[ST_TETS]++; cnt.mass_in += m_t; }
        if (!tet_ok(base, ts)) {
            set_error(P.ws, 4, (int)(t & 0x7fffffff));
            continue;
        }
        if (ts.vol6 == 0.0) {
            int c[3];
            centroid_cell(ts.v, c);
            if (!deposit_cell(P, base[0] + c[0], base[1] + c[1], base[2] + c[2], m_t) && STATS) cnt.dropped += m_t;
            if (STATS) cnt.u[ST_DEGENERATE]++;
            continue;
        }
        const int64_t ncell = (int64_t)ts.dim[0] * ts.dim[1] * ts.dim[2];
        if (STATS) { cnt.u[ST_BBOX_CELLS] += ncell; cnt.u[ST_BIN0 + size_bin(ncell)]++; }
        if (ncell == 1) {
            if (!deposit_cell(P, base[0] + ts.lo[0], base[1] + ts.lo[1], base[2] + ts.lo[2], m_t) && STATS)
                cnt.dropped += m_t;
            if (STATS) cnt.u[ST_SINGLE_CELL]++;
            continue;
        }
        const double rho = 6.0 * m_t / ts.vol6;
        // FP32 guard: ill-conditioned tetrahedra are clipped in float64
        const bool g64 = (sizeof(T) == 4) && !(ts.kappa <= P.kappa_max);
        double dsum = 0.0;
        for (int iz = 0; iz < ts.dim[2]; ++iz)
            for (int iy = 0; iy < ts.dim[1]; ++iy)
                for (int ix = 0; ix < ts.dim[0]; ++ix) {
                    const int cx = ts.lo[0] + ix, cy = ts.lo[1] + iy, cz = ts.lo[2] + iz;
                    const int cls = classify_cell<T>(ts.n, ts.e, ts.pos, ts.neg, (T)cx, (T)cy, (T)cz);
                    double vol = 0.0;
                    if (cls == CELL_INSIDE) {
                        vol = 1.0;
                        if (STATS) cnt.u[ST_INSIDE_CELLS]++;
                    } else if (cls == CELL_PARTIAL) {
                        P3<T> p[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) p[q] = mk<T>(ts.v[q].x - (T)cx, ts.v[q].y - (T)cy, ts.v[q].z - (T)cz);
                        if constexpr (sizeof(T) == 4) {
                            if (g64) {
                                vol = overlap_volume_fp64(p);
                                if (STATS) cnt.u[ST_FP64_REDOS]++;
                            } else {
                                T err;
                                vol = (double)overlap_volume<T>(p, ts.n, ts.lx, ts.ly, err);
                            }
                        } else {
                            T err;
                            vol = (double)overlap_volume<T>(p, ts.n, ts.lx, ts.ly, err);
                        }
                        if (STATS) cnt.u[ST_PARTIAL_CLIPS]++;
                    }
                    if (vol > 0.0) {
                        const double m = rho * vol;
                        dsum += m;
                        if (!deposit_cell(P, (int64_t)base[0] + cx, (int64_t)base[1] + cy, (int64_t)base[2] + cz, m) &&
                            STATS)
                            cnt.dropped += m;
                    }
                }
        // FP32 path: the rounding residual of this tetrahedron's mass goes to its centroid cell
        if (sizeof(T) == 4 && P.fixup && m_t != dsum) {
            int c[3];
            centroid_cell(ts.v, c);
            if (!deposit_cell(P, (int64_t)base[0] + c[0], (int64_t)base[1] + c[1], (int64_t)base[2] + c[2], m_t - dsum) &&
                STATS)
                cnt.dropped += m_t - dsum;
        }
    }
    if (STATS) cnt.flush(P.ws);
}

// ---------------------------------------------------------------------------
// warp-cooperative FP32 path
// ---------------------------------------------------------------------------
struct WarpSmem {
    float v[12][32];      // base-frame vertices (x0 y0 z0 x1 ...), positively oriented
    float n[12][32];      // outward face normals
    float e[4][32];
    float pos[4][32];
    float neg[4][32];
    float lx[32], ly[32];  // reference-plane slopes
    int lo[3][32];
    int dim[3][32];
    int base[3][32];
    double rho[32];
    double dsum[32];      // FP64 sum of what each tetrahedron deposited
    int start[32];        // exclusive prefix of the pair counts
    int guard[32];        // 1: clip this tetrahedron in float64
    unsigned long long q[64];  // queued partial pairs: t | ix << 5 | iy << 24 | iz << 43
};

constexpr int kQBits = 19;  // per-axis cell offset bits in a queue entry
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

// Adds each lane's v into S->dsum[key] when the lanes holding the same key are
// contiguous (key < 0: no contribution): a segmented reduction to the first lane of
// each run, which then updates the shared sum without atomics.
__device__ __forceinline__ void segmented_add(WarpSmem *S, int lane, int key, double v)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_down_sync(kFull, v, o);
        const int k2 = __shfl_down_sync(kFull, key, o);
        if (lane + o < 32 && k2 == key) v += y;
    }
    const int kp = __shfl_up_sync(kFull, key, 1);
    if (key >= 0 && (lane == 0 || kp != key)) S->dsum[key] += v;
}

// The float64 redo of a guarded clip, kept out of line so that the FP32 hot loop
// stays small; vertices passed by value (cell frame, positively oriented).
__device__ __noinline__ double redo_fp64(float x0, float y0, float z0, float x1, float y1, float z1, float x2,
                                         float y2, float z2, float x3, float y3, float z3)
{
    P3<float> p[4];
    p[0] = mk<float>(x0, y0, z0);
    p[1] = mk<float>(x1, y1, z1);
    p[2] = mk<float>(x2, y2, z2);
    p[3] = mk<float>(x3, y3, z3);
    return overlap_volume_fp64(p);
}

template <bool STATS>
__device__ __forceinline__ void clip_round(const DepositParams &P, WarpSmem *S, int count, int lane, Counters &cnt)
{
    int key = -1;
    double m = 0.0;
    if (lane < count) {
        const unsigned long long ent = S->q[lane];
        const int t = (int)(ent & 31u);
        const int cx = S->lo[0][t] + (int)((ent >> 5) & kQMask);
        const int cy = S->lo[1][t] + (int)((ent >> (5 + kQBits)) & kQMask);
        const int cz = S->lo[2][t] + (int)((ent >> (5 + 2 * kQBits)) & kQMask);
        const float fx = (float)cx, fy = (float)cy, fz = (float)cz;
        P3<float> p[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            p[q] = mk<float>(S->v[3 * q][t] - fx, S->v[3 * q + 1][t] - fy, S->v[3 * q + 2][t] - fz);
        double vol;
        if (!S->guard[t]) {
            P3<float> n[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) n[f] = mk<float>(S->n[3 * f][t], S->n[3 * f + 1][t], S->n[3 * f + 2][t]);
            float err;
            vol = (double)overlap_volume<float>(p, n, S->lx[t], S->ly[t], err);
        } else {
            vol = redo_fp64(p[0].x, p[0].y, p[0].z, p[1].x, p[1].y, p[1].z, p[2].x, p[2].y, p[2].z, p[3].x, p[3].y,
                            p[3].z);
            if (STATS) cnt.u[ST_FP64_REDOS]++;
        }
        if (STATS) cnt.u[ST_PARTIAL_CLIPS]++;
        key = t;
        if (vol > 0.0) {
            m = S->rho[t] * vol;
            if (!deposit_cell(P, (int64_t)S->base[0][t] + cx, (int64_t)S->base[1][t] + cy,
                              (int64_t)S->base[2][t] + cz, m) && STATS)
                cnt.dropped += m;
        }
    }
    if (P.fixup) segmented_add(S, lane, key, m);
    __syncwarp();
}

template <bool STATS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_warp_coop(const DepositParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem *S = reinterpret_cast<WarpSmem *>(smem_raw) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    Counters cnt;
    if (STATS) cnt.zero();
    const int nsub = (P.src == SRC_TETS) ? 1 : 6;

    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(&P.ws->work_counter, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if ((int64_t)item >= P.n_items) break;

        // the 32 units (cubes or tetrahedra) of this item
        int64_t unit = -1;
        int64_t ci = 0, cj = 0, ck = 0;
        if (P.src == SRC_LATTICE) {
            // rows of 32 cubes along x
            const int64_t segs = (P.nc[0] + 31) / 32;
            const int64_t row = (int64_t)item / segs, seg = (int64_t)item % segs;
            const int64_t i = seg * 32 + lane;
            if (i < P.nc[0]) {
                ci = i;
                cj = row % P.nc[1];
                ck = row / P.nc[1];
                unit = 1;
            }
        } else {
            const int64_t u = (int64_t)item * 32 + lane;
            if (u < P.n_units) {
                unit = u;
                if (P.src == SRC_CUBE_LIST && !cube_of_unit(P, u, ci, cj, ck)) {
                    set_error(P.ws, 3, (int)(u & 0x7fffffff));
                    unit = -1;
                }
            }
        }

        for (int s = 0; s < nsub; ++s) {
            // ---- 1. one tetrahedron per lane
            int npairs = 0;
            double m_t = 0.0;
            bool coop = false;
            if (unit >= 0) {
                P3<float> v[4];
                int base[3];
                if (P.src == SRC_TETS) {
                    explicit_tet<float>(P, unit, v, base);
                    m_t = P.tet_mass[unit];
                } else {
                    lattice_tet<float>(P, ci, cj, ck, s, v, base);
                    m_t = P.m_tet;
                }
                TetSetup<float> ts;
                tet_setup<float>(v, ts);
                if (STATS) { cnt.u[ST_TETS]++; cnt.mass_in += m_t; }
                const int64_t ncell = (int64_t)ts.dim[0] * ts.dim[1] * ts.dim[2];
                if (!tet_ok(base, ts)) {
                    set_error(P.ws, 4, lane);
                } else if (ts.vol6 == 0.0) {
                    int c[3];
                    centroid_cell(ts.v, c);
                    if (!deposit_cell(P, (int64_t)base[0] + c[0], (int64_t)base[1] + c[1], (int64_t)base[2] + c[2], m_t) &&
                        STATS)
                        cnt.dropped += m_t;
                    if (STATS) cnt.u[ST_DEGENERATE]++;
                } else if (ncell == 1) {
                    if (!deposit_cell(P, (int64_t)base[0] + ts.lo[0], (int64_t)base[1] + ts.lo[1],
                                      (int64_t)base[2] + ts.lo[2], m_t) && STATS)
                        cnt.dropped += m_t;
                    if (STATS) { cnt.u[ST_SINGLE_CELL]++; cnt.u[ST_BBOX_CELLS]++; cnt.u[ST_BIN0]++; }
                } else if (ncell > (int64_t)(1 << 25)) {
                    set_error(P.ws, 2, lane);  // 32 x 2^25 pairs still fit the int32 scan
                } else {
                    coop = true;
                    npairs = (int)ncell;
                    if (STATS) { cnt.u[ST_BBOX_CELLS] += ncell; cnt.u[ST_BIN0 + size_bin(ncell)]++; }
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
                    S->rho[lane] = 6.0 * m_t / ts.vol6;
                    S->lx[lane] = ts.lx;
                    S->ly[lane] = ts.ly;
                    S->guard[lane] = (ts.kappa <= P.kappa_max) ? 0 : 1;
                }
            }
            // ---- 2. pair enumeration
            int incl = npairs;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(kFull, incl, 31);
            S->start[lane] = incl - npairs;
            S->dsum[lane] = 0.0;
            __syncwarp();
            int qn = 0;
            for (int b0 = 0; b0 < total; b0 += 32) {
                const int idx = b0 + lane;
                bool partial = false;
                unsigned long long ent = 0;
                int ikey = -1;
                double im = 0.0;
                if (idx < total) {
                    int t = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1)
                        if (S->start[t + step] <= idx && t + step < 32) t += step;
                    const int local = idx - S->start[t];
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
                        const double m = S->rho[t];
                        if (!deposit_cell(P, (int64_t)S->base[0][t] + (int64_t)cx, (int64_t)S->base[1][t] + (int64_t)cy,
                                          (int64_t)S->base[2][t] + (int64_t)cz, m) && STATS)
                            cnt.dropped += m;
                        ikey = t;
                        im = m;
                        if (STATS) cnt.u[ST_INSIDE_CELLS]++;
                    } else if (cls == CELL_PARTIAL) {
                        partial = true;
                        ent = q_pack(t, ix, iy, iz);
                    }
                }
                if (P.fixup && __any_sync(kFull, ikey >= 0)) segmented_add(S, lane, ikey, im);
                const unsigned bal = __ballot_sync(kFull, partial);
                if (partial) S->q[qn + __popc(bal & lt_mask)] = ent;
                qn += __popc(bal);
                __syncwarp();
                if (qn >= 32) {
                    clip_round<STATS>(P, S, 32, lane, cnt);
                    if (lane < qn - 32) S->q[lane] = S->q[32 + lane];
                    qn -= 32;
                    __syncwarp();
                }
            }
            if (qn > 0) clip_round<STATS>(P, S, qn, lane, cnt);
            // ---- 3. mass residual of each tetrahedron to its centroid cell
            if (coop && P.fixup) {
                const double resid = m_t - S->dsum[lane];
                if (resid != 0.0) {
                    P3<float> vv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) vv[q] = mk<float>(S->v[3 * q][lane], S->v[3 * q + 1][lane], S->v[3 * q + 2][lane]);
                    int c[3];
                    centroid_cell(vv, c);
                    if (!deposit_cell(P, (int64_t)S->base[0][lane] + c[0], (int64_t)S->base[1][lane] + c[1],
                                      (int64_t)S->base[2][lane] + c[2], resid) && STATS)
                        cnt.dropped += resid;
                }
            }
            __syncwarp();
        }
    }
    if (STATS) cnt.flush(P.ws);
}

// ---------------------------------------------------------------------------
// tessellation builder
// ---------------------------------------------------------------------------
__global__ void k_build_tets(const float *__restrict__ pos, long long n0, long long n1, long long n2, long long nc0,
                             long long nc1, int periodic, double box, int32_t *__restrict__ vidx,
                             float *__restrict__ vol, long long n_tets)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_tets;
         t += (long long)gridDim.x * blockDim.x) {
        const long long c = t / 6;
        const int s = (int)(t % 6);
        const long long ci = c % nc0, cj = (c / nc0) % nc1, ck = c / (nc0 * nc1);
        int o1[3], o2[3];
        kuhn_offsets(s, o1, o2);
        long long id[4];
        double x[4][3];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            long long i = ci, j = cj, k = ck;
            if (q == 1) { i += o1[0]; j += o1[1]; k += o1[2]; }
            if (q == 2) { i += o2[0]; j += o2[1]; k += o2[2]; }
            if (q == 3) { i += 1; j += 1; k += 1; }
            if (periodic) { i = wrap_idx(i, n0); j = wrap_idx(j, n1); k = wrap_idx(k, n2); }
            id[q] = i + n0 * (j + n1 * k);
#pragma unroll
            for (int a = 0; a < 3; ++a) x[q][a] = (double)__ldg(pos + 3 * id[q] + a);
        }
        if (periodic) {
#pragma unroll
            for (int q = 1; q < 4; ++q)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double d = x[q][a] - x[0][a];
                    x[q][a] -= (d >= 0.5 * box) ? box : ((d < -0.5 * box) ? -box : 0.0);
                }
        }
        if (vidx) {
#pragma unroll
            for (int q = 0; q < 4; ++q) vidx[4 * t + q] = (int32_t)id[q];
        }
        if (vol) {
            const double ax = x[1][0] - x[0][0], ay = x[1][1] - x[0][1], az = x[1][2] - x[0][2];
            const double bx = x[2][0] - x[0][0], by = x[2][1] - x[0][1], bz = x[2][2] - x[0][2];
            const double cx = x[3][0] - x[0][0], cy = x[3][1] - x[0][1], cz = x[3][2] - x[0][2];
            vol[t] = (float)((ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx)) / 6.0);
        }
    }
}

int persistent_blocks(const void *kernel, int threads, size_t smem)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

}  // namespace

cudaError_t launch_thread_per_tet(const DepositParams &p, bool fp64, bool stats, cudaStream_t st)
{
    const int threads = 128;
    const int64_t n_tets = (p.src == SRC_TETS) ? p.n_units : 6 * p.n_units;
    const void *k = fp64 ? (stats ? (const void *)k_thread_per_tet<double, true> : (const void *)k_thread_per_tet<double, false>)
                         : (stats ? (const void *)k_thread_per_tet<float, true> : (const void *)k_thread_per_tet<float, false>);
    int64_t blocks = (n_tets + threads - 1) / threads;
    const int64_t cap = (int64_t)persistent_blocks(k, threads, 0) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (fp64) {
        if (stats) k_thread_per_tet<double, true><<<(unsigned)blocks, threads, 0, st>>>(p);
        else k_thread_per_tet<double, false><<<(unsigned)blocks, threads, 0, st>>>(p);
    } else {
        if (stats) k_thread_per_tet<float, true><<<(unsigned)blocks, threads, 0, st>>>(p);
        else k_thread_per_tet<float, false><<<(unsigned)blocks, threads, 0, st>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_warp_coop(const DepositParams &p, bool stats, int blocks_per_sm, cudaStream_t st)
{
    const int threads = 256;
    const size_t smem = sizeof(WarpSmem) * (threads / 32);
    const int minb = (blocks_per_sm >= 2) ? 2 : 1;
    const void *k = stats ? (minb == 2 ? (const void *)k_warp_coop<true, 2> : (const void *)k_warp_coop<true, 1>)
                          : (minb == 2 ? (const void *)k_warp_coop<false, 2> : (const void *)k_warp_coop<false, 1>);
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int blocks = persistent_blocks(k, threads, smem);
    const int64_t need = (p.n_items + 7) / 8;
    if (need < blocks) blocks = (int)(need < 1 ? 1 : need);
    void *args[] = {const_cast<DepositParams *>(&p)};
    return cudaLaunchKernel(k, dim3(blocks), dim3(threads), args, smem, st);
}

cudaError_t launch_build_tets(const float *pos, const int64_t n[3], const int64_t nc[3], int periodic, double box,
                              int32_t *vidx, float *vol, int64_t n_tets, cudaStream_t st)
{
    const int threads = 256;
    int64_t blocks = (n_tets + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    k_build_tets<<<(unsigned)blocks, threads, 0, st>>>(pos, n[0], n[1], n[2], nc[0], nc[1], periodic, box, vidx, vol,
                                                        n_tets);
    return cudaGetLastError();
}

}  // namespace pse
