// coop.cuh -- the warp-cooperative deposit kernel k_warp_coop and its launcher, templated
// on the accumulation mode: deposit.cu instantiates the FP64-reduction kernels and
// deposit_comp.cu the compensated-FP32 ones, so the two build in parallel.
//
// One warp takes a batch of 32 tetrahedra (32 Lagrangian cubes x one Kuhn permutation),
// enumerates all their (tetrahedron, cell) pairs 32 at a time, classifies them in
// lock-step, deposits "cell inside tetrahedron" pairs at once and compacts the partial
// pairs into a per-warp queue; whenever 32 are queued every lane clips one (FP32, in
// registers).  Tetrahedra whose conditioning estimate exceeds the guard are clipped in
// FP64.  This is the role of the paper's warp-per-tetrahedron kernel with its
// shared-memory buffer of partial cells (Sec. 6.2), generalised to batches of tetrahedra
// so that small tetrahedra fill the warp too.
#pragma once

#include "common.cuh"

namespace pse {
namespace {

// ---------------------------------------------------------------------------
// warp-cooperative FP32 path
// ---------------------------------------------------------------------------
// Split work item `item` of the binned schedule: chunk [first, first + len) of the
// bounding-box cells of one queued tetrahedron, set up by lane 0 as record 0.  Returns
// the lane's pair count (len on lane 0, else 0).
template <bool STATS, int PASS>
__device__ __forceinline__ int chunk_setup(const DepositParams &P, WarpSmem *S, int lane, int64_t item, int64_t q,
                                           Counters &cnt)
{
    // queue entry e: the last with chunk_start[e] <= item
    int64_t lo = 0, hi = q - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (P.chunk_start[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    // q_cells holds the tetrahedron's pair count (column runs, or cells if guarded)
    const int64_t first = (item - P.chunk_start[lo]) * (int64_t)P.chunk_cells;
    const int64_t npair = P.q_cells[lo];
    const int len = (int)min((int64_t)P.chunk_cells, npair - first);
    if (lane != 0 || len <= 0) return 0;
    const int64_t id = P.q_tet[lo];
    P3<float> v[4], res[4];
    int base[3];
    double m_t;
    if (P.src == SRC_TETS) {
        explicit_tet<float>(P, id, v, base, res);
        m_t = P.tet_mass[id];
    } else {
        int64_t ci, cj, ck;
        if (!cube_of_unit(P, id / 6, ci, cj, ck)) return 0;
        lattice_tet<float>(P, ci, cj, ck, (int)(id % 6), v, base, res);
        m_t = P.m_tet;
    }
    TetSetup<float> ts;
    if (tet_setup<float>(v, ts)) swap12(res);
    if (!dims_fit_queue(ts.dim)) {
        set_error(P.ws, 2, (int)(id & 0x7fffffff));
        return 0;
    }
    // each pass takes the pieces of its own side of the guard
    const bool guard = !(ts.kappa <= P.kappa_max);
    if (guard != (PASS == kPassGuard)) return 0;
    store_record(S, 0, ts, res, base, m_t, P.kappa_max, (int)first);
    return len;
}

constexpr int kCoopThreads = 128;

// PASS kPassFp32 visits every tetrahedron: it counts them, deposits the degenerate and
// single-cell ones, and clips those below the guard by column runs.  PASS kPassGuard visits
// them again and clips only the guarded multi-cell ones, by column runs in FP64.
template <bool STATS, int MINB, bool BINNED, Acc A, int PASS>
__global__ void __launch_bounds__(kCoopThreads, MINB) k_warp_coop(const DepositParams P)
{
    constexpr bool FIRST = PASS == kPassFp32;
    WarpSmem *S = warp_smem(!FIRST);
    bind_residuals(P, S, !FIRST);
    const int lane = threadIdx.x & 31;
    Counters cnt;
    if (STATS) cnt.zero();
    cnt.zero_mass();
    const int nsub = (P.src == SRC_TETS) ? 1 : 6;
    // binned schedule: items [0, n_chunks) are pieces of split tetrahedra (largest work
    // first), the rest are the rows; tetrahedra the bin pass queued are skipped there
    int64_t n_chunks = 0, q = 0;
    bool split = false;
    if (BINNED) {
        split = P.ws->queue_overflow == 0;
        n_chunks = split ? (int64_t)P.ws->n_chunk_items : 0;
        q = split ? min((int64_t)P.ws->queue_count, P.q_cap) : 0;
    }
    // the guarded pass of the warp schedule: the tetrahedra the FP32 pass listed, 32 per item,
    // when it listed all of them
    const int64_t listed = (!FIRST && !BINNED) ? listed_guarded(P) : -1;
    const bool LIST = listed >= 0;
    const int64_t n_items = LIST ? (listed + 31) / 32 : P.n_items;

    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(FIRST ? &P.ws->work_counter : &P.ws->work_counter2, 1ull);
        item = __shfl_sync(kFull, item, 0);
        const bool is_chunk = BINNED && (int64_t)item < n_chunks;
        if (!is_chunk) {
            item -= (unsigned long long)n_chunks;
            if ((int64_t)item >= n_items) break;
        }

        // the 32 units (cubes or tetrahedra) of this item
        int64_t unit = -1;
        int64_t ci = 0, cj = 0, ck = 0;
        int s_listed = 0;
        if (is_chunk) {
            // nothing: chunk_setup below
        } else if (LIST) {
            // one listed tetrahedron per lane: its id decodes like the ids below
            const int64_t k = (int64_t)item * 32 + lane;
            if (k < listed) {
                const int64_t id = P.guard_list[k];
                if (P.src == SRC_TETS) {
                    unit = id;
                } else {
                    const int64_t u = id / 6;
                    s_listed = (int)(id % 6);
                    if (P.src == SRC_LATTICE) {
                        ci = u % P.nc[0];
                        cj = (u / P.nc[0]) % P.nc[1];
                        ck = u / (P.nc[0] * P.nc[1]);
                        unit = 1;
                    } else if (cube_of_unit(P, u, ci, cj, ck)) {
                        unit = u;
                    }
                }
            }
        } else if (P.src == SRC_LATTICE) {
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

        const int nsub_item = (is_chunk || LIST) ? 1 : nsub;
        for (int si = 0; si < nsub_item; ++si) {
            const int s = LIST ? s_listed : si;
            // ---- 1. one tetrahedron per lane (or the queued tetrahedron's chunk on lane 0)
            int npairs = 0;
            double m_t = 0.0;
            int64_t tid = 0;
            bool to_list = false;
            if (is_chunk) {
                npairs = chunk_setup<STATS, PASS>(P, S, lane, (int64_t)item, q, cnt);
                __syncwarp();
            } else if (unit >= 0) {
                P3<float> v[4];
                int base[3];
                // tetrahedron id as the bin pass numbers it (and the guarded-tetrahedron list)
                tid = (P.src == SRC_TETS) ? unit
                                          : 6 * ((P.src == SRC_LATTICE) ? ci + P.nc[0] * (cj + P.nc[1] * ck) : unit) + s;
                if (P.src == SRC_TETS) {
                    explicit_tet<float>(P, unit, v, base);
                    m_t = P.tet_mass[unit];
                } else {
                    lattice_tet<float>(P, ci, cj, ck, s, v, base);
                    m_t = P.m_tet;
                }
                TetSetup<float> ts;
                const bool swapped = tet_setup<float>(v, ts);
                if (STATS && FIRST) {
                    cnt.u[ST_TETS]++;
                    cnt.mass_in += m_t;
                    cnt.u[ST_INVERTED] += (swapped != (P.src != SRC_TETS && kuhn_negative(s))) ? 1 : 0;
                }
                const int64_t ncell = (int64_t)ts.dim[0] * ts.dim[1] * ts.dim[2];
                const bool guard = !(ts.kappa <= P.kappa_max);
                if (!tet_ok(base, ts)) {
                    set_error(P.ws, 4, lane);
                } else if (!FIRST && (ts.vol6 == 0.0 || ncell == 1 || !guard)) {
                    // the guarded pass: nothing to do for this tetrahedron
                } else if (ts.vol6 == 0.0) {
                    int c[3];
                    centroid_cell(ts.v, c);
                    if (!deposit_cell<A>(P, (int64_t)base[0] + c[0], (int64_t)base[1] + c[1], (int64_t)base[2] + c[2], m_t) &&
                        STATS)
                        cnt.dropped += m_t;
                    cnt.add_tgt(P, m_t);
                    cnt.add_dep(m_t);
                    if (STATS) { cnt.u[ST_DEGENERATE]++; cnt.u[ST_OVERLAPPED]++; }
                } else if (ncell == 1) {
                    if (!deposit_cell<A>(P, (int64_t)base[0] + ts.lo[0], (int64_t)base[1] + ts.lo[1],
                                      (int64_t)base[2] + ts.lo[2], m_t) && STATS)
                        cnt.dropped += m_t;
                    cnt.add_tgt(P, m_t);
                    cnt.add_dep(m_t);
                    if (STATS) { cnt.u[ST_SINGLE_CELL]++; cnt.u[ST_BBOX_CELLS]++; cnt.u[ST_BIN0]++; cnt.u[ST_OVERLAPPED]++; }
                } else if (BINNED && split &&
                           (P.model ? ((P.qbits[tid >> 5] >> (tid & 31)) & 1u) != 0
                                    : (ncell > P.split_cells && ncell <= (int64_t)INT32_MAX))) {
                    // queued by the bin pass: its cells are done by the split work items
                    if (FIRST) {
                        cnt.add_tgt(P, m_t);
                        if (STATS) { cnt.u[ST_BBOX_CELLS] += ncell; cnt.u[ST_BIN0 + size_bin(ncell)]++; }
                    }
                } else if (ncell > (int64_t)(1 << 25) || !dims_fit_queue(ts.dim)) {
                    set_error(P.ws, 2, lane);  // 32 x 2^25 pairs still fit the int32 scan
                } else if (FIRST) {
                    cnt.add_tgt(P, m_t);
                    if (STATS) { cnt.u[ST_BBOX_CELLS] += ncell; cnt.u[ST_BIN0 + size_bin(ncell)]++; }
                    if (!guard) {  // guarded ones are left to the second pass
                        npairs = (int)run_count(ts.dim, ts.axis);
                        P3<float> res[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) res[q] = mk<float>(0.f, 0.f, 0.f);
                        store_record(S, lane, ts, res, base, m_t, P.kappa_max, 0);
                    } else {
                        to_list = !BINNED;
                    }
                } else {
                    // guarded: column runs, clipped in float64 from the exact vertices
                    // (the float32 vertices plus their rounding residuals)
                    npairs = (int)run_count(ts.dim, ts.axis);
                    P3<float> res[4], v2[4];
                    int b2[3];
                    if (P.src == SRC_TETS) explicit_tet<float>(P, unit, v2, b2, res);
                    else lattice_tet<float>(P, ci, cj, ck, s, v2, b2, res);
                    if (swapped) swap12(res);
                    store_record(S, lane, ts, res, base, m_t, P.kappa_max, 0);
                }
            }
            if (FIRST && !BINNED) list_guarded(P, to_list, tid, lane);
            // ---- 2. pair enumeration and clips
            coop_pairs<STATS, false, A, PASS>(P, S, lane, npairs, cnt);
            __syncwarp();
        }
    }
    if (STATS) cnt.flush(P.ws);
    if (P.fixup || STATS) cnt.flush_mass(P, P.ws);
}

template <bool BINNED, Acc A, int PASS>
cudaError_t launch_coop_pass(const DepositParams &p, bool stats, int blocks_per_sm, int64_t max_items,
                             cudaStream_t st)
{
    // blocks_per_sm resident blocks of 128 threads: 2 (255 registers per thread, 8 warps per
    // SM), 3 (170 registers, 12 warps) or 4 (128 registers, 16 warps).  The counting
    // variant (stats) is built for 2 only.
    const int threads = kCoopThreads;
    constexpr bool GUARD = PASS == kPassGuard;
    const size_t smem = warp_smem_bytes(threads / 32, GUARD);
    // the guarded pass runs 2 blocks per SM (190 registers): its FP64 pipe is already the
    // bottleneck there (84% busy), so more residency would not help
    const int minb = (stats || GUARD) ? 2 : (blocks_per_sm >= 4 ? 4 : (blocks_per_sm == 3 ? 3 : 2));
    const void *k;
    if constexpr (GUARD) {
        k = stats ? (const void *)k_warp_coop<true, 2, BINNED, A, PASS> : (const void *)k_warp_coop<false, 2, BINNED, A, PASS>;
    } else {
        k = stats ? (const void *)k_warp_coop<true, 2, BINNED, A, PASS>
            : minb == 4 ? (const void *)k_warp_coop<false, 4, BINNED, A, PASS>
            : minb == 3 ? (const void *)k_warp_coop<false, 3, BINNED, A, PASS>
                        : (const void *)k_warp_coop<false, 2, BINNED, A, PASS>;
    }
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int blocks = persistent_blocks(k, threads, smem);
    if (blocks > kMaxWarpBlocks) blocks = kMaxWarpBlocks;
    const int64_t need = (max_items + threads / 32 - 1) / (threads / 32);
    if (need < blocks) blocks = (int)(need < 1 ? 1 : need);
    void *args[] = {const_cast<DepositParams *>(&p)};
    return cudaLaunchKernel(k, dim3(blocks), dim3(threads), args, smem, st);
}

// The FP32 pass, then the guarded pass over the same tetrahedra, on one stream.
template <bool BINNED, Acc A>
cudaError_t launch_coop(const DepositParams &p, bool stats, int blocks_per_sm, int64_t max_items, cudaStream_t st)
{
    cudaError_t e = launch_coop_pass<BINNED, A, kPassFp32>(p, stats, blocks_per_sm, max_items, st);
    if (e != cudaSuccess) return e;
    return launch_coop_pass<BINNED, A, kPassGuard>(p, stats, blocks_per_sm, max_items, st);
}

}  // namespace
}  // namespace pse
