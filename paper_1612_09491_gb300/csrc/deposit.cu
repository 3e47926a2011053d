// deposit.cu -- tetrahedron deposit kernels for sm_103a.
//
//  * k_thread_per_tet<T>: one thread per tetrahedron walks its bounding-box cells,
//    classifies each, clips the partial ones and adds m_t V_ov/|V_t| with a global
//    float64 atomic.  With T = double this is the plain FP64 baseline.
//  * k_warp_coop (coop.cuh): the warp-cooperative FP32 kernel; this file instantiates
//    its FP64-reduction variants, deposit_comp.cu the compensated-FP32 ones.
//  * k_warp_per_tet: the paper's warp-per-tetrahedron design (Sec. 6.2), a baseline.
//  * k_bin_pass, k_chunk_scan: the binned schedule's queue of large tetrahedra.
//  * k_finish: pair conversion and mass renormalisation at the end of an FP32 deposit.
//  * k_build_tets: particle indices and signed volumes of every tetrahedron.
#include "coop.cuh"
#include "costmodel.cuh"

namespace pse {

namespace {

// ---------------------------------------------------------------------------
// thread per tetrahedron
// ---------------------------------------------------------------------------
template <class T, bool STATS>
__global__ void __launch_bounds__(128) k_thread_per_tet(const DepositParams P)
{
    Counters cnt;
    if (STATS) cnt.zero();
    cnt.zero_mass();
    const int64_t n_tets = (P.src == SRC_TETS) ? P.n_units : 6 * P.n_units;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tets;
         t += (int64_t)gridDim.x * blockDim.x) {
        cnt.fold_dep();  // the previous tetrahedron's deposits
        P3<T> v[4];
        P3<float> res[4];
        int base[3];
        double m_t;
        if (P.src == SRC_TETS) {
            explicit_tet<T>(P, t, v, base, res);
            m_t = P.tet_mass[t];
        } else {
            int64_t i, j, k;
            if (!cube_of_unit(P, t / 6, i, j, k)) {
                set_error(P.ws, 3, (int)((t / 6) & 0x7fffffff));
                continue;
            }
            lattice_tet<T>(P, i, j, k, (int)(t % 6), v, base, res);
            m_t = P.m_tet;
        }
        TetSetup<T> ts;
        const bool negative = tet_setup<T>(v, ts);
        if (negative) swap12(res);
        if (STATS) {
            cnt.u[ST_TETS]++;
            cnt.mass_in += m_t;
            cnt.u[ST_INVERTED] += (negative != (P.src != SRC_TETS && kuhn_negative((int)(t % 6)))) ? 1 : 0;
        }
        if (!tet_ok(base, ts)) {
            set_error(P.ws, 4, (int)(t & 0x7fffffff));
            continue;
        }
        cnt.add_tgt(P, m_t);
        if (ts.vol6 == 0.0) {
            int c[3];
            centroid_cell(ts.v, c);
            if (!deposit_cell(P, base[0] + c[0], base[1] + c[1], base[2] + c[2], m_t) && STATS) cnt.dropped += m_t;
            cnt.add_dep(m_t);
            if (STATS) { cnt.u[ST_DEGENERATE]++; cnt.u[ST_OVERLAPPED]++; }
            continue;
        }
        const int64_t ncell = (int64_t)ts.dim[0] * ts.dim[1] * ts.dim[2];
        if (STATS) { cnt.u[ST_BBOX_CELLS] += ncell; cnt.u[ST_BIN0 + size_bin(ncell)]++; }
        if (ncell == 1) {
            if (!deposit_cell(P, base[0] + ts.lo[0], base[1] + ts.lo[1], base[2] + ts.lo[2], m_t) && STATS)
                cnt.dropped += m_t;
            cnt.add_dep(m_t);
            if (STATS) { cnt.u[ST_SINGLE_CELL]++; cnt.u[ST_OVERLAPPED]++; }
            continue;
        }
        // FP32 guard: ill-conditioned tetrahedra are clipped in float64 from their exact vertices
        const bool g64 = (sizeof(T) == 4) && !(ts.kappa <= P.kappa_max);
        double rho = 6.0 * m_t / ts.vol6;
        if constexpr (sizeof(T) == 4) {
            if (g64) rho = 6.0 * m_t / exact_vol6(ts.v, res, ts.vol6);
        }
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
                    if (vol > 0.0) {
                        if (STATS) cnt.u[ST_OVERLAPPED]++;
                        const double m = rho * vol;
                        cnt.add_dep(m);
                        if (!deposit_cell(P, (int64_t)base[0] + cx, (int64_t)base[1] + cy, (int64_t)base[2] + cz, m) &&
                            STATS)
                            cnt.dropped += m;
                    }
                }
    }
    if (STATS) cnt.flush(P.ws);
    if (P.fixup || STATS) cnt.flush_mass(P, P.ws);
}

// ---------------------------------------------------------------------------
// the paper's design (Sec. 6.2), kept as a baseline: one warp per tetrahedron; its
// bounding-box cells are classified 32 at a time and the partial ones buffered and
// clipped 32 at a time (the same pair machinery and clip, with one record per warp)
// ---------------------------------------------------------------------------
template <bool STATS>
__global__ void __launch_bounds__(kCoopThreads, 2) k_warp_per_tet(const DepositParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem *S = reinterpret_cast<WarpSmem *>(smem_raw) + (threadIdx.x >> 5);
    bind_residuals(P, S);
    const int lane = threadIdx.x & 31;
    Counters cnt;
    if (STATS) cnt.zero();
    cnt.zero_mass();
    const int64_t n_tets = (P.src == SRC_TETS) ? P.n_units : 6 * P.n_units;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&P.ws->work_counter, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if ((int64_t)t >= n_tets) break;
        int npairs = 0;
        if (lane == 0) {
            P3<float> v[4], res[4];
            int base[3];
            double m_t;
            bool ok = true;
            if (P.src == SRC_TETS) {
                explicit_tet<float>(P, (int64_t)t, v, base, res);
                m_t = P.tet_mass[t];
            } else {
                int64_t ci, cj, ck;
                ok = cube_of_unit(P, (int64_t)t / 6, ci, cj, ck);
                if (!ok) set_error(P.ws, 3, (int)(((int64_t)t / 6) & 0x7fffffff));
                if (ok) lattice_tet<float>(P, ci, cj, ck, (int)(t % 6), v, base, res);
                m_t = P.m_tet;
            }
            if (ok) {
                TetSetup<float> ts;
                const bool negative = tet_setup<float>(v, ts);
                if (negative) swap12(res);
                if (STATS) {
                    cnt.u[ST_TETS]++;
                    cnt.mass_in += m_t;
                    cnt.u[ST_INVERTED] += (negative != (P.src != SRC_TETS && kuhn_negative((int)(t % 6)))) ? 1 : 0;
                }
                const int64_t ncell = (int64_t)ts.dim[0] * ts.dim[1] * ts.dim[2];
                if (!tet_ok(base, ts)) {
                    set_error(P.ws, 4, (int)(t & 0x7fffffff));
                } else if (ts.vol6 == 0.0 || ncell == 1) {
                    int c[3];
                    if (ts.vol6 == 0.0) centroid_cell(ts.v, c);
                    else { c[0] = ts.lo[0]; c[1] = ts.lo[1]; c[2] = ts.lo[2]; }
                    if (!deposit_cell(P, (int64_t)base[0] + c[0], (int64_t)base[1] + c[1], (int64_t)base[2] + c[2], m_t) &&
                        STATS)
                        cnt.dropped += m_t;
                    cnt.add_tgt(P, m_t);
                    cnt.add_dep(m_t);
                    if (STATS) {
                        cnt.u[ts.vol6 == 0.0 ? ST_DEGENERATE : ST_SINGLE_CELL]++;
                        cnt.u[ST_OVERLAPPED]++;
                        if (ts.vol6 != 0.0) { cnt.u[ST_BBOX_CELLS]++; cnt.u[ST_BIN0]++; }
                    }
                } else if (ncell > (int64_t)(1 << 25) || !dims_fit_queue(ts.dim)) {
                    set_error(P.ws, 2, (int)(t & 0x7fffffff));
                } else {
                    npairs = (int)ncell;
                    cnt.add_tgt(P, m_t);
                    if (STATS) { cnt.u[ST_BBOX_CELLS] += ncell; cnt.u[ST_BIN0 + size_bin(ncell)]++; }
                    store_record(S, 0, ts, res, base, m_t, P.kappa_max, 0);
                }
            }
        }
        __syncwarp();
        coop_pairs<STATS, false, Acc::RUNTIME, kPassAll>(P, S, lane, npairs, cnt);
        __syncwarp();
    }
    if (STATS) cnt.flush(P.ws);
    if (P.fixup || STATS) cnt.flush_mass(P, P.ws);
}

// ---------------------------------------------------------------------------
// binned schedule: the bin pass queues every tetrahedron whose bounding box has more
// than split_cells cells (warp-aggregated appends); the scan turns their cell counts
// into work items of chunk_cells cells.
// ---------------------------------------------------------------------------
// Without a cost model a tetrahedron is queued when its bounding box has more than
// split_cells cells (the row path recomputes the same test).  With one, the bin pass
// predicts each tetrahedron's partial clips (warp MLP on the tensor cores), queues it
// when the prediction exceeds split_cells, and marks it in the qbits bitmap that the row
// path reads.
template <bool MODEL>
__global__ void __launch_bounds__(128) k_bin_pass(const DepositParams P)
{
    __shared__ MlpSmem msm[MODEL ? 4 : 1];
    const int lane = threadIdx.x & 31;
    const int64_t n_tets = (P.src == SRC_TETS) ? P.n_units : 6 * P.n_units;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps iterate together so that the ballot and the warp MLP see every lane
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 < n_tets; t0 += stride) {
        const int64_t t = t0 + lane;
        bool cand = false;
        int64_t ncell = 0, npair = 0;
        float f[kNFeat];
        if (MODEL) {
#pragma unroll
            for (int q = 0; q < kNFeat; ++q) f[q] = 0.f;
        }
        if (t < n_tets) {
            P3<float> v[4];
            int base[3];
            bool ok = true;
            if (P.src == SRC_TETS) {
                explicit_tet<float>(P, t, v, base);
            } else {
                int64_t ci, cj, ck;
                ok = cube_of_unit(P, t / 6, ci, cj, ck);
                if (ok) lattice_tet<float>(P, ci, cj, ck, (int)(t % 6), v, base);
            }
            if (ok) {
                TetSetup<float> ts;
                tet_setup<float>(v, ts);
                ncell = (int64_t)ts.dim[0] * ts.dim[1] * ts.dim[2];
                cand = tet_ok(base, ts) && ts.vol6 != 0.0 && ncell > 1 && ncell <= (int64_t)INT32_MAX;
                // the work items count pairs: column runs (both passes clip runs)
                if (cand) npair = run_count(ts.dim, ts.axis);
                if (MODEL && cand) tet_features(ts, f);
            }
        }
        bool queue;
        if (MODEL) {
            float y[kNOut];
            mlp_warp(P.model, msm[(threadIdx.x >> 5) & 3], lane, f, y);
            queue = cand && expm1f(y[1]) > (float)P.split_cells;
        } else {
            queue = cand && ncell > P.split_cells;
        }
        const unsigned bal = __ballot_sync(kFull, queue);
        if (bal) {
            unsigned long long b0 = 0;
            if (lane == 0) b0 = atomicAdd(&P.ws->queue_count, (unsigned long long)__popc(bal));
            b0 = __shfl_sync(kFull, b0, 0);
            if (queue) {
                const int64_t idx = (int64_t)b0 + __popc(bal & ((1u << lane) - 1u));
                if (idx < P.q_cap) {
                    P.q_tet[idx] = t;
                    P.q_cells[idx] = (int32_t)npair;
                    if (MODEL) atomicOr(P.qbits + (t >> 5), 1u << (t & 31));
                } else {
                    P.ws->queue_overflow = 1;
                }
            }
        }
    }
}

// One block: chunk_start = exclusive prefix of ceil(q_cells / chunk_cells).
__global__ void __launch_bounds__(1024) k_chunk_scan(const DepositParams P)
{
    __shared__ long long part[1024];
    Workspace *ws = P.ws;
    if (ws->queue_overflow) {
        if (threadIdx.x == 0) ws->n_chunk_items = 0;
        return;
    }
    const int64_t q = min((int64_t)ws->queue_count, P.q_cap);
    const int64_t per = (q + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = min(q, b + per);
    const int64_t cc = P.chunk_cells;
    long long sum = 0;
    for (int64_t i = b; i < e; ++i) sum += (P.q_cells[i] + cc - 1) / cc;
    part[threadIdx.x] = sum;
    __syncthreads();
    // inclusive scan of the per-thread sums (Hillis-Steele)
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const long long y = (threadIdx.x >= (unsigned)o) ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    long long run = part[threadIdx.x] - sum;
    for (int64_t i = b; i < e; ++i) {
        P.chunk_start[i] = run;
        run += (P.q_cells[i] + cc - 1) / cc;
    }
    if (threadIdx.x == blockDim.x - 1) {
        P.chunk_start[q] = part[threadIdx.x];
        ws->n_chunk_items = (unsigned long long)part[threadIdx.x];
    }
}

// ---------------------------------------------------------------------------
// end of an FP32 deposit: compensated pairs (hi, lo) become hi + lo in FP64, in place (COMP),
// and the mass renormalisation out *= (sum of m_t) / (sum of deposits) (SCALE)
// ---------------------------------------------------------------------------
template <bool COMP, bool SCALE>
__global__ void k_finish(double *__restrict__ out, long long n, const Workspace *__restrict__ ws)
{
    double f = 1.0;
    if (SCALE) {
        const double dep = ws->mass_deposited;
        if (dep > 0.0) f = ws->mass_target / dep;
        else if (!COMP) return;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v;
        if (COMP) {
            const float2 p = reinterpret_cast<const float2 *>(out)[i];
            v = (double)p.x + (double)p.y;
        } else {
            v = out[i];
        }
        out[i] = v * f;
    }
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
    if (p.comp) return launch_coop_comp(p, stats, blocks_per_sm, false, p.n_items, st);
    return launch_coop<false, Acc::F64>(p, stats, blocks_per_sm, p.n_items, st);
}

cudaError_t launch_warp_per_tet(const DepositParams &p, bool stats, cudaStream_t st)
{
    const int threads = kCoopThreads;
    const size_t smem = warp_smem_bytes(threads / 32, false);
    const void *k = stats ? (const void *)k_warp_per_tet<true> : (const void *)k_warp_per_tet<false>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int blocks = persistent_blocks(k, threads, smem);
    if (blocks > kMaxWarpBlocks) blocks = kMaxWarpBlocks;
    void *args[] = {const_cast<DepositParams *>(&p)};
    return cudaLaunchKernel(k, dim3(blocks), dim3(threads), args, smem, st);
}

cudaError_t launch_binned(const DepositParams &p, bool stats, int blocks_per_sm, cudaStream_t st)
{
    const int64_t n_tets = (p.src == SRC_TETS) ? p.n_units : 6 * p.n_units;
    int64_t blocks = (n_tets + 127) / 128;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    if (p.model) k_bin_pass<true><<<(unsigned)blocks, 128, 0, st>>>(p);
    else k_bin_pass<false><<<(unsigned)blocks, 128, 0, st>>>(p);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_chunk_scan<<<1, 1024, 0, st>>>(p);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    // the chunk count is known only on the device: size the grid for the rows plus the
    // largest possible number of chunk items (the persistent grid is capped anyway)
    if (p.comp) return launch_coop_comp(p, stats, blocks_per_sm, true, p.n_items + p.q_cap, st);
    return launch_coop<true, Acc::F64>(p, stats, blocks_per_sm, p.n_items + p.q_cap, st);
}

cudaError_t launch_finish(double *out, int64_t n, const Workspace *ws, bool comp, bool scale, cudaStream_t st)
{
    const int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    if (comp && scale) k_finish<true, true><<<(unsigned)blocks, threads, 0, st>>>(out, n, ws);
    else if (comp) k_finish<true, false><<<(unsigned)blocks, threads, 0, st>>>(out, n, ws);
    else if (scale) k_finish<false, true><<<(unsigned)blocks, threads, 0, st>>>(out, n, ws);
    return cudaGetLastError();
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
