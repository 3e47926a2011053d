// abi.cu -- extern "C" entry points declared in include/pse.h: argument checks,
// workspace handling, launches and the host-side readback of counters.
#include <cfloat>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pse.h"
#include "internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(PSE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

pse_deposit_opts default_opts()
{
    pse_deposit_opts o;
    std::memset(&o, 0, sizeof(o));
    o.precision = PSE_FP32_FP64ACC;
    o.schedule = PSE_WARP_COOPERATIVE;
    o.guard_eps = 0.0;
    o.spin_limit = 0;
    o.accumulate = 0;
    o.mass_fixup = 1;
    return o;
}

// FP32 guard: a tetrahedron whose conditioning estimate kappa (total face area x longest
// edge / |6V|; about 8 for an undistorted Kuhn tetrahedron) exceeds kappa_max is clipped
// in float64.  kappa_max = 3.2e6 * guard_eps (32 by default): measured against the FP64
// oracle on shell-crossed Zel'dovich and jittered lattices, FP32 clips of tetrahedra
// below this bound keep the per-cell error (relative, floored at 1e-3 of the mean cell
// mass) below guard_eps.
constexpr double kDefaultGuardEps = 1.0e-5;

// resident blocks per SM of the warp-cooperative kernel (1: no register cap; 2: 128 registers)
constexpr int kDefaultBlocksPerSm = 4;  // 128-thread blocks: 128 registers per thread, 16 warps per SM

float kappa_limit(double guard_eps)
{
    const double g = guard_eps > 0.0 ? guard_eps : kDefaultGuardEps;
    return (float)(3.2e6 * g);
}

struct WsLease {
    pse::Workspace *ws = nullptr;
    bool owned = false;
    cudaStream_t st = nullptr;
    ~WsLease()
    {
        if (owned && ws) cudaFreeAsync(ws, st);
    }
};

// need: total bytes (the Workspace header is cleared; anything after it is scratch)
int acquire_ws(void *d_ws, size_t ws_bytes, cudaStream_t st, WsLease &lease, size_t need = pse::kWorkspaceBytes,
               bool clear = true)
{
    lease.st = st;
    if (d_ws == nullptr) {
        if (ws_bytes != 0) return fail(PSE_ERR_INVALID_ARG, "d_ws is NULL but ws_bytes is %zu", ws_bytes);
        void *p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, need, st);
        if (e != cudaSuccess) return fail(PSE_ERR_OOM, "workspace allocation failed: %s", cudaGetErrorString(e));
        lease.ws = static_cast<pse::Workspace *>(p);
        lease.owned = true;
    } else {
        if (ws_bytes < need)
            return fail(PSE_ERR_WORKSPACE, "ws_bytes = %zu < required %zu", ws_bytes, need);
        if (reinterpret_cast<uintptr_t>(d_ws) % 16 != 0) return fail(PSE_ERR_INVALID_ARG, "d_ws must be 16-byte aligned");
        lease.ws = static_cast<pse::Workspace *>(d_ws);
    }
    if (!clear) return PSE_OK;
    cudaError_t e = cudaMemsetAsync(lease.ws, 0, pse::kWorkspaceBytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "workspace clear");
    return PSE_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs of the binned deposit: the call's launch sequence (workspace and output
// clears, bin pass, scan, persistent kernel, renormalisation) is captured once per
// distinct argument set and replayed afterwards.
// ---------------------------------------------------------------------------
struct GraphEntry {
    std::string key;
    int dev;
    cudaGraphExec_t exec;
};
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;       // most recently used last
constexpr size_t kMaxGraphs = 16;
cudaStream_t g_capture_stream[64] = {};

std::string graph_key(const pse::DepositParams &p, int64_t cells, bool accumulate, bool renorm, int bps)
{
    std::string k(reinterpret_cast<const char *>(&p), sizeof(p));
    const int64_t extra[4] = {cells, accumulate ? 1 : 0, renorm ? 1 : 0, bps};
    k.append(reinterpret_cast<const char *>(extra), sizeof(extra));
    return k;
}

int check_grid(const int64_t grid_n[3], int64_t &cells)
{
    if (!grid_n) return fail(PSE_ERR_INVALID_ARG, "grid_n is NULL");
    cells = 1;
    for (int a = 0; a < 3; ++a) {
        if (grid_n[a] < 1 || grid_n[a] > (int64_t(1) << 24))
            return fail(PSE_ERR_INVALID_ARG, "grid_n[%d] = %lld out of range [1, 2^24]", a, (long long)grid_n[a]);
        cells *= grid_n[a];
    }
    return PSE_OK;
}

int check_opts(const pse_deposit_opts &o)
{
    if (o.precision != PSE_FP64_PLAIN && o.precision != PSE_FP32_FP64ACC && o.precision != PSE_FP32_COMPENSATED)
        return fail(PSE_ERR_INVALID_ARG, "unknown precision %d", o.precision);
    if (o.precision == PSE_FP32_COMPENSATED && o.accumulate)
        return fail(PSE_ERR_UNSUPPORTED, "compensated FP32 accumulation overwrites its output (accumulate = 0)");
    if (o.schedule != PSE_THREAD_PER_TET && o.schedule != PSE_WARP_COOPERATIVE && o.schedule != PSE_BINNED_PERSISTENT &&
        o.schedule != PSE_WARP_PER_TET)
        return fail(PSE_ERR_INVALID_ARG, "unknown schedule %d", o.schedule);
    if (o.schedule != PSE_THREAD_PER_TET && o.precision == PSE_FP64_PLAIN)
        return fail(PSE_ERR_UNSUPPORTED, "the warp-cooperative and binned schedules run the FP32 clip (precision 1)");
    if (o.n_cube_ids < 0) return fail(PSE_ERR_INVALID_ARG, "n_cube_ids < 0");
    if (o.n_cube_ids > 0 && !o.d_cube_ids) return fail(PSE_ERR_INVALID_ARG, "n_cube_ids > 0 but d_cube_ids is NULL");
    return PSE_OK;
}

void fill_grid(pse::DepositParams &p, const int64_t grid_n[3], double box)
{
    for (int a = 0; a < 3; ++a) {
        p.g[a] = grid_n[a];
        p.scale_d[a] = (double)grid_n[a] / box;
        p.scale_f[a] = (float)p.scale_d[a];
    }
}

// ---------------------------------------------------------------------------
// Slab streaming: the particle lattice stays in host memory and is copied to the GPU
// one z-slab at a time (slab_cubes cube layers = slab_cubes + 1 particle rows, the last
// one the halo row, taken modulo n2), double-buffered: the copy of slab s + 1 runs on a
// second stream while the kernels of slab s run on `st`.  per_slab(p, st) enqueues the
// work of one slab, p describing it in slab mode.
// ---------------------------------------------------------------------------
template <class F>
int stream_slabs(const float *h_pos, const pse::DepositParams &base, int64_t slab_cubes, cudaStream_t st, F per_slab)
{
    const int64_t n0 = base.n[0], n1 = base.n[1], n2 = base.n[2];
    const size_t row = (size_t)n0 * (size_t)n1 * 3;  // floats per particle row
    const int64_t nslab = (n2 + slab_cubes - 1) / slab_cubes;
    const size_t buf_bytes = (size_t)(slab_cubes + 1) * row * sizeof(float);
    cudaStream_t cs = nullptr;
    cudaEvent_t ready = nullptr, copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
    float *buf[2] = {nullptr, nullptr};
    int rc = PSE_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&freed[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&buf[b]), buf_bytes, st);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ready, st);  // the buffers exist once st gets here
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ready, 0);
    if (e != cudaSuccess) rc = (e == cudaErrorMemoryAllocation) ? fail(PSE_ERR_OOM, "slab buffers: %s",
                                                                        cudaGetErrorString(e))
                                                               : cuda_fail(e, "slab stream set-up");
    for (int64_t sl = 0; sl < nslab && rc == PSE_OK; ++sl) {
        const int b = (int)(sl & 1);
        const int64_t k0 = sl * slab_cubes, k1 = std::min(n2, k0 + slab_cubes);
        if (sl >= 2) e = cudaStreamWaitEvent(cs, freed[b], 0);  // slab sl - 2 no longer reads buf[b]
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(buf[b], h_pos + (size_t)k0 * row, (size_t)(k1 - k0) * row * sizeof(float),
                                cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess)  // halo row
            e = cudaMemcpyAsync(buf[b] + (size_t)(k1 - k0) * row, h_pos + (size_t)(k1 % n2) * row, row * sizeof(float),
                                cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(copied[b], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, copied[b], 0);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "slab copy");
            break;
        }
        pse::DepositParams p = base;
        p.pos = buf[b];
        p.slab = 1;
        p.n[2] = k1 - k0 + 1;
        p.nc[2] = k1 - k0;
        p.src = pse::SRC_LATTICE;
        p.n_units = p.nc[0] * p.nc[1] * p.nc[2];
        p.n_items = ((p.nc[0] + 31) / 32) * p.nc[1] * p.nc[2];
        rc = per_slab(p, st);
        if (rc != PSE_OK) break;
        e = cudaEventRecord(freed[b], st);
        if (e != cudaSuccess) rc = cuda_fail(e, "slab event");
    }
    // st finishes every kernel after the copies it waited for, so the buffers can go
    for (int b = 0; b < 2; ++b) {
        if (buf[b]) cudaFreeAsync(buf[b], st);
        if (copied[b]) cudaEventDestroy(copied[b]);
        if (freed[b]) cudaEventDestroy(freed[b]);
    }
    if (ready) cudaEventDestroy(ready);
    if (cs) cudaStreamDestroy(cs);
    return rc;
}

constexpr int kDefaultSplitCells = 1024;
constexpr int kDefaultChunkCells = 512;

// workspace of a deposit; n_tets < 0: unknown (0 is returned if it matters)
// [Workspace header][warp kernels: residual blocks, guarded-tetrahedron list][binned: queue]
// [cost model: bitmap]
size_t deposit_ws_bytes(const pse_deposit_opts *o, int64_t n_tets)
{
    const int sched = o ? o->schedule : PSE_WARP_COOPERATIVE;
    if (sched == PSE_THREAD_PER_TET) return pse::kWorkspaceBytes;
    const size_t base = pse::kWorkspaceBytes + pse::kResidualBytes + pse::kGuardListBytes;
    if (sched != PSE_BINNED_PERSISTENT) return base;
    if (!o->cost_model) return base + pse::kQueueBytes;
    if (n_tets < 0) return 0;
    return base + pse::kQueueBytes + pse::qbits_bytes(n_tets);
}

// octree deposits: the header, plus the residual blocks and the guarded-tetrahedron list for
// the warp kernel
size_t octree_ws_bytes(const pse_deposit_opts *o)
{
    return (o && o->schedule == PSE_THREAD_PER_TET)
               ? pse::kWorkspaceBytes
               : pse::kWorkspaceBytes + pse::kResidualBytes + pse::kGuardListBytes;
}

// h_pos != NULL: stream the lattice from host memory in z-slabs of slab_cubes cube layers
int run_deposit(pse::DepositParams &p, const pse_deposit_opts &o, int64_t cells, pse_deposit_stats *h_stats,
                void *d_ws, size_t ws_bytes, cudaStream_t st, const float *h_pos = nullptr, int64_t slab_cubes = 0)
{
    const bool binned = o.schedule == PSE_BINNED_PERSISTENT && !p.leaves;
    const pse_tuning *tu = static_cast<const pse_tuning *>(o.tuning);
    const bool stats = h_stats != nullptr;
    const bool streamed = h_pos != nullptr;
    const bool graph = tu && tu->use_graph && d_ws != nullptr && !stats && !streamed;
    WsLease lease;
    // streamed: tetrahedron ids (cost-model bitmap) are slab-local
    const int64_t n_tets = streamed ? 6 * p.nc[0] * p.nc[1] * std::min(slab_cubes, p.nc[2])
                                    : (p.src == pse::SRC_TETS) ? p.n_units : 6 * p.n_units;
    int rc = acquire_ws(d_ws, ws_bytes, st, lease, p.leaves ? octree_ws_bytes(&o) : deposit_ws_bytes(&o, n_tets),
                        false);
    if (rc != PSE_OK) return rc;
    p.ws = lease.ws;
    if (o.schedule != PSE_THREAD_PER_TET)
        p.vres = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(lease.ws) + pse::kWorkspaceBytes);
    unsigned char *const list = reinterpret_cast<unsigned char *>(lease.ws) + pse::kWorkspaceBytes +
                                pse::kResidualBytes;
    unsigned char *const after_res = list + pse::kGuardListBytes;
    if (o.schedule != PSE_THREAD_PER_TET) {
        const int32_t cap = tu ? tu->guard_list_cap : 0;
        p.guard_list = reinterpret_cast<int64_t *>(list);
        p.guard_cap = cap < 0 ? 0 : (cap > 0 && cap < pse::kGuardListCap ? cap : pse::kGuardListCap);
    }
    size_t qbits_len = 0;
    if (binned && o.cost_model) {
        p.model = static_cast<const pse::CostModelDev *>(o.cost_model);
        p.qbits = reinterpret_cast<uint32_t *>(after_res + pse::kQueueBytes);
        qbits_len = pse::qbits_bytes(n_tets);
    }
    if (binned) {
        unsigned char *q = after_res;
        p.q_tet = reinterpret_cast<int64_t *>(q);
        p.chunk_start = reinterpret_cast<int64_t *>(q + (size_t)pse::kQueueCap * 8);
        p.q_cells = reinterpret_cast<int32_t *>(q + (size_t)pse::kQueueCap * 8 + (size_t)(pse::kQueueCap + 1) * 8);
        p.q_cap = pse::kQueueCap;
        p.split_cells = (tu && tu->split_cells > 0) ? tu->split_cells : kDefaultSplitCells;
        p.chunk_cells = (tu && tu->chunk_cells > 0) ? tu->chunk_cells : kDefaultChunkCells;
        if (p.chunk_cells > (1 << 24)) p.chunk_cells = 1 << 24;
    }
    p.kappa_max = kappa_limit(o.guard_eps);
    // FP32 mass renormalisation: the call's deposits are scaled by sum(m_t)/sum(deposits);
    // it needs the output to hold this call's deposits only (accumulate = 0)
    const bool renorm = o.mass_fixup && !o.accumulate && o.precision != PSE_FP64_PLAIN;
    p.fixup = renorm ? 1 : 0;
    const bool comp = o.precision == PSE_FP32_COMPENSATED;
    p.comp = comp ? 1 : 0;
    const int bps = (tu && tu->blocks_per_sm > 0) ? tu->blocks_per_sm : kDefaultBlocksPerSm;
    if (p.n_units > 0 && o.schedule != PSE_THREAD_PER_TET)
        p.n_items = (p.src == pse::SRC_LATTICE) ? ((p.nc[0] + 31) / 32) * p.nc[1] * p.nc[2] : (p.n_units + 31) / 32;

    // the kernels of one deposit pass over the tetrahedra of q, on stream s
    auto launch = [&](const pse::DepositParams &q, cudaStream_t s) -> int {
        if (q.n_units <= 0) return PSE_OK;
        cudaError_t e;
        if (q.leaves) {
            e = pse::launch_octree_deposit(q, o.precision == PSE_FP64_PLAIN, o.schedule == PSE_THREAD_PER_TET, stats,
                                           bps, s);
            if (e != cudaSuccess) return cuda_fail(e, "octree deposit launch");
        } else {
            if (o.schedule == PSE_THREAD_PER_TET) e = pse::launch_thread_per_tet(q, o.precision == PSE_FP64_PLAIN, stats, s);
            else if (o.schedule == PSE_WARP_PER_TET) e = pse::launch_warp_per_tet(q, stats, s);
            else if (binned) e = pse::launch_binned(q, stats, bps, s);
            else e = pse::launch_warp_coop(q, stats, bps, s);
            if (e != cudaSuccess) return cuda_fail(e, "deposit launch");
        }
        return PSE_OK;
    };
    // the whole launch sequence of the call, on stream s
    auto enqueue = [&](cudaStream_t s) -> int {
        cudaError_t e = cudaMemsetAsync(p.ws, 0, pse::kWorkspaceBytes, s);
        if (e != cudaSuccess) return cuda_fail(e, "workspace clear");
        if (qbits_len && !streamed) {
            e = cudaMemsetAsync(p.qbits, 0, qbits_len, s);
            if (e != cudaSuccess) return cuda_fail(e, "queue bitmap clear");
        }
        if (!o.accumulate) {
            e = cudaMemsetAsync(p.out, 0, (size_t)cells * sizeof(double), s);
            if (e != cudaSuccess) return cuda_fail(e, "output clear");
        }
        int r;
        if (!streamed) {
            r = launch(p, s);
        } else {
            // statistics and mass sums run over all slabs; the work counter and the binned
            // schedule's queue state restart with every slab
            r = stream_slabs(h_pos, p, slab_cubes, s, [&](pse::DepositParams &q, cudaStream_t ss) -> int {
                cudaError_t e2 = cudaMemsetAsync(&q.ws->work_counter, 0, 2 * sizeof(q.ws->work_counter), ss);
                if (e2 == cudaSuccess)
                    e2 = cudaMemsetAsync(&q.ws->queue_count, 0,
                                         sizeof(pse::Workspace) - offsetof(pse::Workspace, queue_count), ss);
                if (e2 == cudaSuccess && qbits_len) e2 = cudaMemsetAsync(q.qbits, 0, qbits_len, ss);
                if (e2 != cudaSuccess) return cuda_fail(e2, "slab workspace reset");
                return launch(q, ss);
            });
        }
        if (r != PSE_OK) return r;
        if ((renorm || comp) && p.n_units > 0) {
            e = pse::launch_finish(p.out, cells, p.ws, comp, renorm, s);
            if (e != cudaSuccess) return cuda_fail(e, "deposit finish launch");
        }
        return PSE_OK;
    };

    cudaError_t e;
    if (!graph) {
        rc = enqueue(st);
        if (rc != PSE_OK) return rc;
    } else {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        if (dev < 0 || dev >= 64) return fail(PSE_ERR_UNSUPPORTED, "device index beyond the supported range");
        const std::string key = graph_key(p, cells, o.accumulate != 0, renorm, bps);
        std::lock_guard<std::mutex> lk(g_graph_mu);
        cudaGraphExec_t exec = nullptr;
        for (size_t i = 0; i < g_graphs.size(); ++i)
            if (g_graphs[i].dev == dev && g_graphs[i].key == key) {
                GraphEntry hit = g_graphs[i];
                g_graphs.erase(g_graphs.begin() + (long)i);
                g_graphs.push_back(hit);
                exec = hit.exec;
                break;
            }
        if (!exec) {
            if (!g_capture_stream[dev]) {
                e = cudaStreamCreateWithFlags(&g_capture_stream[dev], cudaStreamNonBlocking);
                if (e != cudaSuccess) return cuda_fail(e, "capture stream");
            }
            cudaStream_t cs = g_capture_stream[dev];
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(e, "graph capture begin");
            const int rc2 = enqueue(cs);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(cs, &g);
            if (rc2 != PSE_OK) {
                if (g) cudaGraphDestroy(g);
                return rc2;
            }
            if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
            e = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
            if (g_graphs.size() >= kMaxGraphs) {
                cudaGraphExecDestroy(g_graphs.front().exec);
                g_graphs.erase(g_graphs.begin());
            }
            g_graphs.push_back(GraphEntry{key, dev, exec});
        }
        e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    }
    if (stats) {
        pse::Workspace hw;
        e = cudaMemcpyAsync(&hw, lease.ws, sizeof(hw), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "stats readback");
        std::memset(h_stats, 0, sizeof(*h_stats));
        h_stats->tets = hw.stats[pse::ST_TETS];
        h_stats->bbox_cells = hw.stats[pse::ST_BBOX_CELLS];
        h_stats->inside_cells = hw.stats[pse::ST_INSIDE_CELLS];
        h_stats->partial_clips = hw.stats[pse::ST_PARTIAL_CLIPS];
        h_stats->fp64_redos = hw.stats[pse::ST_FP64_REDOS];
        h_stats->degenerate_tets = hw.stats[pse::ST_DEGENERATE];
        h_stats->single_cell_tets = hw.stats[pse::ST_SINGLE_CELL];
        for (int b = 0; b < 8; ++b) h_stats->bin_counts[b] = hw.stats[pse::ST_BIN0 + b];
        h_stats->mass_in = hw.mass_in;
        h_stats->mass_dropped = hw.mass_dropped;
        h_stats->inverted_tets = hw.stats[pse::ST_INVERTED];
        h_stats->overlapped_cells = hw.stats[pse::ST_OVERLAPPED];
        h_stats->column_runs = hw.stats[pse::ST_RUNS];
        // the mass this call wrote into the output: its in-grid deposits, times the
        // renormalisation factor when it applied
        const double in_grid = hw.mass_deposited - hw.mass_dropped;
        h_stats->mass_out = (renorm && hw.mass_deposited > 0.0) ? in_grid * (hw.mass_target / hw.mass_deposited)
                                                                 : in_grid;
        if (hw.error_code != 0)
            return fail(PSE_ERR_DEVICE,
                        hw.error_code == 1 ? "a tetrahedron is wider than the periodic grid (detail %d)"
                        : hw.error_code == 2 ? "a tetrahedron overlaps more than 2^25 cells (detail %d)"
                        : hw.error_code == 3 ? "a cube id is out of range (work unit %d)"
                        : hw.error_code == 4 ? "non-finite or out-of-range vertex coordinates (detail %d)"
                                             : "device-side check failed (detail %d)",
                        hw.error_detail);
    }
    return PSE_OK;
}


constexpr int kMaxOctreeLevel = 10;

// histogram counters of levels 0 .. max_level-1, 64 bins per node
size_t hist_bytes(int max_level)
{
    size_t n = 0;
    for (int l = 0; l < max_level; ++l) n += ((size_t)1 << (3 * l)) * 64;
    return (n * sizeof(unsigned) + 255) / 256 * 256;
}

int check_lattice(const pse_lattice *lat)
{
    if (!lat) return fail(PSE_ERR_INVALID_ARG, "lat is NULL");
    for (int a = 0; a < 3; ++a)
        if (lat->n[a] < 2) return fail(PSE_ERR_INVALID_ARG, "lat->n[%d] = %lld < 2", a, (long long)lat->n[a]);
    if (!(lat->box > 0.0) || !std::isfinite(lat->box)) return fail(PSE_ERR_INVALID_ARG, "lat->box must be > 0");
    if (!std::isfinite(lat->particle_mass)) return fail(PSE_ERR_INVALID_ARG, "lat->particle_mass must be finite");
    return PSE_OK;
}

void lattice_params(pse::DepositParams &p, const float *d_pos, const pse_lattice *lat, const pse_deposit_opts &o)
{
    p.periodic = lat->periodic ? 1 : 0;
    p.pos = d_pos;
    for (int a = 0; a < 3; ++a) {
        p.n[a] = lat->n[a];
        p.nc[a] = p.periodic ? lat->n[a] : lat->n[a] - 1;
    }
    p.box = lat->box;
    p.m_tet = lat->particle_mass / 6.0;
    if (o.d_cube_ids) {
        p.src = pse::SRC_CUBE_LIST;
        p.cube_ids = o.d_cube_ids;
        p.n_units = o.n_cube_ids;
    } else {
        p.src = pse::SRC_LATTICE;
        p.n_units = p.nc[0] * p.nc[1] * p.nc[2];
    }
}

// leaves -> finest-level map, checking that they tile the box exactly
int fine_map_of(const int32_t *leaves, int64_t n_leaves, int max_level, std::vector<int32_t> &map)
{
    const int64_t F = (int64_t)1 << max_level;
    map.assign((size_t)(F * F * F), -1);
    for (int64_t l = 0; l < n_leaves; ++l) {
        const int32_t *L = leaves + 4 * l;
        if (L[0] < 0 || L[0] > max_level)
            return fail(PSE_ERR_INVALID_ARG, "leaf %lld: level %d outside [0, %d]", (long long)l, L[0], max_level);
        const int64_t nn = (int64_t)1 << L[0], span = F / nn;
        for (int a = 1; a < 4; ++a)
            if (L[a] < 0 || L[a] >= nn)
                return fail(PSE_ERR_INVALID_ARG, "leaf %lld: node index out of range", (long long)l);
        for (int64_t z = L[3] * span; z < (L[3] + 1) * span; ++z)
            for (int64_t y = L[2] * span; y < (L[2] + 1) * span; ++y)
                for (int64_t x = L[1] * span; x < (L[1] + 1) * span; ++x) {
                    int32_t &m = map[(size_t)(x + F * (y + F * z))];
                    if (m != -1) return fail(PSE_ERR_INVALID_ARG, "leaves %d and %lld overlap", m, (long long)l);
                    m = (int32_t)l;
                }
    }
    for (size_t i = 0; i < map.size(); ++i)
        if (map[i] < 0) return fail(PSE_ERR_INVALID_ARG, "the leaves do not tile the box");
    return PSE_OK;
}

// depth-first refinement from the level histograms (lower-median bin edge rule)
void decide(const std::vector<unsigned> &hist, int max_level, double threshold, int level, int64_t ix, int64_t iy,
            int64_t iz, std::vector<int32_t> &leaves)
{
    bool refine = false;
    if (level < max_level) {
        size_t off = 0;
        for (int l = 0; l < level; ++l) off += ((size_t)1 << (3 * l)) * 64;
        const int64_t nn = (int64_t)1 << level;
        const unsigned *h = hist.data() + off + (size_t)(ix + nn * (iy + nn * iz)) * 64;
        unsigned long long count = 0;
        for (int b = 0; b < 64; ++b) count += h[b];
        if (count > 0) {
            const unsigned long long k = (count - 1) / 2;
            unsigned long long cum = 0;
            int bin = 63;
            for (int b = 0; b < 64; ++b) {
                cum += h[b];
                if (cum > k) { bin = b; break; }
            }
            const double lower_edge = std::pow(10.0, -3.0 + 6.0 * bin / 64.0);
            refine = lower_edge < threshold;
        }
    }
    if (!refine) {
        leaves.push_back(level);
        leaves.push_back((int32_t)ix);
        leaves.push_back((int32_t)iy);
        leaves.push_back((int32_t)iz);
        return;
    }
    for (int c = 0; c < 8; ++c)
        decide(hist, max_level, threshold, level + 1, 2 * ix + (c & 1), 2 * iy + ((c >> 1) & 1), 2 * iz + (c >> 2),
               leaves);
}

int make_octree(const int32_t *leaves, int64_t n_leaves, int32_t bc, int32_t max_level, double box, pse_octree *out)
{
    std::vector<int32_t> map;
    int rc = fine_map_of(leaves, n_leaves, max_level, map);
    if (rc != PSE_OK) return rc;
    pse_octree o;
    std::memset(&o, 0, sizeof(o));
    o.bc = bc;
    o.max_level = max_level;
    o.n_leaves = n_leaves;
    o.box = box;
    o.n_cells = n_leaves * (int64_t)bc * bc * bc;
    o.h_leaves = static_cast<int32_t *>(std::malloc((size_t)n_leaves * 4 * sizeof(int32_t)));
    if (!o.h_leaves) return fail(PSE_ERR_OOM, "host allocation failed");
    std::memcpy(o.h_leaves, leaves, (size_t)n_leaves * 4 * sizeof(int32_t));
    cudaError_t e = cudaMalloc(&o.d_leaves, (size_t)n_leaves * 4 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&o.d_fine_map, map.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemcpy(o.d_leaves, leaves, (size_t)n_leaves * 4 * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(o.d_fine_map, map.data(), map.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pse_free_octree(&o);
        return fail(e == cudaErrorMemoryAllocation ? PSE_ERR_OOM : PSE_ERR_CUDA, "octree upload: %s",
                    cudaGetErrorString(e));
    }
    *out = o;
    return PSE_OK;
}
}  // namespace

namespace pse {
void set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }
}  // namespace pse

extern "C" {

const char *pse_last_error(void) { return g_last_error.c_str(); }

int pse_abi_version(void) { return PSE_ABI_VERSION; }

size_t pse_workspace_size(int op, const pse_lattice *lat, const void *op_params)
{
    switch (op) {
    case PSE_OP_DEPOSIT_UNIFORM:
        return deposit_ws_bytes(static_cast<const pse_deposit_opts *>(op_params),
                                lat ? 6 * (lat->periodic ? lat->n[0] * lat->n[1] * lat->n[2]
                                                         : (lat->n[0] - 1) * (lat->n[1] - 1) * (lat->n[2] - 1))
                                    : -1);
    case PSE_OP_DEPOSIT_TETS:
        return deposit_ws_bytes(static_cast<const pse_deposit_opts *>(op_params), -1);
    case PSE_OP_DEPOSIT_OCTREE:
        return octree_ws_bytes(static_cast<const pse_deposit_opts *>(op_params));
    case PSE_OP_BUILD_OCTREE: {
        if (!op_params) return 0;
        const int32_t ml = *static_cast<const int32_t *>(op_params);
        if (ml < 0 || ml > kMaxOctreeLevel) return 0;
        return pse::kWorkspaceBytes + hist_bytes(ml);
    }
    default:
        return 0;
    }
}

int pse_build_tets_from_lagrangian_grid(const float *d_pos, const pse_lattice *lat, int32_t *d_tet_vidx,
                                        float *d_tet_vol, int64_t *h_n_tets, void *stream)
{
    g_last_error.clear();
    if (!d_pos || !lat) return fail(PSE_ERR_INVALID_ARG, "d_pos and lat must be non-NULL");
    for (int a = 0; a < 3; ++a)
        if (lat->n[a] < 2) return fail(PSE_ERR_INVALID_ARG, "lat->n[%d] = %lld < 2", a, (long long)lat->n[a]);
    if (!(lat->box > 0.0) || !std::isfinite(lat->box)) return fail(PSE_ERR_INVALID_ARG, "lat->box must be > 0");
    int64_t nc[3];
    for (int a = 0; a < 3; ++a) nc[a] = lat->periodic ? lat->n[a] : lat->n[a] - 1;
    const int64_t n_tets = 6 * nc[0] * nc[1] * nc[2];
    if (d_tet_vidx && lat->n[0] * lat->n[1] * lat->n[2] > INT32_MAX)
        return fail(PSE_ERR_INVALID_ARG, "particle indices do not fit int32");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d_tet_vidx || d_tet_vol) {
        cudaError_t e = pse::launch_build_tets(d_pos, lat->n, nc, lat->periodic, lat->box, d_tet_vidx, d_tet_vol, n_tets, st);
        if (e != cudaSuccess) return cuda_fail(e, "build_tets launch");
    }
    if (h_n_tets) {
        *h_n_tets = n_tets;
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "build_tets");
    }
    return PSE_OK;
}

int pse_deposit_uniform(const float *d_pos, const pse_lattice *lat, const int64_t grid_n[3], double *d_cell_mass,
                        const pse_deposit_opts *opts, pse_deposit_stats *h_stats, void *d_ws, size_t ws_bytes,
                        void *stream)
{
    g_last_error.clear();
    if (!d_pos || !lat || !d_cell_mass) return fail(PSE_ERR_INVALID_ARG, "d_pos, lat and d_cell_mass must be non-NULL");
    for (int a = 0; a < 3; ++a)
        if (lat->n[a] < 2) return fail(PSE_ERR_INVALID_ARG, "lat->n[%d] = %lld < 2", a, (long long)lat->n[a]);
    if (!(lat->box > 0.0) || !std::isfinite(lat->box)) return fail(PSE_ERR_INVALID_ARG, "lat->box must be > 0");
    if (!std::isfinite(lat->particle_mass)) return fail(PSE_ERR_INVALID_ARG, "lat->particle_mass must be finite");
    int64_t cells = 0;
    int rc = check_grid(grid_n, cells);
    if (rc != PSE_OK) return rc;
    const pse_deposit_opts o = opts ? *opts : default_opts();
    rc = check_opts(o);
    if (rc != PSE_OK) return rc;

    pse::DepositParams p;
    std::memset(&p, 0, sizeof(p));
    p.periodic = lat->periodic ? 1 : 0;
    p.pos = d_pos;
    for (int a = 0; a < 3; ++a) {
        p.n[a] = lat->n[a];
        p.nc[a] = p.periodic ? lat->n[a] : lat->n[a] - 1;
    }
    p.box = lat->box;
    p.m_tet = lat->particle_mass / 6.0;
    fill_grid(p, grid_n, lat->box);
    p.out = d_cell_mass;
    if (o.d_cube_ids) {
        p.src = pse::SRC_CUBE_LIST;
        p.cube_ids = o.d_cube_ids;
        p.n_units = o.n_cube_ids;
    } else {
        p.src = pse::SRC_LATTICE;
        p.n_units = p.nc[0] * p.nc[1] * p.nc[2];
    }
    return run_deposit(p, o, cells, h_stats, d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

int pse_octree_from_leaves(const int32_t *h_leaves, int64_t n_leaves, int32_t bc, int32_t max_level, double box,
                           pse_octree *out)
{
    g_last_error.clear();
    if (!h_leaves || !out || n_leaves < 1) return fail(PSE_ERR_INVALID_ARG, "h_leaves and out must be non-NULL, n_leaves >= 1");
    if (bc < 1 || bc > 4096) return fail(PSE_ERR_INVALID_ARG, "bc = %d out of range [1, 4096]", bc);
    if (max_level < 0 || max_level > kMaxOctreeLevel) return fail(PSE_ERR_INVALID_ARG, "max_level out of range");
    if (!(box > 0.0) || !std::isfinite(box)) return fail(PSE_ERR_INVALID_ARG, "box must be > 0");
    return make_octree(h_leaves, n_leaves, bc, max_level, box, out);
}

int pse_build_octree_from_tet_sizes(const float *d_pos, const pse_lattice *lat, int32_t bc, int32_t max_level,
                                    double edge_threshold_cells, pse_octree *out, void *d_ws, size_t ws_bytes,
                                    void *stream)
{
    g_last_error.clear();
    int rc = check_lattice(lat);
    if (rc != PSE_OK) return rc;
    if (!d_pos || !out) return fail(PSE_ERR_INVALID_ARG, "d_pos and out must be non-NULL");
    if (!lat->periodic) return fail(PSE_ERR_UNSUPPORTED, "the octree covers a periodic box");
    if (bc < 1 || bc > 4096) return fail(PSE_ERR_INVALID_ARG, "bc = %d out of range [1, 4096]", bc);
    if (max_level < 0 || max_level > kMaxOctreeLevel) return fail(PSE_ERR_INVALID_ARG, "max_level out of range");
    if (!(edge_threshold_cells > 0.0)) return fail(PSE_ERR_INVALID_ARG, "edge_threshold_cells must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t hb = hist_bytes(max_level);
    const size_t need = pse::kWorkspaceBytes + hb;
    void *ws = d_ws;
    bool owned = false;
    if (!ws) {
        if (ws_bytes != 0) return fail(PSE_ERR_INVALID_ARG, "d_ws is NULL but ws_bytes is %zu", ws_bytes);
        cudaError_t e = cudaMallocAsync(&ws, need, st);
        if (e != cudaSuccess) return fail(PSE_ERR_OOM, "workspace allocation failed: %s", cudaGetErrorString(e));
        owned = true;
    } else if (ws_bytes < need) {
        return fail(PSE_ERR_WORKSPACE, "ws_bytes = %zu < required %zu", ws_bytes, need);
    }
    std::vector<unsigned> hist(hb / sizeof(unsigned), 0u);
    cudaError_t e = cudaMemsetAsync(ws, 0, need, st);
    if (max_level > 0 && e == cudaSuccess) {
        pse::DepositParams p;
        std::memset(&p, 0, sizeof(p));
        pse_deposit_opts o = default_opts();
        lattice_params(p, d_pos, lat, o);
        p.bc = bc;
        p.max_level = max_level;
        p.ws = static_cast<pse::Workspace *>(ws);
        unsigned *d_hist = reinterpret_cast<unsigned *>(static_cast<char *>(ws) + pse::kWorkspaceBytes);
        e = pse::launch_octree_hist(p, d_hist, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hist.data(), d_hist, hb, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (owned) cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "octree histograms");
    std::vector<int32_t> leaves;
    decide(hist, max_level, edge_threshold_cells, 0, 0, 0, 0, leaves);
    return make_octree(leaves.data(), (int64_t)(leaves.size() / 4), bc, max_level, lat->box, out);
}

int pse_deposit_octree(const float *d_pos, const pse_lattice *lat, const pse_octree *oct, double *d_leaf_mass,
                       const pse_deposit_opts *opts, pse_deposit_stats *h_stats, void *d_ws, size_t ws_bytes,
                       void *stream)
{
    g_last_error.clear();
    int rc = check_lattice(lat);
    if (rc != PSE_OK) return rc;
    if (!d_pos || !oct || !d_leaf_mass) return fail(PSE_ERR_INVALID_ARG, "d_pos, oct and d_leaf_mass must be non-NULL");
    if (!oct->d_leaves || !oct->d_fine_map || oct->n_leaves < 1) return fail(PSE_ERR_INVALID_ARG, "oct is empty");
    if (!lat->periodic) return fail(PSE_ERR_UNSUPPORTED, "the octree covers a periodic box");
    if (oct->box != lat->box) return fail(PSE_ERR_INVALID_ARG, "oct->box differs from lat->box");
    const pse_deposit_opts o = opts ? *opts : default_opts();
    rc = check_opts(o);
    if (rc != PSE_OK) return rc;
    pse::DepositParams p;
    std::memset(&p, 0, sizeof(p));
    lattice_params(p, d_pos, lat, o);
    p.out = d_leaf_mass;
    p.bc = oct->bc;
    p.max_level = oct->max_level;
    p.leaves = oct->d_leaves;
    p.fine_map = oct->d_fine_map;
    p.fine = (int64_t)1 << oct->max_level;
    return run_deposit(p, o, oct->n_cells, h_stats, d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

void pse_free_octree(pse_octree *oct)
{
    if (!oct) return;
    if (oct->d_leaves) cudaFree(oct->d_leaves);
    if (oct->d_fine_map) cudaFree(oct->d_fine_map);
    std::free(oct->h_leaves);
    std::memset(oct, 0, sizeof(*oct));
}

int pse_deposit_tets(const float *d_verts, const double *d_tet_mass, int64_t n_tets, double box, int32_t periodic,
                     const int64_t grid_n[3], double *d_cell_mass, const pse_deposit_opts *opts,
                     pse_deposit_stats *h_stats, void *d_ws, size_t ws_bytes, void *stream)
{
    g_last_error.clear();
    if (n_tets < 0) return fail(PSE_ERR_INVALID_ARG, "n_tets < 0");
    if ((n_tets > 0 && (!d_verts || !d_tet_mass)) || !d_cell_mass)
        return fail(PSE_ERR_INVALID_ARG, "d_verts, d_tet_mass and d_cell_mass must be non-NULL");
    if (!(box > 0.0) || !std::isfinite(box)) return fail(PSE_ERR_INVALID_ARG, "box must be > 0");
    int64_t cells = 0;
    int rc = check_grid(grid_n, cells);
    if (rc != PSE_OK) return rc;
    const pse_deposit_opts o = opts ? *opts : default_opts();
    rc = check_opts(o);
    if (rc != PSE_OK) return rc;
    if (o.d_cube_ids) return fail(PSE_ERR_INVALID_ARG, "d_cube_ids applies to lattices only");

    pse::DepositParams p;
    std::memset(&p, 0, sizeof(p));
    p.src = pse::SRC_TETS;
    p.periodic = periodic ? 1 : 0;
    p.verts = d_verts;
    p.tet_mass = d_tet_mass;
    p.n_units = n_tets;
    p.box = box;
    fill_grid(p, grid_n, box);
    p.out = d_cell_mass;
    return run_deposit(p, o, cells, h_stats, d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// the paper's count criterion
// ---------------------------------------------------------------------------
namespace {
void emit_leaves(const std::vector<std::vector<char>> &refine, int level, int64_t ix, int64_t iy, int64_t iz,
                 std::vector<int32_t> &leaves)
{
    const int64_t nn = (int64_t)1 << level;
    const bool r = level < (int)refine.size() && refine[level][(size_t)(ix + nn * (iy + nn * iz))];
    if (!r) {
        leaves.push_back(level);
        leaves.push_back((int32_t)ix);
        leaves.push_back((int32_t)iy);
        leaves.push_back((int32_t)iz);
        return;
    }
    for (int c = 0; c < 8; ++c)
        emit_leaves(refine, level + 1, 2 * ix + (c & 1), 2 * iy + ((c >> 1) & 1), 2 * iz + (c >> 2), leaves);
}
}  // namespace

int pse_build_octree_count(const float *d_pos, const pse_lattice *lat, int32_t bc, int32_t max_level,
                           double count_threshold, int32_t subblock, pse_octree *out, void *stream)
{
    g_last_error.clear();
    int rc = check_lattice(lat);
    if (rc != PSE_OK) return rc;
    if (!d_pos || !out) return fail(PSE_ERR_INVALID_ARG, "d_pos and out must be non-NULL");
    if (!lat->periodic) return fail(PSE_ERR_UNSUPPORTED, "the octree covers a periodic box");
    if (bc < 1 || bc > 4096) return fail(PSE_ERR_INVALID_ARG, "bc = %d out of range [1, 4096]", bc);
    if (max_level < 0 || max_level > kMaxOctreeLevel) return fail(PSE_ERR_INVALID_ARG, "max_level out of range");
    if (!(count_threshold > 0.0)) return fail(PSE_ERR_INVALID_ARG, "count_threshold must be > 0");
    if (subblock < 1) return fail(PSE_ERR_INVALID_ARG, "subblock must be >= 1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nb = ((lat->n[0] + subblock - 1) / subblock) * ((lat->n[1] + subblock - 1) / subblock) *
                       ((lat->n[2] + subblock - 1) / subblock);
    const int64_t max_nodes = max_level > 0 ? ((int64_t)1 << (3 * (max_level - 1))) : 1;
    double *d_boxes = nullptr, *d_counts = nullptr;
    int32_t *d_nodes = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_boxes), (size_t)nb * 7 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&d_counts), (size_t)max_nodes * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&d_nodes), (size_t)max_nodes * 4 * sizeof(int32_t), st);
    if (e == cudaSuccess) e = pse::launch_subblock_boxes(d_pos, lat->n, subblock, lat->box, d_boxes, st);
    // level by level: the nodes whose parent was refined, their estimated counts, the decisions
    std::vector<std::vector<char>> refine;
    std::vector<int32_t> nodes = {0, 0, 0, 0};
    for (int l = 0; l < max_level && e == cudaSuccess && !nodes.empty(); ++l) {
        const int64_t nn = (int64_t)1 << l;
        refine.emplace_back((size_t)(nn * nn * nn), 0);
        const int64_t cnt = (int64_t)nodes.size() / 4;
        std::vector<double> counts((size_t)cnt);
        e = cudaMemcpyAsync(d_nodes, nodes.data(), nodes.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = pse::launch_node_counts(d_boxes, nb, d_nodes, cnt, lat->box, d_counts, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(counts.data(), d_counts, (size_t)cnt * sizeof(double),
                                                  cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        std::vector<int32_t> next;
        for (int64_t i = 0; i < cnt; ++i) {
            if (!(counts[(size_t)i] > count_threshold)) continue;
            const int32_t x = nodes[4 * i + 1], y = nodes[4 * i + 2], z = nodes[4 * i + 3];
            refine[(size_t)l][(size_t)(x + nn * (y + nn * z))] = 1;
            if (l + 1 < max_level)
                for (int c = 0; c < 8; ++c) {
                    next.push_back(l + 1);
                    next.push_back(2 * x + (c & 1));
                    next.push_back(2 * y + ((c >> 1) & 1));
                    next.push_back(2 * z + (c >> 2));
                }
        }
        nodes.swap(next);
    }
    cudaFreeAsync(d_boxes, st);
    cudaFreeAsync(d_counts, st);
    cudaFreeAsync(d_nodes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "octree counts");
    std::vector<int32_t> leaves;
    emit_leaves(refine, 0, 0, 0, 0, leaves);
    return make_octree(leaves.data(), (int64_t)(leaves.size() / 4), bc, max_level, lat->box, out);
}

// ---------------------------------------------------------------------------
// restriction up the octree
// ---------------------------------------------------------------------------
int pse_octree_restrict(const pse_octree *oct, const double *d_leaf_mass, double *d_pyramid, void *stream)
{
    g_last_error.clear();
    if (!oct || !d_leaf_mass || !d_pyramid) return fail(PSE_ERR_INVALID_ARG, "oct, d_leaf_mass and d_pyramid must be non-NULL");
    if (!oct->d_leaves || !oct->d_fine_map || oct->n_leaves < 1) return fail(PSE_ERR_INVALID_ARG, "oct is empty");
    cudaError_t e = pse::launch_octree_restrict(oct->d_fine_map, oct->d_leaves, oct->max_level, oct->bc, d_leaf_mass,
                                                d_pyramid, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSE_OK : cuda_fail(e, "restriction launch");
}

// ---------------------------------------------------------------------------
// slab streaming from host memory
// ---------------------------------------------------------------------------
namespace {
int check_streamed(const float *h_pos, const pse_lattice *lat, int64_t slab_cubes, const pse_deposit_opts &o)
{
    int rc = check_lattice(lat);
    if (rc != PSE_OK) return rc;
    if (!h_pos) return fail(PSE_ERR_INVALID_ARG, "h_pos is NULL");
    if (!lat->periodic) return fail(PSE_ERR_UNSUPPORTED, "slab streaming needs a periodic lattice");
    if (slab_cubes < 1) return fail(PSE_ERR_INVALID_ARG, "slab_cubes must be >= 1");
    if (o.d_cube_ids) return fail(PSE_ERR_UNSUPPORTED, "slab streaming deposits whole lattices (d_cube_ids must be NULL)");
    if (o.tuning && static_cast<const pse_tuning *>(o.tuning)->use_graph)
        return fail(PSE_ERR_UNSUPPORTED, "slab streaming does not replay graphs (use_graph must be 0)");
    return PSE_OK;
}
}  // namespace

int pse_deposit_uniform_streamed(const float *h_pos, const pse_lattice *lat, int64_t slab_cubes,
                                 const int64_t grid_n[3], double *d_cell_mass, const pse_deposit_opts *opts,
                                 pse_deposit_stats *h_stats, void *d_ws, size_t ws_bytes, void *stream)
{
    g_last_error.clear();
    const pse_deposit_opts o = opts ? *opts : default_opts();
    int rc = check_opts(o);
    if (rc != PSE_OK) return rc;
    rc = check_streamed(h_pos, lat, slab_cubes, o);
    if (rc != PSE_OK) return rc;
    if (!d_cell_mass) return fail(PSE_ERR_INVALID_ARG, "d_cell_mass is NULL");
    int64_t cells = 0;
    rc = check_grid(grid_n, cells);
    if (rc != PSE_OK) return rc;
    pse::DepositParams p;
    std::memset(&p, 0, sizeof(p));
    lattice_params(p, h_pos, lat, o);
    fill_grid(p, grid_n, lat->box);
    p.out = d_cell_mass;
    return run_deposit(p, o, cells, h_stats, d_ws, ws_bytes, static_cast<cudaStream_t>(stream), h_pos, slab_cubes);
}

int pse_deposit_octree_streamed(const float *h_pos, const pse_lattice *lat, int64_t slab_cubes, const pse_octree *oct,
                                double *d_leaf_mass, const pse_deposit_opts *opts, pse_deposit_stats *h_stats,
                                void *d_ws, size_t ws_bytes, void *stream)
{
    g_last_error.clear();
    const pse_deposit_opts o = opts ? *opts : default_opts();
    int rc = check_opts(o);
    if (rc != PSE_OK) return rc;
    rc = check_streamed(h_pos, lat, slab_cubes, o);
    if (rc != PSE_OK) return rc;
    if (!oct || !d_leaf_mass) return fail(PSE_ERR_INVALID_ARG, "oct and d_leaf_mass must be non-NULL");
    if (!oct->d_leaves || !oct->d_fine_map || oct->n_leaves < 1) return fail(PSE_ERR_INVALID_ARG, "oct is empty");
    if (oct->box != lat->box) return fail(PSE_ERR_INVALID_ARG, "oct->box differs from lat->box");
    pse::DepositParams p;
    std::memset(&p, 0, sizeof(p));
    lattice_params(p, h_pos, lat, o);
    p.out = d_leaf_mass;
    p.bc = oct->bc;
    p.max_level = oct->max_level;
    p.leaves = oct->d_leaves;
    p.fine_map = oct->d_fine_map;
    p.fine = (int64_t)1 << oct->max_level;
    return run_deposit(p, o, oct->n_cells, h_stats, d_ws, ws_bytes, static_cast<cudaStream_t>(stream), h_pos,
                       slab_cubes);
}

int pse_build_octree_streamed(const float *h_pos, const pse_lattice *lat, int64_t slab_cubes, int32_t bc,
                              int32_t max_level, double edge_threshold_cells, pse_octree *out, void *stream)
{
    g_last_error.clear();
    const pse_deposit_opts o = default_opts();
    int rc = check_streamed(h_pos, lat, slab_cubes, o);
    if (rc != PSE_OK) return rc;
    if (!out) return fail(PSE_ERR_INVALID_ARG, "out is NULL");
    if (bc < 1 || bc > 4096) return fail(PSE_ERR_INVALID_ARG, "bc = %d out of range [1, 4096]", bc);
    if (max_level < 0 || max_level > kMaxOctreeLevel) return fail(PSE_ERR_INVALID_ARG, "max_level out of range");
    if (!(edge_threshold_cells > 0.0)) return fail(PSE_ERR_INVALID_ARG, "edge_threshold_cells must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t hb = hist_bytes(max_level);
    std::vector<unsigned> hist(hb / sizeof(unsigned), 0u);
    if (max_level > 0) {
        unsigned *d_hist = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_hist), hb, st);
        if (e != cudaSuccess) return fail(PSE_ERR_OOM, "histogram allocation failed: %s", cudaGetErrorString(e));
        e = cudaMemsetAsync(d_hist, 0, hb, st);
        pse::DepositParams p;
        std::memset(&p, 0, sizeof(p));
        lattice_params(p, h_pos, lat, o);
        p.bc = bc;
        p.max_level = max_level;
        if (e == cudaSuccess) {
            // the histograms accumulate over the slabs
            rc = stream_slabs(h_pos, p, slab_cubes, st, [&](pse::DepositParams &q, cudaStream_t ss) -> int {
                cudaError_t e2 = pse::launch_octree_hist(q, d_hist, ss);
                return e2 == cudaSuccess ? PSE_OK : cuda_fail(e2, "histogram launch");
            });
        }
        if (e == cudaSuccess && rc == PSE_OK) e = cudaMemcpyAsync(hist.data(), d_hist, hb, cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(d_hist, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (rc != PSE_OK) return rc;
        if (e != cudaSuccess) return cuda_fail(e, "octree histograms");
    }
    std::vector<int32_t> leaves;
    decide(hist, max_level, edge_threshold_cells, 0, 0, 0, 0, leaves);
    return make_octree(leaves.data(), (int64_t)(leaves.size() / 4), bc, max_level, lat->box, out);
}

// ---------------------------------------------------------------------------
// cost model
// ---------------------------------------------------------------------------
size_t pse_costmodel_bytes(void) { return pse::costmodel_bytes(); }

int pse_costmodel_set(void *d_model, const float *h_params, void *stream)
{
    g_last_error.clear();
    if (!d_model || !h_params) return fail(PSE_ERR_INVALID_ARG, "d_model and h_params must be non-NULL");
    if (reinterpret_cast<uintptr_t>(d_model) % 16 != 0) return fail(PSE_ERR_INVALID_ARG, "d_model must be 16-byte aligned");
    for (int i = 16; i < 32; ++i)
        if (!(h_params[i] > 0.0f) || !std::isfinite(h_params[i]))
            return fail(PSE_ERR_INVALID_ARG, "feature scale %d must be finite and > 0", i - 16);
    cudaError_t e = pse::costmodel_set(static_cast<pse::CostModelDev *>(d_model), h_params,
                                       static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSE_OK : cuda_fail(e, "cost model upload");
}

int pse_costmodel_get(const void *d_model, float *h_params, float *h_grad, void *stream)
{
    g_last_error.clear();
    if (!d_model) return fail(PSE_ERR_INVALID_ARG, "d_model is NULL");
    cudaError_t e = pse::costmodel_get(static_cast<const pse::CostModelDev *>(d_model), h_params, h_grad,
                                       static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSE_OK : cuda_fail(e, "cost model download");
}

namespace {
int lattice_grid_params(const float *d_pos, const pse_lattice *lat, const int64_t grid_n[3], pse::DepositParams &p)
{
    if (!d_pos) return fail(PSE_ERR_INVALID_ARG, "d_pos is NULL");
    int rc = check_lattice(lat);
    if (rc != PSE_OK) return rc;
    int64_t cells = 0;
    rc = check_grid(grid_n, cells);
    if (rc != PSE_OK) return rc;
    std::memset(&p, 0, sizeof(p));
    p.periodic = lat->periodic ? 1 : 0;
    p.pos = d_pos;
    for (int a = 0; a < 3; ++a) {
        p.n[a] = lat->n[a];
        p.nc[a] = p.periodic ? lat->n[a] : lat->n[a] - 1;
    }
    p.box = lat->box;
    p.m_tet = lat->particle_mass / 6.0;
    fill_grid(p, grid_n, lat->box);
    p.src = pse::SRC_LATTICE;
    p.n_units = p.nc[0] * p.nc[1] * p.nc[2];
    return PSE_OK;
}
}  // namespace

int pse_costmodel_features(const float *d_pos, const pse_lattice *lat, const int64_t grid_n[3], float *d_feat,
                           void *stream)
{
    g_last_error.clear();
    pse::DepositParams p;
    int rc = lattice_grid_params(d_pos, lat, grid_n, p);
    if (rc != PSE_OK) return rc;
    if (!d_feat) return fail(PSE_ERR_INVALID_ARG, "d_feat is NULL");
    if (p.n_units == 0) return PSE_OK;
    cudaError_t e = pse::launch_features(p, d_feat, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSE_OK : cuda_fail(e, "features launch");
}

int pse_tet_counts(const float *d_pos, const pse_lattice *lat, const int64_t grid_n[3], double guard_eps,
                   int32_t *d_counts, void *stream)
{
    g_last_error.clear();
    pse::DepositParams p;
    int rc = lattice_grid_params(d_pos, lat, grid_n, p);
    if (rc != PSE_OK) return rc;
    if (!d_counts) return fail(PSE_ERR_INVALID_ARG, "d_counts is NULL");
    p.kappa_max = kappa_limit(guard_eps);
    if (p.n_units == 0) return PSE_OK;
    cudaError_t e = pse::launch_tet_counts(p, d_counts, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSE_OK : cuda_fail(e, "counts launch");
}

int pse_costmodel_predict(const void *d_model, const float *d_feat, int64_t n, float *d_out, void *stream)
{
    g_last_error.clear();
    if (!d_model || (n > 0 && (!d_feat || !d_out)) || n < 0)
        return fail(PSE_ERR_INVALID_ARG, "d_model, d_feat and d_out must be non-NULL and n >= 0");
    if (n == 0) return PSE_OK;
    cudaError_t e = pse::launch_predict(static_cast<const pse::CostModelDev *>(d_model), d_feat, n, d_out,
                                        static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSE_OK : cuda_fail(e, "predict launch");
}

int pse_costmodel_train_step(void *d_model, const float *d_feat, const float *d_target, const int64_t *d_index,
                             int64_t batch, float lr, int32_t flags, double *d_loss, void *stream)
{
    g_last_error.clear();
    if (!d_model || !d_feat || !d_target || !d_loss || batch < 1)
        return fail(PSE_ERR_INVALID_ARG, "d_model, d_feat, d_target and d_loss must be non-NULL and batch >= 1");
    if (!(lr >= 0.0f) || !std::isfinite(lr)) return fail(PSE_ERR_INVALID_ARG, "lr must be finite and >= 0");
    if (flags & ~(PSE_TRAIN_FP32 | PSE_TRAIN_GRAD_ONLY)) return fail(PSE_ERR_INVALID_ARG, "unknown flags %d", flags);
    cudaError_t e = pse::launch_train_step(static_cast<pse::CostModelDev *>(d_model), d_feat, d_target, d_index, batch, lr,
                                           (flags & PSE_TRAIN_FP32) != 0, (flags & PSE_TRAIN_GRAD_ONLY) == 0, d_loss,
                                           static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PSE_OK : cuda_fail(e, "training step launch");
}

}  // extern "C"
