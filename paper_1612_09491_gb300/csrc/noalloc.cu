// noalloc.cu -- an octree-build entry point for callers that cannot allocate memory.
//
// Some callers cannot call cudaMalloc: plugins inside a host application that owns the
// device allocator, or real-time loops that must not block on the allocator.
// pse_build_octree_leaves_noalloc
// builds the same octree leaf list as pse_build_octree_from_tet_sizes, but it
// allocates nothing: its scratch (the work counters and the per-level size
// histograms) lives in a file-scope device array of kScratchBytes, and the leaf
// list is written into a device buffer the caller provides.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/pse.h"
#include "internal.h"

namespace {

// 256 KB: the work counters plus the histograms of levels 0..3 (max_level <= 4).
constexpr size_t kScratchBytes = 256 * 1024;
constexpr int kMaxLevelNoAlloc = 4;
constexpr int kMaxDevices = 64;

// One copy of this array exists on every device that loads the library; it stays
// resident until the process exits.  Host code must not pass its name to a kernel:
// in host code it is only a stand-in, its device address comes from
// cudaGetSymbolAddress (resolved once per device below).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
void *g_ctx[kMaxDevices] = {};  // the context the cached address belongs to

// The current driver context (nullptr if it cannot be read): a device reset creates a new
// one, and with it a new copy of g_scratch at another address.
void *current_context()
{
    using GetCurrent = int (*)(void **);
    static GetCurrent fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<GetCurrent>(f);
    });
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

// The first histogram bin whose lower edge 10^(-3 + 6 b / 64) cells is not below the
// threshold, computed on the host exactly as the allocating build computes the edges: a
// node is refined when its lower-median bin lies below this cutoff.
int refine_cutoff(double threshold)
{
    int b = 0;
    while (b < 64 && std::pow(10.0, -3.0 + 6.0 * b / 64.0) < threshold) ++b;
    return b;
}


size_t hist_bytes_of(int max_level)
{
    size_t n = 0;
    for (int l = 0; l < max_level; ++l) n += ((size_t)1 << (3 * l)) * 64;
    return (n * sizeof(unsigned) + 255) / 256 * 256;
}

// Depth-first traversal of the refinement decisions (lower-median bin edge below the
// threshold), writing leaves (level, ix, iy, iz) into out; *count receives the number
// of leaves even when it exceeds cap.  One thread: the tree has at most 8^4 leaves.
__global__ void k_octree_decide(const unsigned *__restrict__ hist, int max_level, int cutoff,
                                int32_t *__restrict__ out, long long cap, long long *__restrict__ count)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int lv[8], cx[8], cy[8], cz[8], child[8];
    int sp = 0;
    lv[0] = 0; cx[0] = 0; cy[0] = 0; cz[0] = 0; child[0] = -1;
    long long nleaf = 0;
    while (sp >= 0) {
        if (child[sp] < 0) {  // first visit: decide
            const int level = lv[sp];
            bool refine = false;
            if (level < max_level) {
                long long off = 0;
                for (int l = 0; l < level; ++l) off += ((long long)1 << (3 * l)) * 64;
                const long long nn = (long long)1 << level;
                const unsigned *h = hist + off + (cx[sp] + nn * (cy[sp] + nn * cz[sp])) * 64;
                unsigned long long c = 0;
                for (int b = 0; b < 64; ++b) c += h[b];
                if (c > 0) {
                    const unsigned long long k = (c - 1) / 2;
                    unsigned long long cum = 0;
                    int bin = 63;
                    for (int b = 0; b < 64; ++b) {
                        cum += h[b];
                        if (cum > k) { bin = b; break; }
                    }
                    refine = bin < cutoff;
                }
            }
            if (!refine) {
                if (nleaf < cap) {
                    out[4 * nleaf] = level;
                    out[4 * nleaf + 1] = cx[sp];
                    out[4 * nleaf + 2] = cy[sp];
                    out[4 * nleaf + 3] = cz[sp];
                }
                ++nleaf;
                --sp;
                continue;
            }
            child[sp] = 0;
        }
        if (child[sp] == 8) {
            --sp;
            continue;
        }
        const int c = child[sp]++;
        lv[sp + 1] = lv[sp] + 1;
        cx[sp + 1] = 2 * cx[sp] + (c & 1);
        cy[sp + 1] = 2 * cy[sp] + ((c >> 1) & 1);
        cz[sp + 1] = 2 * cz[sp] + (c >> 2);
        child[sp + 1] = -1;
        ++sp;
    }
    *count = nleaf;
}

int fail(int code, const char *msg)
{
    pse::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" {

int pse_build_octree_leaves_noalloc(const float *d_pos, const pse_lattice *lat, int32_t bc, int32_t max_level,
                                    double edge_threshold_cells, int32_t *d_leaves, int64_t cap,
                                    int64_t *d_n_leaves, void *stream)
{
    pse::set_last_error("");
    if (!d_pos || !lat || !d_leaves || !d_n_leaves || cap < 1)
        return fail(PSE_ERR_INVALID_ARG, "d_pos, lat, d_leaves and d_n_leaves must be non-NULL and cap >= 1");
    for (int a = 0; a < 3; ++a)
        if (lat->n[a] < 2) return fail(PSE_ERR_INVALID_ARG, "lat->n must be >= 2 on every axis");
    if (!lat->periodic) return fail(PSE_ERR_UNSUPPORTED, "the octree covers a periodic box");
    if (!(lat->box > 0.0) || !std::isfinite(lat->box)) return fail(PSE_ERR_INVALID_ARG, "lat->box must be > 0");
    if (bc < 1 || bc > 4096) return fail(PSE_ERR_INVALID_ARG, "bc out of range [1, 4096]");
    if (!(edge_threshold_cells > 0.0)) return fail(PSE_ERR_INVALID_ARG, "edge_threshold_cells must be > 0");
    if (max_level < 0) return fail(PSE_ERR_INVALID_ARG, "max_level must be >= 0");
    const size_t need = pse::kWorkspaceBytes + hist_bytes_of(max_level);
    if (max_level > kMaxLevelNoAlloc || need > kScratchBytes) {
        char m[256];
        std::snprintf(m, sizeof(m),
                      "max_level %d needs %zu bytes of scratch; this entry point has a fixed %zu-byte scratch "
                      "array (max_level <= %d); use pse_build_octree_from_tet_sizes",
                      max_level, need, kScratchBytes, kMaxLevelNoAlloc);
        return fail(PSE_ERR_INVALID_ARG, m);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PSE_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PSE_ERR_UNSUPPORTED, "device index beyond the supported range");
    void *base = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_mu);
        void *ctx = current_context();
        if (!g_addr[dev] || ctx != g_ctx[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) return fail(PSE_ERR_CUDA, cudaGetErrorString(e));
            g_addr[dev] = p;
            g_ctx[dev] = ctx;
        }
        base = g_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: clear what must start at zero
    e = cudaMemsetAsync(base, 0, need, st);
    if (e != cudaSuccess) return fail(PSE_ERR_CUDA, cudaGetErrorString(e));
    unsigned *hist = reinterpret_cast<unsigned *>(static_cast<unsigned char *>(base) + pse::kWorkspaceBytes);
    if (max_level > 0) {
        pse::DepositParams p;
        std::memset(&p, 0, sizeof(p));
        p.src = pse::SRC_LATTICE;
        p.periodic = 1;
        p.pos = d_pos;
        for (int a = 0; a < 3; ++a) {
            p.n[a] = lat->n[a];
            p.nc[a] = lat->n[a];
        }
        p.n_units = p.nc[0] * p.nc[1] * p.nc[2];
        p.box = lat->box;
        p.m_tet = lat->particle_mass / 6.0;
        p.bc = bc;
        p.max_level = max_level;
        p.ws = static_cast<pse::Workspace *>(base);
        e = pse::launch_octree_hist(p, hist, st);
        if (e != cudaSuccess) return fail(PSE_ERR_CUDA, cudaGetErrorString(e));
    }
    k_octree_decide<<<1, 32, 0, st>>>(hist, max_level, refine_cutoff(edge_threshold_cells), d_leaves, (long long)cap,
                                      reinterpret_cast<long long *>(d_n_leaves));
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PSE_ERR_CUDA, cudaGetErrorString(e));
    return PSE_OK;
}

}  // extern "C"
