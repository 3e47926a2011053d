// internal.h -- launch parameters shared by the C-ABI glue (abi.cu) and the
// deposit kernels (deposit.cu).  Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace pse {

enum TetSource : int32_t { SRC_LATTICE = 0, SRC_CUBE_LIST = 1, SRC_TETS = 2 };

// device counters in the workspace (uint64 unless noted)
enum StatSlot : int32_t {
    ST_TETS = 0,
    ST_BBOX_CELLS,
    ST_INSIDE_CELLS,
    ST_PARTIAL_CLIPS,
    ST_FP64_REDOS,
    ST_DEGENERATE,
    ST_SINGLE_CELL,
    ST_INVERTED,  // tetrahedra whose orientation differs from the Lagrangian one (shell crossing)
    ST_OVERLAPPED,  // (tetrahedron, cell) pairs that received a deposit
    ST_RUNS,        // column runs clipped (warp schedules)
    ST_BIN0,  // 8 bins
    ST_NUM_U64 = ST_BIN0 + 8
};

struct Workspace {
    unsigned long long work_counter;   // dynamic work fetching (first pass)
    unsigned long long work_counter2;  // the same for the guarded pass; the two are reset together
    unsigned long long stats[ST_NUM_U64];
    double mass_in;
    double mass_dropped;
    double mass_target;     // sum of m_t over processed tetrahedra (FP32 mass renormalisation)
    double mass_deposited;  // sum of every computed deposit, in the grid or dropped
    int error_code;                    // first device-side error (0 = none)
    int error_detail;
    // binned schedule
    unsigned long long queue_count;    // split tetrahedra appended by the bin pass (may exceed q_cap)
    unsigned long long n_chunk_items;  // work items of the split tetrahedra (0 if the queue overflowed)
    int queue_overflow;                // 1: the queue was too small; every tetrahedron goes the row path
    // guarded tetrahedra the FP32 pass listed for the guarded pass (may exceed guard_cap:
    // then the list is incomplete and the guarded pass scans every tetrahedron again)
    unsigned long long guard_count;
};

constexpr size_t kWorkspaceBytes = 512;
static_assert(sizeof(Workspace) <= kWorkspaceBytes, "workspace layout");

struct DepositParams {
    // tetrahedron source
    int32_t src;
    int32_t periodic;
    const float *pos;          // SRC_LATTICE / SRC_CUBE_LIST: float32 [n0*n1*n2][3]
    int64_t n[3];              // particles per axis (slab mode: n[2] = rows held in pos)
    int32_t slab;              // 1: pos holds the particle rows of a z-slab plus one halo row; z
                               //    indices are slab-local and never wrapped (x, y still are)
    int64_t nc[3];             // cubes per axis (n for periodic, n-1 for open)
    const int64_t *cube_ids;   // SRC_CUBE_LIST
    const float *verts;        // SRC_TETS: float32 [n_tets][4][3]
    const double *tet_mass;    // SRC_TETS
    int64_t n_units;           // cubes (lattice / list) or tetrahedra (explicit)
    double box;
    double m_tet;              // lattice: particle_mass / 6
    // grid
    int64_t g[3];
    double scale_d[3];         // g_a / box
    float scale_f[3];
    double *out;
    float *vres;               // warp kernels: kMaxWarpBlocks * 4 residual blocks (see kResidualBytes)
    // numerics
    float kappa_max;           // FP32 path: tetrahedra with kappa above this clip in float64
    int32_t fixup;             // accumulate mass_target / mass_deposited for the renormalisation
    int32_t comp;              // 1: compensated FP32 accumulation, out holds (hi, lo) float pairs
    // octree target (deposit onto leaf blocks)
    int32_t bc;                // cells per leaf block side
    int32_t max_level;
    const int32_t *leaves;     // [n_leaves][4]: level, ix, iy, iz
    const int32_t *fine_map;   // [F^3]: leaf of every finest-level node, x fastest
    int64_t fine;              // F = 2^max_level
    // scheduling
    int64_t n_items;
    Workspace *ws;
    // binned schedule: tetrahedra whose bounding box has more than split_cells cells are
    // queued by the bin pass and split into work items of chunk_cells cells
    int64_t *q_tet;            // [q_cap] unit * 6 + s (lattice sources) or tetrahedron index
    int32_t *q_cells;          // [q_cap] bounding-box cell count
    int64_t *chunk_start;      // [q_cap + 1] exclusive prefix of the chunk counts
    int64_t q_cap;
    int32_t split_cells;       // bbox cells (no cost model) or predicted partial clips (cost model)
    int32_t chunk_cells;
    const struct CostModelDev *model;  // nullable: queue by the cost model's prediction
    uint32_t *qbits;           // cost model: bit t set = tetrahedron t was queued ([ceil(T/32)])
    // warp and octree schedules: ids (unit * 6 + s, or the tetrahedron index) of the guarded
    // multi-cell tetrahedra, appended by the FP32 pass; the guarded pass visits only these
    // when all of them fit (guard_cap 0: no list, every tetrahedron is scanned again)
    int64_t *guard_list;
    int64_t guard_cap;
};

// warp kernels (every schedule but thread-per-tetrahedron): the float32 rounding residuals
// of guarded records live in global memory, one [12][32] float block per warp of the
// grid, right after the Workspace header; their grids are capped at kMaxWarpBlocks blocks
// of 4 warps (persistent kernels, so the cap only bounds the parallelism).  Keeping them
// out of shared memory lets 4 blocks of 128 threads share an SM.
constexpr int kMaxWarpBlocks = 1024;
constexpr size_t kResidualBytes = (size_t)kMaxWarpBlocks * 4 * 12 * 32 * sizeof(float);

// the guarded-tetrahedron list of the warp and octree schedules, after the residual blocks
constexpr int64_t kGuardListCap = int64_t(1) << 22;
constexpr size_t kGuardListBytes = (size_t)kGuardListCap * 8;

// binned schedule: queue capacity and the bytes it takes after the guarded-tetrahedron list
constexpr int64_t kQueueCap = int64_t(1) << 21;
constexpr size_t kQueueBytes = ((size_t)kQueueCap * (8 + 4) + (size_t)(kQueueCap + 1) * 8 + 255) / 256 * 256;
// cost-model binning: one bit per tetrahedron after the queue
inline size_t qbits_bytes(int64_t n_tets) { return ((size_t)(n_tets + 31) / 32 * 4 + 255) / 256 * 256; }

// message returned by pse_last_error() on this host thread (abi.cu)
void set_last_error(const char *msg);

// launchers (deposit.cu)
cudaError_t launch_thread_per_tet(const DepositParams &p, bool fp64, bool stats, cudaStream_t st);
cudaError_t launch_warp_coop(const DepositParams &p, bool stats, int blocks_per_sm, cudaStream_t st);
cudaError_t launch_binned(const DepositParams &p, bool stats, int blocks_per_sm, cudaStream_t st);
cudaError_t launch_warp_per_tet(const DepositParams &p, bool stats, cudaStream_t st);

// cost model (costmodel.cu)
struct CostModelDev;
size_t costmodel_bytes();
cudaError_t launch_tet_counts(const DepositParams &p, int32_t *counts, cudaStream_t st);
cudaError_t launch_features(const DepositParams &p, float *feat, cudaStream_t st);
cudaError_t launch_predict(const CostModelDev *m, const float *feat, int64_t n, float *out, cudaStream_t st);
cudaError_t launch_refresh(CostModelDev *m, bool bump, cudaStream_t st);
cudaError_t launch_train_step(CostModelDev *m, const float *feat, const float *target, const int64_t *index,
                              int64_t batch, float lr, bool fp32, bool update, double *loss, cudaStream_t st);
cudaError_t costmodel_set(CostModelDev *m, const float *h_params, cudaStream_t st);
cudaError_t costmodel_get(const CostModelDev *m, float *h_params, float *h_grad, cudaStream_t st);
cudaError_t launch_octree_hist(const DepositParams &p, unsigned *hist, cudaStream_t st);
cudaError_t launch_octree_deposit(const DepositParams &p, bool fp64, bool thread_per_tet, bool stats,
                                  int blocks_per_sm, cudaStream_t st);
// the warp-cooperative kernel with compensated FP32 accumulation (deposit_comp.cu)
cudaError_t launch_coop_comp(const DepositParams &p, bool stats, int blocks_per_sm, bool binned, int64_t max_items,
                             cudaStream_t st);
// end of an FP32 deposit: FP32 pairs to FP64 (comp) and / or the mass renormalisation (scale)
cudaError_t launch_finish(double *out, int64_t n, const Workspace *ws, bool comp, bool scale, cudaStream_t st);
cudaError_t launch_subblock_boxes(const float *pos, const int64_t n[3], int s, double box, double *boxes,
                                  cudaStream_t st);
cudaError_t launch_node_counts(const double *boxes, int64_t nb, const int32_t *nodes, int64_t n_nodes, double box,
                               double *counts, cudaStream_t st);
cudaError_t launch_octree_restrict(const int32_t *fine_map, const int32_t *leaves, int max_level, int bc,
                                   const double *leaf_mass, double *pyramid, cudaStream_t st);
cudaError_t launch_build_tets(const float *pos, const int64_t n[3], const int64_t nc[3], int periodic,
                              double box, int32_t *vidx, float *vol, int64_t n_tets, cudaStream_t st);

}  // namespace pse
