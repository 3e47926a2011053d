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
    ST_BIN0,  // 8 bins
    ST_NUM_U64 = ST_BIN0 + 8
};

struct Workspace {
    unsigned long long work_counter;   // dynamic work fetching
    unsigned long long stats[ST_NUM_U64];
    double mass_in;
    double mass_dropped;
    double mass_target;     // sum of m_t over processed tetrahedra (FP32 mass renormalisation)
    double mass_deposited;  // sum of every computed deposit, in the grid or dropped
    int error_code;                    // first device-side error (0 = none)
    int error_detail;
};

constexpr size_t kWorkspaceBytes = 512;
static_assert(sizeof(Workspace) <= kWorkspaceBytes, "workspace layout");

struct DepositParams {
    // tetrahedron source
    int32_t src;
    int32_t periodic;
    const float *pos;          // SRC_LATTICE / SRC_CUBE_LIST: float32 [n0*n1*n2][3]
    int64_t n[3];              // particles per axis
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
    // numerics
    float kappa_max;           // FP32 path: tetrahedra with kappa above this clip in float64
    int32_t fixup;             // accumulate mass_target / mass_deposited for the renormalisation
    // octree target (deposit onto leaf blocks)
    int32_t bc;                // cells per leaf block side
    int32_t max_level;
    const int32_t *leaves;     // [n_leaves][4]: level, ix, iy, iz
    const int32_t *fine_map;   // [F^3]: leaf of every finest-level node, x fastest
    int64_t fine;              // F = 2^max_level
    // scheduling
    int64_t n_items;
    Workspace *ws;
};

// message returned by pse_last_error() on this host thread (abi.cu)
void set_last_error(const char *msg);

// launchers (deposit.cu)
cudaError_t launch_thread_per_tet(const DepositParams &p, bool fp64, bool stats, cudaStream_t st);
cudaError_t launch_warp_coop(const DepositParams &p, bool stats, int blocks_per_sm, cudaStream_t st);
cudaError_t launch_octree_hist(const DepositParams &p, unsigned *hist, cudaStream_t st);
cudaError_t launch_octree_deposit(const DepositParams &p, bool fp64, bool thread_per_tet, bool stats,
                                  int blocks_per_sm, cudaStream_t st);
cudaError_t launch_scale(double *out, int64_t n, const Workspace *ws, cudaStream_t st);
cudaError_t launch_build_tets(const float *pos, const int64_t n[3], const int64_t nc[3], int periodic,
                              double box, int32_t *vidx, float *vol, int64_t n_tets, cudaStream_t st);

}  // namespace pse
