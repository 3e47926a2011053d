/*
 * pse.h -- C ABI of the GB300 (sm_103a) exact tetrahedron-deposit library.
 *
 * The phase-space-element density of Kaehler (arXiv:1612.09491), Sec. 2, Eq. 1:
 * tracer particles sit on a Lagrangian lattice; each Lagrangian cube of 8
 * neighbouring particles is split into 6 tetrahedra of mass m_p/6, and the
 * density at x is m * sum_i 1/V_i(x) over the tetrahedra covering x.  Integrated
 * over a deposit cell C that is
 *
 *     M[C] = sum_t (m_t / |V_t|) * vol(T_t  intersect  C),
 *
 * which every deposit entry point below computes exactly (up to rounding):
 * each tetrahedron is clipped against every cell it overlaps (Sec. 6.3).
 *
 * Conventions shared by all entry points
 * --------------------------------------
 *  - Pointers prefixed d_ are DEVICE memory owned by the caller; h_ are HOST
 *    memory owned by the caller.  The library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued asynchronously on it.  An entry point that
 *    returns host-side results (h_stats, h_n_tets, octree metadata)
 *    synchronises `stream` before returning; the others do not.
 *  - Positions: float32 [n0*n1*n2][3], particle (i,j,k) at flat index
 *    i + n0*(j + n1*k) (x fastest: the particle IDs' Lagrangian order, Sec. 3).
 *  - Tessellation: the Kuhn split of each Lagrangian cube around its 000-111
 *    diagonal (the paper cuts each cube into six tetrahedra without fixing which, Sec. 2):
 *    tetrahedron s (0..5) of cube (i,j,k) visits corners 000, e_a, e_a+e_b, 111
 *    for the axis permutation (a,b,c) = xyz, xzy, yxz, yzx, zxy, zyx.
 *    Its id is 6*cube + s, with cube = i + n0*(j + n1*k) (periodic lattices)
 *    or i + (n0-1)*(j + (n1-1)*k) (open lattices).
 *  - Periodic boxes: every cube corner is unwrapped to the periodic image
 *    nearest to corner 000; deposit cells are folded modulo the grid size.
 *  - Grids: cubic box [0, box)^3 split into g0*g1*g2 cells; cell (ix,iy,iz) covers
 *    [ix*h0,(ix+1)*h0) x ... with h_a = box/g_a; cell masses are float64 at flat
 *    index ix + g0*(iy + g1*iz).  Density = mass / (h0*h1*h2).
 *  - A tetrahedron whose float64 volume is exactly zero deposits all of its
 *    mass into the cell that contains its vertex centroid.
 *  - Return value: PSE_OK (0) or a negative PSE_ERR_* code; the message of the
 *    last failure on the calling host thread is pse_last_error().
 *  - Calls are safe to run concurrently when they use distinct streams, output
 *    buffers and workspaces.
 */
#ifndef PSE_H_
#define PSE_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PSE_API __attribute__((visibility("default")))
#else
#define PSE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define PSE_ABI_VERSION 2

#define PSE_OK 0
#define PSE_ERR_INVALID_ARG -1 /* a null pointer, a bad size or an inconsistent option */
#define PSE_ERR_CUDA -2        /* a CUDA runtime call failed (message in pse_last_error) */
#define PSE_ERR_OOM -3         /* the library could not allocate device or host memory */
#define PSE_ERR_TIMEOUT -4     /* a bounded device-side wait ran out (spin_limit) */
#define PSE_ERR_UNSUPPORTED -5 /* a valid request the library does not implement */
#define PSE_ERR_WORKSPACE -6   /* ws_bytes smaller than pse_workspace_size() */
#define PSE_ERR_DEVICE -7      /* a device-side check failed (e.g. a tetrahedron wider than box/2) */

/* precision (pse_deposit_opts.precision) */
#define PSE_FP64_PLAIN 0   /* every step in float64 */
#define PSE_FP32_FP64ACC 1 /* float32 clip; float64 clip of guarded tetrahedra; float64 accumulation */
#define PSE_FP32_COMPENSATED 2 /* the float32 clip of PSE_FP32_FP64ACC; each cell sums its deposits as a
                                  float32 pair (hi, lo) with an error-free two-sum on every add, held in
                                  the cell's own 8 output bytes and turned into float64 hi + lo at the
                                  end of the call (needs accumulate = 0) */

/* schedule (pse_deposit_opts.schedule) */
#define PSE_THREAD_PER_TET 0    /* one thread per tetrahedron (the plain baseline) */
#define PSE_WARP_COOPERATIVE 1  /* one warp per batch of tetrahedra, lanes over (tet, cell) pairs */
#define PSE_BINNED_PERSISTENT 2 /* size-binned persistent kernel: a bin pass queues every tetrahedron whose
                                   bounding box exceeds pse_tuning.split_cells; one persistent kernel
                                   takes work items (pieces of the queued tetrahedra first, then rows of
                                   cubes) from one atomic counter.  FP32 path, uniform grids. */
#define PSE_WARP_PER_TET 3      /* the paper's GPU kernel design (Sec. 6.2) on this GPU, kept as a baseline:
                                   one warp per tetrahedron, lanes striding over its bounding-box cells,
                                   partial cells buffered in shared memory and clipped 32 at a time.  FP32
                                   path, uniform grids (octree deposits use the warp-cooperative kernel). */

/* operation ids for pse_workspace_size */
#define PSE_OP_DEPOSIT_UNIFORM 1
#define PSE_OP_DEPOSIT_OCTREE 2
#define PSE_OP_BUILD_OCTREE 3
#define PSE_OP_DEPOSIT_TETS 4

typedef struct pse_lattice {
    int64_t n[3];         /* particles per axis (>= 2 each) */
    double box;           /* side of the cubic box, > 0 */
    int32_t periodic;     /* 1: periodic lattice and grid; 0: open (cells outside the grid are dropped) */
    int32_t reserved;
    double particle_mass; /* m_p; every tetrahedron carries m_p/6 */
} pse_lattice;

typedef struct pse_deposit_opts {
    int32_t precision;       /* PSE_FP64_PLAIN, PSE_FP32_FP64ACC or PSE_FP32_COMPENSATED */
    int32_t schedule;        /* PSE_THREAD_PER_TET, PSE_WARP_COOPERATIVE or PSE_BINNED_PERSISTENT */
    const void *cost_model;  /* nullable device cost model (pse_costmodel_*): the binned schedule then splits
                                the tetrahedra whose predicted partial clips exceed split_cells, instead
                                of those whose bounding box exceeds split_cells cells (lattice deposits
                                need pse_workspace_size(PSE_OP_DEPOSIT_UNIFORM, lat, opts) bytes) */
    const void *tuning;      /* nullable host pointer to a pse_tuning block; NULL = built-in defaults */
    double guard_eps;        /* FP32 clip guard: clip a tetrahedron in float64, from its exact vertices,
                                when the estimated relative error of its FP32 clip exceeds guard_eps
                                (<=0: default) */
    int64_t spin_limit;      /* iteration bound of every device-side wait (<=0: default) */
    int32_t accumulate;      /* 0: the call overwrites the output; 1: it adds to it */
    int32_t mass_fixup;      /* FP32 path with accumulate = 0: 1 rescales the call's output by
                                sum(m_t) / sum(computed deposits), so total mass is conserved to float64
                                rounding (every cell moves by the same relative ~1e-8) */
    const int64_t *d_cube_ids; /* NULL: every cube; else deposit only these Lagrangian cubes (device int64
                                  [n_cube_ids], each in [0, number of cubes); n_cube_ids may be 0).
                                  Accuracy of such subset deposits with the FP32 clip: a cell that
                                  holds only a sliver of one tetrahedron carries the clip's absolute
                                  error (about 1e-7 of a whole cell at that tetrahedron's density),
                                  so relative to its own small mass it is good to about 1e-4 */
    int64_t n_cube_ids;
} pse_deposit_opts;

typedef struct pse_deposit_stats {
    uint64_t tets;             /* tetrahedra processed */
    uint64_t bbox_cells;       /* (tetrahedron, cell) pairs inside bounding boxes */
    uint64_t inside_cells;     /* pairs classified "cell inside tetrahedron" */
    uint64_t partial_clips;    /* pairs that went through the exact clip */
    uint64_t fp64_redos;       /* partial cells of guarded tetrahedra, clipped in float64 (the warp
                                  schedules clip them by column runs in a pass of their own; the
                                  others re-clip each such cell in float64) */
    uint64_t degenerate_tets;  /* zero-volume tetrahedra (centroid rule) */
    uint64_t single_cell_tets; /* tetrahedra whose bounding box is one cell */
    uint64_t bin_counts[8];    /* binned schedule: tetrahedra per size bin */
    double mass_in;            /* sum of m_t over the processed tetrahedra */
    double mass_dropped;       /* open grids: mass that fell outside the grid */
    uint64_t inverted_tets;    /* lattice tetrahedra turned inside out by shell crossing: signed volume of
                                  the other sign than in the Lagrangian lattice (they deposit positive
                                  mass, Sec. 2); explicit tetrahedra: negative signed volume */
    uint64_t overlapped_cells; /* (tetrahedron, cell) pairs that received a deposit (overlap > 0) */
    uint64_t column_runs;      /* warp schedules: runs of cells along a tetrahedron's divergence axis that
                                  one column clip served (the clip work unit; see partial_clips) */
    double mass_out;           /* mass this call wrote into the output: its in-grid deposits, after the
                                  renormalisation when that applied (equals mass_in - mass_dropped to
                                  float64 rounding when it did) */
} pse_deposit_stats;

/*
 * Adaptive deposit grid (Sec. 4): an octree over the periodic box [0, box)^3 whose
 * leaves each carry a block of bc^3 cells (every leaf patch has the same cell count).
 * A node at level l has side box/2^l; its leaf block has cells of side box/(bc 2^l).
 * Leaves are listed depth first, children in the order c = cx + 2 cy + 4 cz.
 * All pointers are owned by the library: release them with pse_free_octree().
 */
typedef struct pse_octree {
    int32_t bc;             /* cells per leaf block side */
    int32_t max_level;      /* deepest level that may hold leaves (<= 10) */
    int64_t n_leaves;
    double box;
    int32_t *d_leaves;      /* device [n_leaves][4]: level, ix, iy, iz of each leaf */
    int32_t *d_fine_map;    /* device [8^max_level]: leaf of every finest-level node, x fastest */
    int32_t *h_leaves;      /* host copy of d_leaves */
    int64_t n_cells;        /* n_leaves * bc^3: length of a leaf-mass array; leaf l's block starts at
                               l * bc^3 and its cells are x fastest */
} pse_octree;

typedef struct pse_tuning {
    int32_t blocks_per_sm;   /* resident 128-thread blocks per SM of the warp-cooperative kernels: 2 (up
                                to 255 registers per thread), 3 (170) or 4 (128); <= 0: 4 */
    int32_t warps_per_block; /* reserved (8) */
    int32_t split_cells;     /* binned schedule: a tetrahedron whose bounding box has more cells than
                                this is split across warps; <= 0: default 1024 */
    int32_t chunk_cells;     /* binned schedule: bounding-box cells per split work item; <= 0: default 512 */
    int32_t use_graph;       /* with a caller workspace and h_stats NULL: 1 = replay the call's launch
                                sequence as a CUDA graph (captured once per distinct argument set) */
    int32_t guard_list_cap;  /* warp and octree schedules: the FP32 pass lists the guarded tetrahedra
                                (at most 4,194,304 per call, or per slab when streamed) so that the
                                guarded pass visits only them; when more are guarded it scans every
                                tetrahedron again.  0: the full list; > 0: a smaller capacity; < 0: no
                                list (always scan again).  Results are the same either way. */
    int32_t reserved[4];
} pse_tuning;

/*
 * Build the tetrahedra of the Lagrangian tessellation (Sec. 2: 6 tetrahedra per
 * Lagrangian cube) from a lattice of particle positions.
 *   d_pos       float32 [n0*n1*n2][3] device, read only.
 *   d_tet_vidx  nullable int32 [T][4] device: particle indices of vertices v0..v3.
 *   d_tet_vol   nullable float32 [T] device: signed volume (box units^3, periodic unwrap applied).
 *   h_n_tets    nullable host: receives T = 6 * number of cubes.
 * Synchronises `stream` only if h_n_tets is non-null.  T must fit int32 when d_tet_vidx is
 * requested (PSE_ERR_INVALID_ARG otherwise).
 */
PSE_API int pse_build_tets_from_lagrangian_grid(const float *d_pos, const pse_lattice *lat, int32_t *d_tet_vidx,
                                        float *d_tet_vol, int64_t *h_n_tets, void *stream);

/*
 * Deposit the whole tessellation (or the cubes in opts->d_cube_ids) onto a uniform
 * grid: d_cell_mass[ix + g0*(iy + g1*iz)] (+)= sum_t m_t/|V_t| vol(T_t ∩ C)  (Eq. 1
 * over cells; the clip is Sec. 6.3's operation, computed here by half-space clipping
 * and the divergence theorem).
 *   grid_n      host int64[3], cells per axis (>= 1 each).
 *   d_cell_mass float64 [g0*g1*g2] device, written (accumulate = 0) or added to.
 *   opts        nullable: NULL = PSE_FP32_FP64ACC, PSE_WARP_COOPERATIVE, overwrite, mass fix-up on.
 *   h_stats     nullable host: filled with counters; when non-null the call synchronises.
 *   d_ws        device workspace (16-byte aligned) of ws_bytes >= pse_workspace_size(
 *               PSE_OP_DEPOSIT_UNIFORM, lat, opts); NULL with ws_bytes = 0 makes the library
 *               allocate it stream-ordered for this call.
 * Device-side failures (a bad cube id, non-finite coordinates, a bounding box beyond
 * the int32 cell range) are recorded in the workspace and returned as PSE_ERR_DEVICE
 * by calls that pass h_stats; calls without h_stats do not synchronise and do not
 * report them.
 */
PSE_API int pse_deposit_uniform(const float *d_pos, const pse_lattice *lat, const int64_t grid_n[3],
                        double *d_cell_mass, const pse_deposit_opts *opts, pse_deposit_stats *h_stats,
                        void *d_ws, size_t ws_bytes, void *stream);

/*
 * Deposit explicit tetrahedra (test and tooling entry point; the same kernels as
 * pse_deposit_uniform with a different tetrahedron source).
 *   d_verts    float32 [n_tets][4][3] device, box units, already unwrapped.
 *   d_tet_mass float64 [n_tets] device: m_t of each tetrahedron.
 *   box, periodic, grid_n, d_cell_mass, opts, h_stats, d_ws, ws_bytes, stream: as above
 *   (opts->d_cube_ids must be NULL).
 */
PSE_API int pse_deposit_tets(const float *d_verts, const double *d_tet_mass, int64_t n_tets, double box,
                     int32_t periodic, const int64_t grid_n[3], double *d_cell_mass,
                     const pse_deposit_opts *opts, pse_deposit_stats *h_stats, void *d_ws,
                     size_t ws_bytes, void *stream);

/*
 * An octree from an explicit leaf list (host int32 [n_leaves][4]: level, ix, iy, iz).
 * The leaves must tile the box exactly (PSE_ERR_INVALID_ARG otherwise).  Allocates
 * and fills *out (synchronous; free with pse_free_octree).
 */
PSE_API int pse_octree_from_leaves(const int32_t *h_leaves, int64_t n_leaves, int32_t bc, int32_t max_level,
                                   double box, pse_octree *out);

/*
 * Build the octree from the tetrahedra's sizes (Sec. 4 builds it from tetrahedron
 * counts; this rule refines where tetrahedra are small): a node at level l is refined
 * iff l < max_level and the median, over the tetrahedra whose vertex centroid lies in
 * the node, of the tetrahedron's mean edge length is below edge_threshold_cells times
 * the node's cell size box/(bc 2^l).  Nodes without tetrahedra are leaves.  The median
 * is taken from a 64-bin histogram of log10(edge / cell size) over [-3, 3): the lower
 * edge of the bin holding the lower median.  Periodic lattices only.
 *   d_ws: ws_bytes >= pse_workspace_size(PSE_OP_BUILD_OCTREE, lat, &max_level) (int32), or NULL/0.
 * Synchronises `stream`; allocates *out (free with pse_free_octree).
 */
PSE_API int pse_build_octree_from_tet_sizes(const float *d_pos, const pse_lattice *lat, int32_t bc,
                                            int32_t max_level, double edge_threshold_cells, pse_octree *out,
                                            void *d_ws, size_t ws_bytes, void *stream);

/*
 * Deposit the tessellation (or opts->d_cube_ids) onto the leaf blocks of `oct`:
 * d_leaf_mass[l * bc^3 + cx + bc (cy + bc cz)] (+)= sum_t m_t/|V_t| vol(T_t ∩ C) for cell
 * (cx, cy, cz) of leaf l.  Periodic lattices only.  Other arguments as
 * pse_deposit_uniform (d_leaf_mass has oct->n_cells float64 entries), except the
 * workspace: ws_bytes >= pse_workspace_size(PSE_OP_DEPOSIT_OCTREE, lat, opts).
 */
PSE_API int pse_deposit_octree(const float *d_pos, const pse_lattice *lat, const pse_octree *oct,
                               double *d_leaf_mass, const pse_deposit_opts *opts, pse_deposit_stats *h_stats,
                               void *d_ws, size_t ws_bytes, void *stream);

/* Release what pse_octree_from_leaves / pse_build_octree_from_tet_sizes allocated; zeroes *oct. */
PSE_API void pse_free_octree(pse_octree *oct);

/*
 * The leaf list of pse_build_octree_from_tet_sizes, for callers that cannot allocate
 * memory (plugins whose host application owns the device allocator, real-time loops that
 * must not wait on it).  The paper has no counterpart: this is an
 * interface variant, not part of the method.  It allocates nothing and does not
 * synchronise: its scratch (work counters and the size histograms) is a fixed 256 KB
 * device array inside the library -- every GPU that loads the library holds it until
 * the process exits -- and its result goes to caller buffers.
 *   d_leaves    device int32 [cap][4]: leaves (level, ix, iy, iz) in the order of
 *               pse_build_octree_from_tet_sizes; at most cap are written.
 *   d_n_leaves  device int64 [1]: the number of leaves (may exceed cap: then call again).
 *   max_level   <= 4 (the fixed scratch holds the histograms of levels 0..3); a larger
 *               value returns PSE_ERR_INVALID_ARG without touching the device.
 * The first call on each device (and the first after a device reset, which creates a new
 * context and a new copy of the array) resolves the array's device address with that
 * device current; make that call outside stream capture.  The refinement threshold is
 * turned into a histogram-bin cutoff on the host exactly as the allocating build turns
 * it, so thresholds on a bin edge give the same leaves.  Every call reuses the same
 * array (it is cleared at the start of each call): calls that overlap on the GPU, on
 * any stream, race and give wrong results.
 */
PSE_API int pse_build_octree_leaves_noalloc(const float *d_pos, const pse_lattice *lat, int32_t bc,
                                            int32_t max_level, double edge_threshold_cells, int32_t *d_leaves,
                                            int64_t cap, int64_t *d_n_leaves, void *stream);

/*
 * The paper's own refinement criterion (Sec. 4), as an alternative to the size rule of
 * pse_build_octree_from_tet_sizes: the Lagrangian lattice is cut into subblocks of
 * subblock^3 cubes (the paper uses 8^3); the axis-aligned bounding box of each subblock's
 * particles stands for its tetrahedra, assumed spread evenly over the box.  A node is
 * refined while the estimated number of tetrahedra overlapping it,
 *     sum over subblocks of 6 * cubes * vol(box ∩ node) / vol(box)   (periodic images),
 * exceeds count_threshold and its level is below max_level (the minimal node size).
 * Leaves and output as for pse_build_octree_from_tet_sizes.  Synchronous.
 */
PSE_API int pse_build_octree_count(const float *d_pos, const pse_lattice *lat, int32_t bc, int32_t max_level,
                                   double count_threshold, int32_t subblock, pse_octree *out, void *stream);

/*
 * Coarse node masses for multi-resolution use (the paper keeps the masses of the inner
 * nodes of its adaptive grid for rendering at several resolutions, Sec. 8): every node of
 * levels 0 .. max_level-1 gets its own bc^3 block of cell masses.
 *   d_leaf_mass  device float64 [n_leaves * bc^3], as written by pse_deposit_octree.
 *   d_pyramid    device float64 [P * bc^3], P = sum_{l < max_level} 8^l; node (l, x, y, z)
 *                is row (8^0 + ... + 8^(l-1)) + x + 2^l (y + 2^l z), cells x fastest.
 *                A leaf's row is its block; an inner node's cell holds the sum of the 8
 *                cells of the level below that it covers; a node below a leaf is 0.
 * For every node of the tree the row equals the deposit on the uniform grid of that
 * level restricted to the node.  Asynchronous.
 */
PSE_API int pse_octree_restrict(const pse_octree *oct, const double *d_leaf_mass, double *d_pyramid, void *stream);

/*
 * Slab streaming (periodic lattices whose positions live in host memory): the lattice
 * is deposited in z-slabs of slab_cubes cube layers.  Each slab's slab_cubes + 1 particle
 * rows (the last one a halo row, taken modulo n2) are copied into one of two device
 * buffers while the previous slab is deposited (double buffering on a second stream).
 * The result equals the one-shot deposit of the whole lattice (same cube set).
 *   h_pos       host float32 [n0*n1*n2][3]; pinned memory lets the copies overlap the
 *               kernels (pageable memory works, without overlap).
 *   slab_cubes  cube layers per slab (>= 1).
 * The other arguments are those of pse_deposit_uniform / pse_deposit_octree
 * (opts->d_cube_ids must be NULL and use_graph 0).  The statistics and the FP32 mass
 * renormalisation cover the whole lattice.  The calls allocate two slab buffers
 * (stream-ordered) and do not synchronise unless h_stats is given.
 */
PSE_API int pse_deposit_uniform_streamed(const float *h_pos, const pse_lattice *lat, int64_t slab_cubes,
                                         const int64_t grid_n[3], double *d_cell_mass, const pse_deposit_opts *opts,
                                         pse_deposit_stats *h_stats, void *d_ws, size_t ws_bytes, void *stream);
PSE_API int pse_deposit_octree_streamed(const float *h_pos, const pse_lattice *lat, int64_t slab_cubes,
                                        const pse_octree *oct, double *d_leaf_mass, const pse_deposit_opts *opts,
                                        pse_deposit_stats *h_stats, void *d_ws, size_t ws_bytes, void *stream);
/* pse_build_octree_from_tet_sizes over a streamed lattice (histograms accumulated slab
 * by slab).  Synchronous, like the one-shot build. */
PSE_API int pse_build_octree_streamed(const float *h_pos, const pse_lattice *lat, int64_t slab_cubes, int32_t bc,
                                      int32_t max_level, double edge_threshold_cells, pse_octree *out, void *stream);

/*
 * Learned cost model of the binned schedule (the paper has none: it balances work by
 * estimated cost per tetrahedron, Sec. 5, and notes the spread of work, Sec. 6.2).
 * A model is a caller-owned, 16-byte aligned device buffer of pse_costmodel_bytes().
 * Its parameters are a float32 vector of PSE_COSTMODEL_NPARAMS values:
 *   mu[16], sigma[16]        feature standardisation z = (f - mu) / sigma
 *   W1[64][16], b1[64]       ReLU layer
 *   W2[64][64], b2[64]       ReLU layer
 *   W3[2][64], b3[2]         outputs: log(1 + overlapped cells), log(1 + partial clips)
 * The forward pass rounds z, the weights and the hidden activations to bfloat16 and
 * accumulates in float32 (tensor cores for prediction).  The model only decides which
 * tetrahedra the binned schedule splits; deposited values never depend on it.
 */
#define PSE_COSTMODEL_NFEAT 16
#define PSE_COSTMODEL_NPARAMS 5410
#define PSE_TRAIN_FP32 1      /* train step in float32 without bfloat16 rounding (gradient checks) */
#define PSE_TRAIN_GRAD_ONLY 2 /* compute the gradient (readable with pse_costmodel_get) but do not update */

PSE_API size_t pse_costmodel_bytes(void);
/* Upload parameters (host float32 [PSE_COSTMODEL_NPARAMS]); resets the optimiser state.
 * Synchronises `stream`.  PSE_ERR_INVALID_ARG if a sigma is not finite and > 0. */
PSE_API int pse_costmodel_set(void *d_model, const float *h_params, void *stream);
/* Download parameters and/or the last training step's gradient (host float32
 * [PSE_COSTMODEL_NPARAMS] each, nullable; the gradient of mu and sigma is 0).  Synchronises. */
PSE_API int pse_costmodel_get(const void *d_model, float *h_params, float *h_grad, void *stream);
/* Features of every lattice tetrahedron (id 6 * cube + s) on the grid grid_n:
 * d_feat float32 [T][16], T = 6 * cubes.  The features are, in grid units: bounding-box
 * extent (3), offset of its low corner in its cell (3), log2 bounding-box cells,
 * log2 volume, log2 surface area, longest / shortest / mean edge, log2 max(kappa, 1),
 * volume over bounding-box volume, log2 longest over shortest edge, cube root of the
 * volume over the mean edge.  Asynchronous. */
PSE_API int pse_costmodel_features(const float *d_pos, const pse_lattice *lat, const int64_t grid_n[3],
                                   float *d_feat, void *stream);
/* Labels from the exact deposit: d_counts int32 [T][2] = (cells whose overlap exceeds
 * 1e-6 of the cell volume, partial clips) of every lattice tetrahedron on grid grid_n, from the same
 * classification and FP32 clip (FP64 guard at guard_eps, <= 0: default) as
 * pse_deposit_uniform.  Nothing is deposited.  Asynchronous. */
PSE_API int pse_tet_counts(const float *d_pos, const pse_lattice *lat, const int64_t grid_n[3], double guard_eps,
                           int32_t *d_counts, void *stream);
/* Predictions d_out float32 [n][2] for features d_feat float32 [n][16].  Asynchronous. */
PSE_API int pse_costmodel_predict(const void *d_model, const float *d_feat, int64_t n, float *d_out, void *stream);
/* One Adam step (lr; beta 0.9 / 0.999, eps 1e-8) on the mean squared error
 * (1 / 2B) sum (y - target)^2 of a batch of B rows of d_feat float32 [*][16] and
 * d_target float32 [*][2]: rows d_index[0..B) (device int64, nullable = rows 0..B).
 * d_loss (device float64 [1]) receives the loss before the update.  flags:
 * PSE_TRAIN_FP32, PSE_TRAIN_GRAD_ONLY.  Asynchronous. */
PSE_API int pse_costmodel_train_step(void *d_model, const float *d_feat, const float *d_target,
                                     const int64_t *d_index, int64_t batch, float lr, int32_t flags, double *d_loss,
                                     void *stream);

/*
 * Measurement helpers (no counterpart in the paper): the peaks the deposit's roofline is
 * taken against, measured on the running GPU.  Both enqueue one kernel on `stream`;
 * time it with events on that stream.
 *   pse_microbench_fma: `blocks` blocks of 256 threads, each thread running 8 independent
 *     FP32 FMA chains of `iters` steps: 2 * 8 * iters * 256 * blocks FLOP.  d_out: device
 *     float32 [blocks * 256] (written only to keep the chains alive).
 *   pse_microbench_red: `blocks` blocks of 256 threads, each adding 1.0 to `per_thread`
 *     pseudo-random cells of d_grid (device float64 [n_cells]) with FP64 global reductions.
 * PSE_ERR_INVALID_ARG for NULL pointers or sizes < 1.
 */
PSE_API int pse_microbench_fma(float *d_out, int64_t blocks, int64_t iters, void *stream);
PSE_API int pse_microbench_red(double *d_grid, int64_t n_cells, int64_t blocks, int64_t per_thread, void *stream);

/*
 * Bytes of device workspace an operation needs.  op = PSE_OP_*; lat may be NULL;
 * op_params: for PSE_OP_BUILD_OCTREE a host int32 max_level (required); for the deposit
 * ops a nullable host pse_deposit_opts (NULL = the default warp-cooperative schedule).
 * Every schedule but PSE_THREAD_PER_TET needs about 6 MB for the rounding residuals of
 * guarded tetrahedra (one block per warp of the persistent grid); the binned schedule
 * needs room for its queue on top.  Returns 0 for an unknown op.
 */
PSE_API size_t pse_workspace_size(int op, const pse_lattice *lat, const void *op_params);

/* Message of the last failed call on this host thread ("" if none).  Never NULL. */
PSE_API const char *pse_last_error(void);

/* PSE_ABI_VERSION of the loaded library. */
PSE_API int pse_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PSE_H_ */
