/*
 * oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, FP64 CPU implementation of the exact tetrahedron deposit of the
 * phase-space-element method (Kaehler, arXiv:1612.09491).  Only the tests, the
 * smoke check and the bench's CPU-baseline leg load this library.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * What it computes (Eq. 1 of Sec. 2, integrated over one deposit cell):
 *
 *     M[c] = sum_t (m_t / |V_t|) * vol(T_t  intersect  C_c)
 *
 * where T_t are the tetrahedra of the Lagrangian tessellation (each Lagrangian
 * cube of 8 neighbouring particles split into 6 tetrahedra of mass m_p/6,
 * Sec. 2) and C_c runs over the cubical cells of the deposit grid.
 *
 * How (the CPU deposit of Sec. 6.1 and the intersection of Sec. 6.3, in that order):
 *   1. loop over Lagrangian cubes (OpenMP; every thread owns a private mass
 *      buffer, the buffers are summed at the end in thread order -- Sec. 6);
 *   2. build the cube's 6 tetrahedra; take each tetrahedron's bounding box and
 *      loop over the deposit cells it touches (Sec. 6.1);
 *   3. per cell, test the trivial configurations first: the tetrahedron inside the
 *      cell, the cell inside the tetrahedron, or no intersection (Sec. 6.1);
 *   4. otherwise split the tetrahedron against the six face planes of the cell
 *      one after the other, keeping the part on the cell's side of each plane as
 *      a set of tetrahedra, and sum the volumes of what survives (Sec. 6.3);
 *   5. add (m_t/|V_t|) * volume to the cell (periodic images folded back).
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - the 6-tetrahedron split is the Kuhn (Freudenthal) split around the
 *     diagonal from corner 000 to corner 111;
 *   - m_t = particle_mass / 6, and |V_t| is the unsigned volume;
 *   - periodic box: every cube corner is unwrapped to the periodic image nearest
 *     to corner 000, and cell indices are folded modulo the grid size;
 *   - a tetrahedron with exactly zero FP64 volume deposits all of m_t into the
 *     cell that contains its vertex centroid;
 *   - cell c covers [c*h, (c+1)*h) per axis.
 *
 * Pins (tests/test_oracle_pins.py): closed-form Kuhn simplex volumes, uniform
 * density of the undisplaced lattice, tetrahedron-in-cell and cell-in-tetrahedron
 * closed forms, mass conservation, per-tetrahedron partition of unity, an exact
 * rational evaluation by a different algorithm (Lasserre's recursion), the
 * one-plane truncated-power formula, inclusion-exclusion over orthants, Monte
 * Carlo, and translation / axis-permutation symmetry.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_MEM -3

/* ------------------------------------------------------------------ */
/* geometry helpers                                                     */
/* ------------------------------------------------------------------ */

static double det3(const double a[3], const double b[3], const double c[3])
{
    return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
           a[2] * (b[0] * c[1] - b[1] * c[0]);
}

/* 6 * signed volume of the tetrahedron (p0, p1, p2, p3) */
static double tet_vol6(const double p[4][3])
{
    double a[3], b[3], c[3];
    for (int k = 0; k < 3; ++k) {
        a[k] = p[1][k] - p[0][k];
        b[k] = p[2][k] - p[0][k];
        c[k] = p[3][k] - p[0][k];
    }
    return det3(a, b, c);
}

static double tet_abs_vol(const double p[4][3]) { return fabs(tet_vol6(p)) / 6.0; }

/* An axis-aligned half-space: keep x[axis] <= s (keep_below = 1) or x[axis] >= s. */
typedef struct {
    int axis;
    int keep_below;
    double s;
} halfspace_t;

/* signed distance into the kept side: >= 0 means kept */
static double hs_dist(const halfspace_t *h, const double x[3])
{
    return h->keep_below ? (h->s - x[h->axis]) : (x[h->axis] - h->s);
}

/* point where the edge a->b crosses the plane, given d[a] >= 0 > d[b] */
static void cross_point(const halfspace_t *h, const double a[3], const double b[3], double da,
                        double db, double out[3])
{
    double t = da / (da - db);
    for (int k = 0; k < 3; ++k) out[k] = a[k] + t * (b[k] - a[k]);
    out[h->axis] = h->s; /* exactly on the plane */
}

static void copy3(double dst[3], const double src[3]) { memcpy(dst, src, 3 * sizeof(double)); }

static double clip_rec(const double p[4][3], const halfspace_t *hs, int nh);

/* volume of the triangular prism A(a0,a1,a2)--B(b0,b1,b2) (a_k joined to b_k),
 * triangulated into 3 tetrahedra, each further clipped by the remaining planes */
static double prism_rec(const double a[3][3], const double b[3][3], const halfspace_t *hs, int nh)
{
    double t[4][3];
    double v = 0.0;
    copy3(t[0], a[0]); copy3(t[1], a[1]); copy3(t[2], a[2]); copy3(t[3], b[0]);
    v += clip_rec(t, hs, nh);
    copy3(t[0], a[1]); copy3(t[1], a[2]); copy3(t[2], b[0]); copy3(t[3], b[1]);
    v += clip_rec(t, hs, nh);
    copy3(t[0], a[2]); copy3(t[1], b[0]); copy3(t[2], b[1]); copy3(t[3], b[2]);
    v += clip_rec(t, hs, nh);
    return v;
}

/*
 * Volume of (tetrahedron p) intersected with the half-spaces hs[0..nh-1]:
 * split against hs[0], keep the kept side as tetrahedra, recurse on each piece
 * with the remaining half-spaces (Sec. 6.3: every intermediate tetrahedron is
 * pruned against all remaining planes before the next one is processed).
 * Cases by the number k of kept vertices: 4 -> unchanged; 0 -> nothing;
 * 1 -> one tetrahedron; 2 -> a prism (3 tetrahedra); 3 -> the tetrahedron minus
 * its cut-off corner, also a prism (3 tetrahedra).
 */
static double clip_rec(const double p[4][3], const halfspace_t *hs, int nh)
{
    if (nh == 0) return tet_abs_vol(p);
    double d[4];
    int in[4], out[4], ni = 0, no = 0;
    for (int v = 0; v < 4; ++v) {
        d[v] = hs_dist(&hs[0], p[v]);
        if (d[v] >= 0.0) in[ni++] = v; else out[no++] = v;
    }
    if (no == 0) return clip_rec(p, hs + 1, nh - 1);
    if (ni == 0) return 0.0;
    if (ni == 1) {
        double t[4][3];
        int i = in[0];
        copy3(t[0], p[i]);
        for (int m = 0; m < 3; ++m)
            cross_point(&hs[0], p[i], p[out[m]], d[i], d[out[m]], t[m + 1]);
        return clip_rec(t, hs + 1, nh - 1);
    }
    if (ni == 2) {
        double a[3][3], b[3][3];
        int i1 = in[0], i2 = in[1], o1 = out[0], o2 = out[1];
        copy3(a[0], p[i1]);
        cross_point(&hs[0], p[i1], p[o1], d[i1], d[o1], a[1]);
        cross_point(&hs[0], p[i1], p[o2], d[i1], d[o2], a[2]);
        copy3(b[0], p[i2]);
        cross_point(&hs[0], p[i2], p[o1], d[i2], d[o1], b[1]);
        cross_point(&hs[0], p[i2], p[o2], d[i2], d[o2], b[2]);
        return prism_rec(a, b, hs + 1, nh - 1);
    }
    /* ni == 3 */
    {
        double a[3][3], b[3][3];
        int o = out[0];
        for (int m = 0; m < 3; ++m) {
            copy3(a[m], p[in[m]]);
            cross_point(&hs[0], p[in[m]], p[o], d[in[m]], d[o], b[m]);
        }
        return prism_rec(a, b, hs + 1, nh - 1);
    }
}

/* vol(T intersect [lo, hi]) by the six-plane split (planes x, y, z; low side first) */
static double tet_box_volume(const double p[4][3], const double lo[3], const double hi[3])
{
    halfspace_t hs[6];
    for (int a = 0; a < 3; ++a) {
        hs[2 * a].axis = a; hs[2 * a].keep_below = 0; hs[2 * a].s = lo[a];
        hs[2 * a + 1].axis = a; hs[2 * a + 1].keep_below = 1; hs[2 * a + 1].s = hi[a];
    }
    return clip_rec(p, hs, 6);
}

/* ------------------------------------------------------------------ */
/* trivial classification of a (tetrahedron, cell) pair (Sec. 6.1)      */
/* ------------------------------------------------------------------ */

enum { CLS_OUTSIDE = 0, CLS_CELL_IN_TET = 1, CLS_TET_IN_CELL = 2, CLS_PARTIAL = 3 };

static int classify(const double p[4][3], const double lo[3], const double hi[3])
{
    /* all four vertices beyond the same cell face -> no intersection */
    for (int a = 0; a < 3; ++a) {
        int below = 0, above = 0;
        for (int v = 0; v < 4; ++v) {
            if (p[v][a] <= lo[a]) ++below;
            if (p[v][a] >= hi[a]) ++above;
        }
        if (below == 4 || above == 4) return CLS_OUTSIDE;
    }
    /* all four vertices inside the cell */
    int all_in = 1;
    for (int v = 0; v < 4 && all_in; ++v)
        for (int a = 0; a < 3; ++a)
            if (p[v][a] < lo[a] || p[v][a] > hi[a]) { all_in = 0; break; }
    if (all_in) return CLS_TET_IN_CELL;
    /* all eight cell corners on the inner side of all four faces of T */
    double s6 = tet_vol6(p);
    static const int face[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
    int cell_in = 1;
    for (int f = 0; f < 4 && cell_in; ++f) {
        const double *A = p[face[f][0]], *B = p[face[f][1]], *C = p[face[f][2]];
        double u[3], w[3], n[3];
        for (int k = 0; k < 3; ++k) { u[k] = B[k] - A[k]; w[k] = C[k] - A[k]; }
        n[0] = u[1] * w[2] - u[2] * w[1];
        n[1] = u[2] * w[0] - u[0] * w[2];
        n[2] = u[0] * w[1] - u[1] * w[0];
        if (s6 < 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; } /* outward */
        double e = n[0] * A[0] + n[1] * A[1] + n[2] * A[2];
        int any_out = 0, all_out = 1;
        for (int c = 0; c < 8; ++c) {
            double q[3] = {(c & 1) ? hi[0] : lo[0], (c & 2) ? hi[1] : lo[1], (c & 4) ? hi[2] : lo[2]};
            double s = n[0] * q[0] + n[1] * q[1] + n[2] * q[2] - e;
            if (s > 0) any_out = 1; else all_out = 0;
        }
        if (all_out) return CLS_OUTSIDE;
        if (any_out) cell_in = 0;
    }
    if (cell_in) return CLS_CELL_IN_TET;
    return CLS_PARTIAL;
}

/* ------------------------------------------------------------------ */
/* one tetrahedron deposited onto a uniform periodic (or open) grid     */
/* ------------------------------------------------------------------ */

typedef struct {
    double box;
    int periodic;
    int64_t g[3];
    double h[3];
} grid_t;

typedef struct {
    double tets, bbox_cells, overlapped_cells, partial_cells, degenerate_tets, lost_mass;
} ostats_t;

static int64_t fold(int64_t c, int64_t g)
{
    int64_t r = c % g;
    return r < 0 ? r + g : r;
}

static void add_cell(double *mass, const grid_t *gr, int64_t ix, int64_t iy, int64_t iz, double m,
                     ostats_t *st)
{
    if (gr->periodic) {
        ix = fold(ix, gr->g[0]); iy = fold(iy, gr->g[1]); iz = fold(iz, gr->g[2]);
    } else if (ix < 0 || iy < 0 || iz < 0 || ix >= gr->g[0] || iy >= gr->g[1] || iz >= gr->g[2]) {
        st->lost_mass += m;
        return;
    }
    mass[ix + gr->g[0] * (iy + gr->g[1] * iz)] += m;
}

static void deposit_one_tet(const double p[4][3], double m_t, const grid_t *gr, double *mass,
                            ostats_t *st)
{
    st->tets += 1;
    double vol = tet_abs_vol(p);
    if (vol == 0.0) { /* degenerate: all mass to the cell of the vertex centroid */
        double c[3];
        for (int a = 0; a < 3; ++a) c[a] = 0.25 * (p[0][a] + p[1][a] + p[2][a] + p[3][a]);
        st->degenerate_tets += 1;
        add_cell(mass, gr, (int64_t)floor(c[0] / gr->h[0]), (int64_t)floor(c[1] / gr->h[1]),
                 (int64_t)floor(c[2] / gr->h[2]), m_t, st);
        return;
    }
    double rho = m_t / vol;
    int64_t lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        double mn = p[0][a], mx = p[0][a];
        for (int v = 1; v < 4; ++v) { mn = fmin(mn, p[v][a]); mx = fmax(mx, p[v][a]); }
        lo[a] = (int64_t)floor(mn / gr->h[a]);
        hi[a] = (int64_t)floor(mx / gr->h[a]);
    }
    for (int64_t iz = lo[2]; iz <= hi[2]; ++iz)
        for (int64_t iy = lo[1]; iy <= hi[1]; ++iy)
            for (int64_t ix = lo[0]; ix <= hi[0]; ++ix) {
                double clo[3] = {ix * gr->h[0], iy * gr->h[1], iz * gr->h[2]};
                double chi[3] = {(ix + 1) * gr->h[0], (iy + 1) * gr->h[1], (iz + 1) * gr->h[2]};
                st->bbox_cells += 1;
                double v;
                switch (classify(p, clo, chi)) {
                case CLS_OUTSIDE: v = 0.0; break;
                case CLS_TET_IN_CELL: v = vol; break;
                case CLS_CELL_IN_TET: v = gr->h[0] * gr->h[1] * gr->h[2]; break;
                default:
                    st->partial_cells += 1;
                    v = tet_box_volume(p, clo, chi);
                    break;
                }
                if (v > 0.0) {
                    st->overlapped_cells += 1;
                    add_cell(mass, gr, ix, iy, iz, rho * v, st);
                }
            }
}

/* ------------------------------------------------------------------ */
/* the Lagrangian tessellation (Sec. 2)                                 */
/* ------------------------------------------------------------------ */

/* Kuhn split: tetrahedron s walks 000 -> e_{pi0} -> e_{pi0}+e_{pi1} -> 111 */
static const int KUHN_PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static void lattice_tet(const float *pos, const int64_t n[3], double box, int periodic, int64_t ci,
                        int64_t cj, int64_t ck, int s, double p[4][3])
{
    int off[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 1}};
    off[1][KUHN_PERM[s][0]] = 1;
    off[2][KUHN_PERM[s][0]] = 1;
    off[2][KUHN_PERM[s][1]] = 1;
    for (int v = 0; v < 4; ++v) {
        int64_t i = ci + off[v][0], j = cj + off[v][1], k = ck + off[v][2];
        if (periodic) { i = fold(i, n[0]); j = fold(j, n[1]); k = fold(k, n[2]); }
        const float *x = pos + 3 * (i + n[0] * (j + n[1] * k));
        for (int a = 0; a < 3; ++a) p[v][a] = (double)x[a];
    }
    if (periodic) { /* nearest periodic image relative to corner 000 */
        for (int v = 1; v < 4; ++v)
            for (int a = 0; a < 3; ++a) {
                double d = p[v][a] - p[0][a];
                p[v][a] = p[0][a] + (d - box * floor(d / box + 0.5));
            }
    }
}

static int64_t n_cubes_of(const int64_t n[3], int periodic)
{
    if (periodic) return n[0] * n[1] * n[2];
    return (n[0] - 1) * (n[1] - 1) * (n[2] - 1);
}

static void cube_ijk(int64_t cube, const int64_t n[3], int periodic, int64_t *i, int64_t *j, int64_t *k)
{
    int64_t m0 = periodic ? n[0] : n[0] - 1, m1 = periodic ? n[1] : n[1] - 1;
    *i = cube % m0;
    *j = (cube / m0) % m1;
    *k = cube / (m0 * m1);
}

/* ------------------------------------------------------------------ */
/* exported entry points                                                */
/* ------------------------------------------------------------------ */

static int setup_grid(grid_t *gr, double box, int periodic, const int64_t grid_n[3])
{
    if (!(box > 0)) return OR_ERR_ARG;
    gr->box = box;
    gr->periodic = periodic;
    for (int a = 0; a < 3; ++a) {
        if (grid_n[a] <= 0) return OR_ERR_ARG;
        gr->g[a] = grid_n[a];
        gr->h[a] = box / (double)grid_n[a];
    }
    return OR_OK;
}

static int pick_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    return nthreads < 1 ? 1 : nthreads;
}

/* stats_out (nullable) receives: tets, bbox_cells, overlapped_cells, partial_cells,
 * degenerate_tets, lost_mass, threads_used */
int oracle_deposit_lattice(const float *pos, const int64_t n[3], double box, int periodic,
                           double particle_mass, const int64_t grid_n[3], double *cell_mass,
                           const int64_t *cube_ids, int64_t n_cube_ids, int nthreads,
                           double *stats_out)
{
    grid_t gr;
    if (!pos || !n || !cell_mass || setup_grid(&gr, box, periodic, grid_n) != OR_OK) return OR_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (n[a] < 2) return OR_ERR_ARG;
    int64_t ncell = gr.g[0] * gr.g[1] * gr.g[2];
    int64_t ncube = cube_ids ? n_cube_ids : n_cubes_of(n, periodic);
    int nt = pick_threads(nthreads);
    double **priv = (double **)calloc((size_t)nt, sizeof(double *));
    ostats_t *pst = (ostats_t *)calloc((size_t)nt, sizeof(ostats_t));
    if (!priv || !pst) { free(priv); free(pst); return OR_ERR_MEM; }
    for (int t = 0; t < nt; ++t) {
        priv[t] = (double *)calloc((size_t)ncell, sizeof(double));
        if (!priv[t]) {
            for (int u = 0; u < t; ++u) free(priv[u]);
            free(priv); free(pst);
            return OR_ERR_MEM;
        }
    }
    double m_t = particle_mass / 6.0;
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t q = 0; q < ncube; ++q) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int64_t cube = cube_ids ? cube_ids[q] : q;
        int64_t i, j, k;
        cube_ijk(cube, n, periodic, &i, &j, &k);
        for (int s = 0; s < 6; ++s) {
            double p[4][3];
            lattice_tet(pos, n, box, periodic, i, j, k, s, p);
            deposit_one_tet(p, m_t, &gr, priv[tid], &pst[tid]);
        }
    }
    /* fixed-order reduction of the private buffers */
    memset(cell_mass, 0, (size_t)ncell * sizeof(double));
    ostats_t tot = {0, 0, 0, 0, 0, 0};
    for (int t = 0; t < nt; ++t) {
        for (int64_t c = 0; c < ncell; ++c) cell_mass[c] += priv[t][c];
        free(priv[t]);
        tot.tets += pst[t].tets; tot.bbox_cells += pst[t].bbox_cells;
        tot.overlapped_cells += pst[t].overlapped_cells; tot.partial_cells += pst[t].partial_cells;
        tot.degenerate_tets += pst[t].degenerate_tets; tot.lost_mass += pst[t].lost_mass;
    }
    free(priv); free(pst);
    if (stats_out) {
        stats_out[0] = tot.tets; stats_out[1] = tot.bbox_cells; stats_out[2] = tot.overlapped_cells;
        stats_out[3] = tot.partial_cells; stats_out[4] = tot.degenerate_tets; stats_out[5] = tot.lost_mass;
        stats_out[6] = nt;
    }
    return OR_OK;
}

/* explicit tetrahedra: verts [n_tets][4][3] (box units, already unwrapped), masses [n_tets] */
int oracle_deposit_tets(const double *verts, const double *tet_mass, int64_t n_tets, double box,
                        int periodic, const int64_t grid_n[3], double *cell_mass, double *stats_out)
{
    grid_t gr;
    if (!verts || !tet_mass || !cell_mass || setup_grid(&gr, box, periodic, grid_n) != OR_OK) return OR_ERR_ARG;
    int64_t ncell = gr.g[0] * gr.g[1] * gr.g[2];
    memset(cell_mass, 0, (size_t)ncell * sizeof(double));
    ostats_t st = {0, 0, 0, 0, 0, 0};
    for (int64_t t = 0; t < n_tets; ++t) {
        double p[4][3];
        memcpy(p, verts + 12 * t, sizeof(p));
        deposit_one_tet(p, tet_mass[t], &gr, cell_mass, &st);
    }
    if (stats_out) {
        stats_out[0] = st.tets; stats_out[1] = st.bbox_cells; stats_out[2] = st.overlapped_cells;
        stats_out[3] = st.partial_cells; stats_out[4] = st.degenerate_tets; stats_out[5] = st.lost_mass;
        stats_out[6] = 1;
    }
    return OR_OK;
}

/* vol(T intersect box[lo, hi]) */
double oracle_tet_box_volume(const double *tet12, const double lo[3], const double hi[3])
{
    double p[4][3];
    memcpy(p, tet12, sizeof(p));
    return tet_box_volume(p, lo, hi);
}

/* vol(T intersect the given axis-aligned half-spaces), applied in the given order */
double oracle_tet_halfspaces_volume(const double *tet12, const int *axes, const int *keep_below,
                                    const double *s, int nh)
{
    double p[4][3];
    memcpy(p, tet12, sizeof(p));
    halfspace_t hs[16];
    if (nh < 0 || nh > 16) return -1.0;
    for (int i = 0; i < nh; ++i) { hs[i].axis = axes[i]; hs[i].keep_below = keep_below[i]; hs[i].s = s[i]; }
    return clip_rec(p, hs, nh);
}

/* the tetrahedron (cube, s) of the lattice, box units, unwrapped: out[12] */
int oracle_lattice_tet(const float *pos, const int64_t n[3], double box, int periodic, int64_t cube,
                       int s, double *out)
{
    if (!pos || !n || !out || s < 0 || s > 5) return OR_ERR_ARG;
    if (cube < 0 || cube >= n_cubes_of(n, periodic)) return OR_ERR_ARG;
    int64_t i, j, k;
    cube_ijk(cube, n, periodic, &i, &j, &k);
    double p[4][3];
    lattice_tet(pos, n, box, periodic, i, j, k, s, p);
    memcpy(out, p, sizeof(p));
    return OR_OK;
}

/* per-cell overlaps of one tetrahedron with a uniform grid (no folding):
 * writes up to cap entries (ix, iy, iz) into cells[3*i] and the overlap volume into vols[i];
 * returns the number of overlapped cells (may exceed cap), or a negative error */
int64_t oracle_tet_cells(const double *tet12, const double h[3], int64_t *cells, double *vols, int64_t cap)
{
    double p[4][3];
    memcpy(p, tet12, sizeof(p));
    int64_t lo[3], hi[3], cnt = 0;
    for (int a = 0; a < 3; ++a) {
        if (!(h[a] > 0)) return OR_ERR_ARG;
        double mn = p[0][a], mx = p[0][a];
        for (int v = 1; v < 4; ++v) { mn = fmin(mn, p[v][a]); mx = fmax(mx, p[v][a]); }
        lo[a] = (int64_t)floor(mn / h[a]);
        hi[a] = (int64_t)floor(mx / h[a]);
    }
    double vol = tet_abs_vol(p);
    for (int64_t iz = lo[2]; iz <= hi[2]; ++iz)
        for (int64_t iy = lo[1]; iy <= hi[1]; ++iy)
            for (int64_t ix = lo[0]; ix <= hi[0]; ++ix) {
                double clo[3] = {ix * h[0], iy * h[1], iz * h[2]};
                double chi[3] = {(ix + 1) * h[0], (iy + 1) * h[1], (iz + 1) * h[2]};
                double v;
                switch (classify(p, clo, chi)) {
                case CLS_OUTSIDE: v = 0.0; break;
                case CLS_TET_IN_CELL: v = vol; break;
                case CLS_CELL_IN_TET: v = h[0] * h[1] * h[2]; break;
                default: v = tet_box_volume(p, clo, chi); break;
                }
                if (v > 0.0) {
                    if (cnt < cap) {
                        cells[3 * cnt] = ix; cells[3 * cnt + 1] = iy; cells[3 * cnt + 2] = iz;
                        vols[cnt] = v;
                    }
                    ++cnt;
                }
            }
    return cnt;
}

double oracle_tet_volume(const double *tet12)
{
    double p[4][3];
    memcpy(p, tet12, sizeof(p));
    return tet_abs_vol(p);
}

/* ------------------------------------------------------------------ */
/* adaptive deposit grid: octree of cubic leaf blocks (Sec. 4)          */
/* ------------------------------------------------------------------ */
/*
 * The root node is the whole box [0, box)^3 (periodic box; the paper's root is the
 * tracers' bounding box).  A node at level l has side box/2^l and, if it is a
 * leaf, carries a block of bc^3 cells of side h_l = box/(bc*2^l) (every leaf has
 * the same cell count, Sec. 4).  Reading of the refinement rule used here (the
 * paper refines on an overlap count; this rule refines on tetrahedron size): a
 * node is refined iff l < max_level and the median, over the tetrahedra whose
 * vertex centroid lies in the node, of the tetrahedron's mean edge length is
 * below threshold_cells * h_l.  A node without tetrahedra is a leaf.  The median
 * is the exact lower median (element (count-1)/2 of the sorted values).
 * Leaves are listed depth first, children in the order c = cx + 2 cy + 4 cz.
 */

typedef struct {
    double *edge;     /* mean edge length of every tetrahedron (box units) */
    double *cen;      /* vertex centroid folded into [0, box)^3 */
    int64_t count;
} tetsizes_t;

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

typedef struct {
    const tetsizes_t *ts;
    double box, threshold;
    int bc, max_level;
    int32_t *leaves;
    int64_t cap, n_leaves;
    double *nodes;   /* optional per visited node: level, ix, iy, iz, count, median_cells, refined */
    int64_t node_cap, n_nodes;
} octbuild_t;

static void build_node(octbuild_t *B, int level, int64_t ix, int64_t iy, int64_t iz, int64_t *idx, int64_t cnt)
{
    double side = B->box / (double)(1LL << level);
    double h = side / B->bc;
    double med = -1.0;
    int refine = 0;
    if (cnt > 0) {
        double *v = (double *)malloc((size_t)cnt * sizeof(double));
        for (int64_t i = 0; i < cnt; ++i) v[i] = B->ts->edge[idx[i]];
        qsort(v, (size_t)cnt, sizeof(double), cmp_double);
        med = v[(cnt - 1) / 2];
        free(v);
        refine = (level < B->max_level) && (med < B->threshold * h);
    }
    if (B->nodes && B->n_nodes < B->node_cap) {
        double *o = B->nodes + 7 * B->n_nodes;
        o[0] = level; o[1] = (double)ix; o[2] = (double)iy; o[3] = (double)iz;
        o[4] = (double)cnt; o[5] = (med >= 0) ? med / h : -1.0; o[6] = refine;
    }
    B->n_nodes++;
    if (!refine) {
        if (B->n_leaves < B->cap) {
            int32_t *o = B->leaves + 4 * B->n_leaves;
            o[0] = level; o[1] = (int32_t)ix; o[2] = (int32_t)iy; o[3] = (int32_t)iz;
        }
        B->n_leaves++;
        return;
    }
    /* partition the tetrahedra among the 8 children by centroid */
    double half = side * 0.5;
    int64_t *part[8];
    int64_t pc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = 0; c < 8; ++c) part[c] = (int64_t *)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < cnt; ++i) {
        const double *x = B->ts->cen + 3 * idx[i];
        int cx = x[0] >= ix * side + half, cy = x[1] >= iy * side + half, cz = x[2] >= iz * side + half;
        int c = cx + 2 * cy + 4 * cz;
        part[c][pc[c]++] = idx[i];
    }
    for (int c = 0; c < 8; ++c) {
        build_node(B, level + 1, 2 * ix + (c & 1), 2 * iy + ((c >> 1) & 1), 2 * iz + (c >> 2), part[c], pc[c]);
        free(part[c]);
    }
}

/* returns the number of leaves (may exceed cap: call again with a larger buffer), or < 0 */
int64_t oracle_build_octree(const float *pos, const int64_t n[3], double box, int periodic, int bc, int max_level,
                            double threshold_cells, int32_t *leaves_out, int64_t cap, double *nodes_out,
                            int64_t node_cap, int64_t *n_nodes_out)
{
    if (!pos || !n || bc < 1 || max_level < 0 || max_level > 12 || !(box > 0)) return OR_ERR_ARG;
    int64_t ncube = n_cubes_of(n, periodic);
    tetsizes_t ts;
    ts.count = 6 * ncube;
    ts.edge = (double *)malloc((size_t)ts.count * sizeof(double));
    ts.cen = (double *)malloc((size_t)ts.count * 3 * sizeof(double));
    int64_t *idx = (int64_t *)malloc((size_t)ts.count * sizeof(int64_t));
    if (!ts.edge || !ts.cen || !idx) { free(ts.edge); free(ts.cen); free(idx); return OR_ERR_MEM; }
    for (int64_t q = 0; q < ncube; ++q) {
        int64_t i, j, k;
        cube_ijk(q, n, periodic, &i, &j, &k);
        for (int s = 0; s < 6; ++s) {
            double p[4][3];
            lattice_tet(pos, n, box, periodic, i, j, k, s, p);
            int64_t t = 6 * q + s;
            double e = 0.0;
            for (int a = 0; a < 4; ++a)
                for (int b = a + 1; b < 4; ++b) {
                    double d0 = p[b][0] - p[a][0], d1 = p[b][1] - p[a][1], d2 = p[b][2] - p[a][2];
                    e += sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                }
            ts.edge[t] = e / 6.0;
            for (int a = 0; a < 3; ++a) {
                double c = 0.25 * (p[0][a] + p[1][a] + p[2][a] + p[3][a]);
                c -= box * floor(c / box);
                if (c >= box) c = 0.0;
                ts.cen[3 * t + a] = c;
            }
            idx[t] = t;
        }
    }
    octbuild_t B;
    B.ts = &ts; B.box = box; B.threshold = threshold_cells; B.bc = bc; B.max_level = max_level;
    B.leaves = leaves_out; B.cap = leaves_out ? cap : 0; B.n_leaves = 0;
    B.nodes = nodes_out; B.node_cap = nodes_out ? node_cap : 0; B.n_nodes = 0;
    build_node(&B, 0, 0, 0, 0, idx, ts.count);
    free(ts.edge); free(ts.cen); free(idx);
    if (n_nodes_out) *n_nodes_out = B.n_nodes;
    return B.n_leaves;
}

/* ---- deposit onto the leaf blocks ---- */

typedef struct {
    double box;
    int periodic, bc, max_level;
    int64_t fine;          /* 2^max_level finest nodes per axis */
    int32_t *fine_map;     /* leaf id of every finest node, x fastest */
    const int32_t *leaves; /* [n_leaves][4] */
    int64_t n_leaves;
} octree_t;

static int make_fine_map(octree_t *T)
{
    int64_t F = T->fine, nf = F * F * F;
    T->fine_map = (int32_t *)malloc((size_t)nf * sizeof(int32_t));
    if (!T->fine_map) return OR_ERR_MEM;
    for (int64_t i = 0; i < nf; ++i) T->fine_map[i] = -1;
    for (int64_t l = 0; l < T->n_leaves; ++l) {
        const int32_t *L = T->leaves + 4 * l;
        if (L[0] < 0 || L[0] > T->max_level) return OR_ERR_ARG;
        int64_t span = 1LL << (T->max_level - L[0]);
        for (int a = 1; a < 4; ++a)
            if (L[a] < 0 || L[a] >= (1LL << L[0])) return OR_ERR_ARG;
        for (int64_t z = L[3] * span; z < (L[3] + 1) * span; ++z)
            for (int64_t y = L[2] * span; y < (L[2] + 1) * span; ++y)
                for (int64_t x = L[1] * span; x < (L[1] + 1) * span; ++x) {
                    int32_t *m = &T->fine_map[x + F * (y + F * z)];
                    if (*m != -1) return OR_ERR_ARG; /* overlapping leaves */
                    *m = (int32_t)l;
                }
    }
    for (int64_t i = 0; i < nf; ++i)
        if (T->fine_map[i] < 0) return OR_ERR_ARG; /* leaves do not tile the box */
    return OR_OK;
}

/* Returns OR_OK, or OR_ERR_MEM if the list of touched (leaf, periodic image) pairs
 * could not grow (nothing is deposited for this tetrahedron then). */
static int deposit_one_tet_octree(const double p[4][3], double m_t, const octree_t *T, double *mass, ostats_t *st)
{
    const double box = T->box;
    const int64_t F = T->fine;
    const double df = box / (double)F;
    const int64_t bc = T->bc, bc3 = bc * bc * bc;
    st->tets += 1;
    double vol = tet_abs_vol(p);
    if (vol == 0.0) { /* degenerate: the cell that contains the vertex centroid */
        double c[3];
        int64_t f[3], k[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = 0.25 * (p[0][a] + p[1][a] + p[2][a] + p[3][a]);
            int64_t fu = (int64_t)floor(c[a] / df);
            f[a] = fold(fu, F);
            k[a] = (fu - f[a]) / F;
        }
        st->degenerate_tets += 1;
        if (!T->periodic && (k[0] || k[1] || k[2])) { st->lost_mass += m_t; return OR_OK; }
        int32_t leaf = T->fine_map[f[0] + F * (f[1] + F * f[2])];
        const int32_t *L = T->leaves + 4 * leaf;
        double side = box / (double)(1LL << L[0]), h = side / bc;
        int64_t cc[3];
        for (int a = 0; a < 3; ++a) {
            double lo = L[1 + a] * side + k[a] * box;
            cc[a] = (int64_t)floor((c[a] - lo) / h);
            if (cc[a] < 0) cc[a] = 0;
            if (cc[a] >= bc) cc[a] = bc - 1;
        }
        mass[leaf * bc3 + cc[0] + bc * (cc[1] + bc * cc[2])] += m_t;
        return OR_OK;
    }
    double rho = m_t / vol;
    double mn[3], mx[3];
    int64_t f0[3], f1[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = mx[a] = p[0][a];
        for (int v = 1; v < 4; ++v) { mn[a] = fmin(mn[a], p[v][a]); mx[a] = fmax(mx[a], p[v][a]); }
        f0[a] = (int64_t)floor(mn[a] / df);
        f1[a] = (int64_t)floor(mx[a] / df);
    }
    /* distinct (leaf, periodic image) pairs touched by the bounding box; the list grows
     * on the heap, so a large tetrahedron over a deep tree keeps every leaf it touches */
    int64_t (*keys)[4] = NULL;
    int64_t nk = 0, cap = 0;
    for (int64_t fz = f0[2]; fz <= f1[2]; ++fz)
        for (int64_t fy = f0[1]; fy <= f1[1]; ++fy)
            for (int64_t fx = f0[0]; fx <= f1[0]; ++fx) {
                int64_t g[3] = {fold(fx, F), fold(fy, F), fold(fz, F)};
                int64_t k[3] = {(fx - g[0]) / F, (fy - g[1]) / F, (fz - g[2]) / F};
                if (!T->periodic && (k[0] || k[1] || k[2])) continue;
                int64_t leaf = T->fine_map[g[0] + F * (g[1] + F * g[2])];
                int dup = 0;
                for (int64_t q = 0; q < nk && !dup; ++q)
                    dup = keys[q][0] == leaf && keys[q][1] == k[0] && keys[q][2] == k[1] && keys[q][3] == k[2];
                if (dup) continue;
                if (nk == cap) {
                    int64_t ncap = cap ? 2 * cap : 64;
                    int64_t (*grown)[4] = (int64_t (*)[4])realloc(keys, (size_t)ncap * sizeof(*keys));
                    if (!grown) { free(keys); return OR_ERR_MEM; }
                    keys = grown;
                    cap = ncap;
                }
                keys[nk][0] = leaf; keys[nk][1] = k[0]; keys[nk][2] = k[1]; keys[nk][3] = k[2];
                ++nk;
            }
    double deposited = 0.0;
    for (int64_t q = 0; q < nk; ++q) {
        const int32_t *L = T->leaves + 4 * keys[q][0];
        double side = box / (double)(1LL << L[0]), h = side / bc;
        double lo[3];
        int64_t c0[3], c1[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = L[1 + a] * side + keys[q][1 + a] * box;
            c0[a] = (int64_t)floor((mn[a] - lo[a]) / h);
            c1[a] = (int64_t)floor((mx[a] - lo[a]) / h);
            if (c0[a] < 0) c0[a] = 0;
            if (c1[a] > bc - 1) c1[a] = bc - 1;
        }
        double *blk = mass + keys[q][0] * bc3;
        for (int64_t cz = c0[2]; cz <= c1[2]; ++cz)
            for (int64_t cy = c0[1]; cy <= c1[1]; ++cy)
                for (int64_t cx = c0[0]; cx <= c1[0]; ++cx) {
                    double clo[3] = {lo[0] + cx * h, lo[1] + cy * h, lo[2] + cz * h};
                    double chi[3] = {lo[0] + (cx + 1) * h, lo[1] + (cy + 1) * h, lo[2] + (cz + 1) * h};
                    st->bbox_cells += 1;
                    double v;
                    switch (classify(p, clo, chi)) {
                    case CLS_OUTSIDE: v = 0.0; break;
                    case CLS_TET_IN_CELL: v = vol; break;
                    case CLS_CELL_IN_TET: v = h * h * h; break;
                    default:
                        st->partial_cells += 1;
                        v = tet_box_volume(p, clo, chi);
                        break;
                    }
                    if (v > 0.0) {
                        st->overlapped_cells += 1;
                        blk[cx + bc * (cy + bc * cz)] += rho * v;
                        deposited += rho * v;
                    }
                }
    }
    free(keys);
    if (!T->periodic) st->lost_mass += m_t - deposited;
    return OR_OK;
}

/* leaf_mass [n_leaves * bc^3]: block of leaf l at l*bc^3, cells x fastest */
int oracle_deposit_octree(const float *pos, const int64_t n[3], double box, int periodic, double particle_mass,
                          int bc, int max_level, const int32_t *leaves, int64_t n_leaves, double *leaf_mass,
                          const int64_t *cube_ids, int64_t n_cube_ids, int nthreads, double *stats_out)
{
    if (!pos || !n || !leaves || !leaf_mass || bc < 1 || max_level < 0 || max_level > 10 || !(box > 0))
        return OR_ERR_ARG;
    octree_t T;
    T.box = box; T.periodic = periodic; T.bc = bc; T.max_level = max_level;
    T.fine = 1LL << max_level; T.leaves = leaves; T.n_leaves = n_leaves; T.fine_map = NULL;
    int rc = make_fine_map(&T);
    if (rc != OR_OK) { free(T.fine_map); return rc; }
    int64_t ncell = n_leaves * (int64_t)bc * bc * bc;
    int64_t ncube = cube_ids ? n_cube_ids : n_cubes_of(n, periodic);
    int nt = pick_threads(nthreads);
    double **priv = (double **)calloc((size_t)nt, sizeof(double *));
    ostats_t *pst = (ostats_t *)calloc((size_t)nt, sizeof(ostats_t));
    if (!priv || !pst) { free(priv); free(pst); free(T.fine_map); return OR_ERR_MEM; }
    for (int t = 0; t < nt; ++t) {
        priv[t] = (double *)calloc((size_t)ncell, sizeof(double));
        if (!priv[t]) {
            for (int u = 0; u < t; ++u) free(priv[u]);
            free(priv); free(pst); free(T.fine_map);
            return OR_ERR_MEM;
        }
    }
    double m_t = particle_mass / 6.0;
    int failed = 0;
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t q = 0; q < ncube; ++q) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int64_t cube = cube_ids ? cube_ids[q] : q;
        int64_t i, j, k;
        cube_ijk(cube, n, periodic, &i, &j, &k);
        for (int s = 0; s < 6; ++s) {
            double p[4][3];
            lattice_tet(pos, n, box, periodic, i, j, k, s, p);
            if (deposit_one_tet_octree(p, m_t, &T, priv[tid], &pst[tid]) != OR_OK) {
#pragma omp atomic write
                failed = 1;
            }
        }
    }
    if (failed) {
        for (int t = 0; t < nt; ++t) free(priv[t]);
        free(priv); free(pst); free(T.fine_map);
        return OR_ERR_MEM;
    }
    memset(leaf_mass, 0, (size_t)ncell * sizeof(double));
    ostats_t tot = {0, 0, 0, 0, 0, 0};
    for (int t = 0; t < nt; ++t) {
        for (int64_t c = 0; c < ncell; ++c) leaf_mass[c] += priv[t][c];
        free(priv[t]);
        tot.tets += pst[t].tets; tot.bbox_cells += pst[t].bbox_cells;
        tot.overlapped_cells += pst[t].overlapped_cells; tot.partial_cells += pst[t].partial_cells;
        tot.degenerate_tets += pst[t].degenerate_tets; tot.lost_mass += pst[t].lost_mass;
    }
    free(priv); free(pst); free(T.fine_map);
    if (stats_out) {
        stats_out[0] = tot.tets; stats_out[1] = tot.bbox_cells; stats_out[2] = tot.overlapped_cells;
        stats_out[3] = tot.partial_cells; stats_out[4] = tot.degenerate_tets; stats_out[5] = tot.lost_mass;
        stats_out[6] = nt;
    }
    return OR_OK;
}
