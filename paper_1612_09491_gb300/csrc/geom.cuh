// geom.cuh -- per-tetrahedron geometry, cell classification and the exact
// tetrahedron / cube overlap volume, for the deposit kernels (sm_103a).
//
// Coordinates are GRID units (a cell is a unit cube) relative to a tetrahedron's
// base cell; the clip works in the frame of one cell, where that cell is [0,1]^3.
//
// Overlap volume (the operation of Sec. 6.3, computed by a different method than
// the paper's recursive split): for the cell C = [0,1)^3 = column x [0,1) with
// column = [0,1)^2 in (x, y), take the field F = (0, 0, chi_col(x,y) clamp(z,0,1)),
// whose divergence is the indicator of C.  Integrating along z over the convex
// tetrahedron T (between its lower and upper surfaces) gives
//
//     vol(T ∩ C) = Σ_faces f of T  ∫_{F_f} chi_col(x,y) clamp(z,0,1) n_z dA
//                = Σ_f  ∫∫_{proj_xy(F_f) ∩ column} clamp(z_f(x,y), 0, 1) dx dy  (signed by n_z)
//
// so only the four face triangles of T are clipped, never the polytope T ∩ C.
// Per face: Sutherland-Hodgman clips against x >= 0, x < 1, y >= 0, y < 1 and
// z >= 0 on an edge list (the polygon stays a closed chain; every slot is a
// compile-time register), then a split at z = 1: the part below contributes the
// projected integral of z (a fan from an anchor o on the face plane,
// Σ_edges ½ cross_xy(a-o, b-o) (z_o + z_a + z_b)/3), the part above contributes
// its projected area.  Faces with n_z = 0 contribute nothing.
//
// The result is a continuous function of the four vertices: a vertex or a face
// lying exactly on a cell plane needs no tie rule (whichever side a tie goes,
// the clipped polygon is the same, and anything lying in a plane x = const or
// y = const has zero projected area), so rounding in near-degenerate
// configurations costs rounding-sized errors only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#ifndef PSE_HD
#define PSE_HD __host__ __device__ __forceinline__
#endif

namespace pse {

template <class T>
struct P3 {
    T x, y, z;
};

template <class T>
PSE_HD P3<T> mk(T x, T y, T z)
{
    P3<T> p;
    p.x = x; p.y = y; p.z = z;
    return p;
}

template <int AX, class T>
PSE_HD T get(const P3<T> &p)
{
    if constexpr (AX == 0) return p.x;
    else if constexpr (AX == 1) return p.y;
    else return p.z;
}

template <int AX, class T>
PSE_HD void put(P3<T> &p, T v)
{
    if constexpr (AX == 0) p.x = v;
    else if constexpr (AX == 1) p.y = v;
    else p.z = v;
}

PSE_HD float fdiv(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
PSE_HD double fdiv(double a, double b) { return a / b; }
PSE_HD float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
PSE_HD double fmaT(double a, double b, double c) { return fma(a, b, c); }

template <class T>
PSE_HD T cross_xy(const P3<T> &a, const P3<T> &b)
{
    return a.x * b.y - a.y * b.x;
}

template <class T>
PSE_HD P3<T> sub(const P3<T> &a, const P3<T> &b)
{
    return mk<T>(a.x - b.x, a.y - b.y, a.z - b.z);
}

template <class T>
PSE_HD P3<T> cross(const P3<T> &a, const P3<T> &b)
{
    return mk<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

template <class T>
PSE_HD T dot(const P3<T> &a, const P3<T> &b)
{
    return a.x * b.x + a.y * b.y + a.z * b.z;
}

// Faces of a positively oriented tetrahedron, outward vertex order; face f is
// opposite vertex f.
PSE_HD void face_vertices(int f, int &a, int &b, int &c)
{
    a = (f == 0) ? 1 : 0;
    b = (f == 0) ? 2 : (f == 1) ? 3 : (f == 2) ? 1 : 2;
    c = (f == 0) ? 3 : (f == 1) ? 2 : (f == 2) ? 3 : 1;
}

template <class T>
PSE_HD P3<T> pick4(const P3<T> (&p)[4], int i)
{
    P3<T> r = p[0];
    r = (i == 1) ? p[1] : r;
    r = (i == 2) ? p[2] : r;
    r = (i == 3) ? p[3] : r;
    return r;
}

// ---------------------------------------------------------------------------
// Sutherland-Hodgman clip of an edge-list polygon against one cell plane.
// Slots [0, NE) hold the current edges (a -> b); the edge this clip creates on
// the plane (exit -> entry) goes to slot NE.  Dropped edges collapse onto the
// anchor o, which makes their fan contribution exactly zero.
// ---------------------------------------------------------------------------
template <class T, int AX, bool UP, int NE>
PSE_HD void clip_plane(P3<T> (&A)[9], P3<T> (&B)[9], const P3<T> &o, bool &crossed)
{
    P3<T> ex = o, en = o;
    bool got = false;
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        const T ca = get<AX>(A[k]), cb = get<AX>(B[k]);
        const bool ia = UP ? (ca < T(1)) : (ca >= T(0));
        const bool ib = UP ? (cb < T(1)) : (cb >= T(0));
        if (ia != ib) {
            const T s = UP ? T(1) : T(0);
            const T t = fdiv(s - ca, cb - ca);
            P3<T> I = mk<T>(fmaT(t, B[k].x - A[k].x, A[k].x), fmaT(t, B[k].y - A[k].y, A[k].y),
                            fmaT(t, B[k].z - A[k].z, A[k].z));
            put<AX>(I, s);
            if (ia) { B[k] = I; ex = I; } else { A[k] = I; en = I; }
            got = true;
        } else if (!ia) {
            A[k] = o;
            B[k] = o;
        }
    }
    A[NE] = ex;
    B[NE] = en;
    crossed = got;
}

template <class T, int NE>
PSE_HD void collapse_slot(P3<T> (&A)[9], P3<T> (&B)[9], const P3<T> &o)
{
    A[NE] = o;
    B[NE] = o;
}

// Split the edge-list polygon at z = 1: the part with z < 1 stays in slots [0, NE)
// (its new edge on z = 1 goes to slot NE); the part with z >= 1 is not stored, its
// doubled projected area about the column centre (½, ½) is returned.
template <class T, int NE>
PSE_HD T split_z1(P3<T> (&A)[9], P3<T> (&B)[9], const P3<T> &o)
{
    P3<T> ex = o, en = o;
    bool got = false;
    T hi2 = T(0);
    const T h = T(0.5);
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        const T ca = A[k].z, cb = B[k].z;
        const bool ia = ca < T(1), ib = cb < T(1);
        if (ia != ib) {
            const T t = fdiv(T(1) - ca, cb - ca);
            const P3<T> I = mk<T>(fmaT(t, B[k].x - A[k].x, A[k].x), fmaT(t, B[k].y - A[k].y, A[k].y), T(1));
            if (ia) {
                hi2 += (I.x - h) * (B[k].y - h) - (I.y - h) * (B[k].x - h);
                B[k] = I;
                ex = I;
            } else {
                hi2 += (A[k].x - h) * (I.y - h) - (A[k].y - h) * (I.x - h);
                A[k] = I;
                en = I;
            }
            got = true;
        } else if (!ia) {
            hi2 += (A[k].x - h) * (B[k].y - h) - (A[k].y - h) * (B[k].x - h);
            A[k] = o;
            B[k] = o;
        }
    }
    A[NE] = ex;
    B[NE] = en;
    if (got) hi2 += (en.x - h) * (ex.y - h) - (en.y - h) * (ex.x - h);
    return hi2;
}

// ---------------------------------------------------------------------------
// Exact overlap volume of a positively oriented tetrahedron p[4] with [0,1]^3.
// n[f], e[f]: outward face normals (unnormalised) and offsets in the cell frame
// (inside iff n.x <= e); inv_n2[f] = 1/|n_f|^2.
// ---------------------------------------------------------------------------
template <class T>
PSE_HD T overlap_volume(const P3<T> (&p)[4], const P3<T> (&n)[4], const T (&e)[4], const T (&inv_n2)[4])
{
    T vol = T(0);
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        int ia, ib, ic;
        face_vertices(f, ia, ib, ic);
        const P3<T> a = pick4(p, ia), b = pick4(p, ib), c = pick4(p, ic);
        const T mnx = fmin(a.x, fmin(b.x, c.x)), mxx = fmax(a.x, fmax(b.x, c.x));
        const T mny = fmin(a.y, fmin(b.y, c.y)), mxy = fmax(a.y, fmax(b.y, c.y));
        const T mnz = fmin(a.z, fmin(b.z, c.z)), mxz = fmax(a.z, fmax(b.z, c.z));
        // outside the column, or entirely below z = 0 (clamp = 0): nothing
        if (mxx < T(0) || mnx >= T(1) || mxy < T(0) || mny >= T(1) || mxz < T(0)) continue;
        const P3<T> nf = (f == 0) ? n[0] : (f == 1) ? n[1] : (f == 2) ? n[2] : n[3];
        if (nf.z == T(0)) continue;  // vertical face: zero projected area
        const T ef = (f == 0) ? e[0] : (f == 1) ? e[1] : (f == 2) ? e[2] : e[3];
        const T i2 = (f == 0) ? inv_n2[0] : (f == 1) ? inv_n2[1] : (f == 2) ? inv_n2[2] : inv_n2[3];
        // anchor: the cell centre projected onto the face plane
        const T sc = (T(0.5) * (nf.x + nf.y + nf.z) - ef) * i2;
        const P3<T> o = mk<T>(T(0.5) - sc * nf.x, T(0.5) - sc * nf.y, T(0.5) - sc * nf.z);

        P3<T> A[9], B[9];
        A[0] = a; B[0] = b;
        A[1] = b; B[1] = c;
        A[2] = c; B[2] = a;
        bool cr;
        if (mnx < T(0)) clip_plane<T, 0, false, 3>(A, B, o, cr); else collapse_slot<T, 3>(A, B, o);
        if (mxx >= T(1)) clip_plane<T, 0, true, 4>(A, B, o, cr); else collapse_slot<T, 4>(A, B, o);
        if (mny < T(0)) clip_plane<T, 1, false, 5>(A, B, o, cr); else collapse_slot<T, 5>(A, B, o);
        if (mxy >= T(1)) clip_plane<T, 1, true, 6>(A, B, o, cr); else collapse_slot<T, 6>(A, B, o);
        if (mnz < T(0)) clip_plane<T, 2, false, 7>(A, B, o, cr); else collapse_slot<T, 7>(A, B, o);
        T hi2 = T(0);
        if (mxz >= T(1)) hi2 = split_z1<T, 8>(A, B, o); else collapse_slot<T, 8>(A, B, o);
        // below z = 1: projected integral of z, fan from the anchor
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const P3<T> u = sub(A[k], o), w = sub(B[k], o);
            acc = fmaT(cross_xy(u, w), (o.z + A[k].z + B[k].z), acc);
        }
        vol += acc * T(1.0 / 6.0) + T(0.5) * hi2;
    }
    return vol;
}

// ---------------------------------------------------------------------------
// Per-tetrahedron set-up in grid units.
// ---------------------------------------------------------------------------
template <class T>
struct TetSetup {
    P3<T> v[4];     // vertices relative to the base cell corner, positively oriented
    P3<T> n[4];     // outward face normals (face f opposite vertex f)
    T e[4];         // n_f . x <= e_f inside (base-cell frame)
    T inv_n2[4];
    T pos[4], neg[4];  // sum of positive / negative components of n_f (corner extremes)
    int lo[3], dim[3]; // bounding-box cells relative to the base: [lo, lo + dim)
    double vol6;       // |6 V| in grid units (float64)
    float kappa;       // conditioning estimate (surface * extent / volume)
};

template <class T>
PSE_HD void tet_setup(P3<T> (&v)[4], TetSetup<T> &s)
{
    // float64 signed volume of the vertices as given
    const double ax = (double)v[1].x - (double)v[0].x, ay = (double)v[1].y - (double)v[0].y,
                 az = (double)v[1].z - (double)v[0].z;
    const double bx = (double)v[2].x - (double)v[0].x, by = (double)v[2].y - (double)v[0].y,
                 bz = (double)v[2].z - (double)v[0].z;
    const double cx = (double)v[3].x - (double)v[0].x, cy = (double)v[3].y - (double)v[0].y,
                 cz = (double)v[3].z - (double)v[0].z;
    const double d6 = ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx);
    if (d6 < 0.0) {  // make it positively oriented: swap v1 and v2
        const P3<T> t = v[1];
        v[1] = v[2];
        v[2] = t;
    }
    s.vol6 = fabs(d6);
#pragma unroll
    for (int i = 0; i < 4; ++i) s.v[i] = v[i];
    T area2 = T(0);
    T lmax2 = T(0);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        int ia, ib, ic;
        face_vertices(f, ia, ib, ic);
        const P3<T> a = pick4(s.v, ia), b = pick4(s.v, ib), c = pick4(s.v, ic);
        const P3<T> nn = cross(sub(b, a), sub(c, a));
        const T n2 = dot(nn, nn);
        s.n[f] = nn;
        s.e[f] = dot(nn, a);
        s.inv_n2[f] = (n2 > T(0)) ? T(1) / n2 : T(0);
        s.pos[f] = fmax(nn.x, T(0)) + fmax(nn.y, T(0)) + fmax(nn.z, T(0));
        s.neg[f] = fmin(nn.x, T(0)) + fmin(nn.y, T(0)) + fmin(nn.z, T(0));
        area2 += sqrt(n2);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i + 1; j < 4; ++j) {
            const P3<T> d = sub(s.v[j], s.v[i]);
            lmax2 = fmax(lmax2, dot(d, d));
        }
    int lo[3], hi[3];
    {
        const T mnx = fmin(fmin(v[0].x, v[1].x), fmin(v[2].x, v[3].x));
        const T mxx = fmax(fmax(v[0].x, v[1].x), fmax(v[2].x, v[3].x));
        const T mny = fmin(fmin(v[0].y, v[1].y), fmin(v[2].y, v[3].y));
        const T mxy = fmax(fmax(v[0].y, v[1].y), fmax(v[2].y, v[3].y));
        const T mnz = fmin(fmin(v[0].z, v[1].z), fmin(v[2].z, v[3].z));
        const T mxz = fmax(fmax(v[0].z, v[1].z), fmax(v[2].z, v[3].z));
        // non-finite or huge coordinates give an empty range (dim 0), which callers reject
        const T big = T(16777216);
        const bool fin = (mnx > -big && mxx < big && mny > -big && mxy < big && mnz > -big && mxz < big);
        lo[0] = fin ? (int)floor(mnx) : 0; hi[0] = fin ? (int)floor(mxx) : -1;
        lo[1] = fin ? (int)floor(mny) : 0; hi[1] = fin ? (int)floor(mxy) : -1;
        lo[2] = fin ? (int)floor(mnz) : 0; hi[2] = fin ? (int)floor(mxz) : -1;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        s.lo[a] = lo[a];
        s.dim[a] = hi[a] - lo[a] + 1;
    }
    const double denom = s.vol6 > 0.0 ? s.vol6 : 1e-300;
    s.kappa = (float)((double)area2 * sqrt((double)lmax2) / denom);
}

// Cell classification for the cell with corner c (base-cell frame, integers).
enum { CELL_OUTSIDE = 0, CELL_INSIDE = 1, CELL_PARTIAL = 2 };

template <class T>
PSE_HD int classify_cell(const P3<T> (&n)[4], const T (&e)[4], const T (&pos)[4],
                                             const T (&neg)[4], T cx, T cy, T cz)
{
    bool inside = true, outside = false;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const T s = fmaT(n[f].x, cx, fmaT(n[f].y, cy, fmaT(n[f].z, cz, -e[f])));
        inside = inside && (s + pos[f] <= T(0));
        outside = outside || (s + neg[f] >= T(0));
    }
    return outside ? CELL_OUTSIDE : (inside ? CELL_INSIDE : CELL_PARTIAL);
}

}  // namespace pse
