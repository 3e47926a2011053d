// geom.cuh -- per-tetrahedron geometry, cell classification and the exact
// tetrahedron / cube overlap volume, for the deposit kernels (sm_103a).
//
// Coordinates are GRID units (a cell is a unit cube) relative to a tetrahedron's
// base cell; the clip works in the frame of one cell, where that cell is [0,1]^3.
//
// Overlap volume (the operation of Sec. 6.3, computed by a different method than
// the paper's recursive split).  For the cell C = [0,1)^3 = column x [0,1) with
// column = [0,1)^2 in (x, y), take a field F = (0, 0, chi_col(x,y) clamp(z,0,1) - g(x,y))
// with any g that does not depend on z: its divergence is the indicator of C.
// Integrating along z over the convex tetrahedron T gives
//
//   vol(T ∩ C) = Σ_faces f  ∫∫_{proj_xy(F_f) ∩ column} (clamp(z_f(x,y), 0, 1) - g(x,y)) dx dy
//
// (signed by the sign of the face normal's z component), so only the four face
// triangles of T are clipped, never the polytope T ∩ C.  g integrates to zero
// over the closed surface; it is there for accuracy: g = l(x, y), the plane of
// the tetrahedron's most horizontal face moved through its centroid, makes the
// integrands of the large faces of a flat ("sliver") tetrahedron small instead
// of O(1) numbers that cancel.
//
// Per face: Sutherland-Hodgman clips against the column's four sides on an edge
// list (the polygon stays a closed chain; every slot is a compile-time register),
// then splits at z = 0 and z = 1.  Each region integrates a linear function of
// (x, y) by a fan from an anchor, Σ_edges ½ cross_xy(a-o, b-o) (f(o)+f(a)+f(b))/3:
// below z = 0, f = 0 - l; above z = 1, f = 1 - l (anchor: the local origin, these
// integrands are defined on the whole plane); between, f = z_f - l (anchor: the
// local origin projected onto the face plane).
//
// The arithmetic runs in a local frame whose origin q is the tetrahedron's
// centroid clamped into the cell and rounded to a multiple of 1/256, so the
// cell planes stay exact and rounding is relative to the size of the pieces.
// The result is a continuous function of the four vertices: a vertex or a face
// lying exactly on a cell plane needs no tie rule (whichever side a tie goes,
// the clipped polygon is the same, and anything lying in a plane x = const or
// y = const has zero projected area), so near-degenerate configurations cost
// rounding-sized errors only.  The clip also returns the sum of the magnitudes
// of its terms, which bounds its rounding error (used by the FP32 guard).
#pragma once

#include <cmath>
#include <math.h>
#include <cstdint>
#include <limits>
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

// unit roundoff of each arithmetic type (the classification tolerance is a few of these)
template <class T>
PSE_HD T roundoff();
template <>
PSE_HD float roundoff<float>() { return 1.1920928955078125e-07f; }  // 2^-23
template <>
PSE_HD double roundoff<double>() { return 2.220446049250313e-16; }  // 2^-52

// products rounded on their own (never fused), so that cross_xy(u, u) is exactly 0
PSE_HD float mul_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
PSE_HD double mul_rn(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}

template <class T>
PSE_HD T cross_xy(const P3<T> &a, const P3<T> &b)
{
    return mul_rn(a.x, b.y) - mul_rn(a.y, b.x);
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
// Polygon clipping on an edge list (slots of directed edges a -> b; the polygon
// stays a closed chain; a dropped edge collapses to a point and keeps zero length).  A slab pass
// clips against the two parallel planes lo <= c < hi of one axis at once and appends
// the two edges it creates on them (exit -> entry).  Classification uses a rounding
// tolerance: a coordinate within tol of a plane counts as lying on it (on lo: inside;
// on hi: outside), so a polygon that is convex up to rounding crosses each plane at
// most twice.  Every edge is processed without branches.
// ---------------------------------------------------------------------------
template <class T>
PSE_HD T coord(const P3<T> &p, int ax)
{
    return ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
}

// t clamped to [0, 1] (NaN -> 0): an edge's crossing point stays on the edge, finite even for
// edges parallel to the plane, so an edge that a pass drops can be kept as a zero-length edge
// at that point (it adds exactly nothing to any sum) instead of being moved elsewhere.
PSE_HD float sat01(float x)
{
#ifdef __CUDA_ARCH__
    return __saturatef(x);
#else
    return x > 0.f ? (x < 1.f ? x : 1.f) : 0.f;
#endif
}
PSE_HD double sat01(double x) { return x > 0.0 ? (x < 1.0 ? x : 1.0) : 0.0; }

// point of edge a -> b at parameter t, with coordinate `ax` set exactly to s
template <class T>
PSE_HD P3<T> at_plane(const P3<T> &a, const P3<T> &b, T t, int ax, T s)
{
    P3<T> r = mk<T>(fmaT(t, b.x - a.x, a.x), fmaT(t, b.y - a.y, a.y), fmaT(t, b.z - a.z, a.z));
    r.x = (ax == 0) ? s : r.x;
    r.y = (ax == 1) ? s : r.y;
    r.z = (ax == 2) ? s : r.z;
    return r;
}

// Clip slots [0, NE) against lo <= c_ax < hi; new edges go to slots NE (on lo) and NE+1 (on hi).
template <class T, int NE>
PSE_HD void clip_slab(P3<T> (&A)[7], P3<T> (&B)[7], int ax, T lo, T hi, T tol)
{
    const P3<T> z0 = mk<T>(T(0), T(0), T(0));
    P3<T> xl = z0, nl = z0, xh = z0, nh = z0;  // exit / entry points on lo and on hi
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        const P3<T> a = A[k], b = B[k];
        const T ca = coord(a, ax), cb = coord(b, ax);
        const bool a_lo = ca < lo - tol, b_lo = cb < lo - tol;   // below the slab
        const bool a_hi = ca >= hi - tol, b_hi = cb >= hi - tol; // above the slab (on hi counts as above)
        const T inv = fdiv(T(1), cb - ca);
        const P3<T> pl = at_plane(a, b, sat01((lo - ca) * inv), ax, lo);
        const P3<T> ph = at_plane(a, b, sat01((hi - ca) * inv), ax, hi);
        // an edge wholly outside becomes the zero-length edge (pl, pl) or (ph, ph)
        const P3<T> na = a_lo ? pl : (a_hi ? ph : a);
        const P3<T> nb = b_lo ? pl : (b_hi ? ph : b);
        A[k] = na;
        B[k] = nb;
        xl = (!a_lo && b_lo) ? pl : xl;
        nl = (a_lo && !b_lo) ? pl : nl;
        xh = (!a_hi && b_hi) ? ph : xh;
        nh = (a_hi && !b_hi) ? ph : nh;
    }
    A[NE] = xl;
    B[NE] = nl;
    A[NE + 1] = xh;
    B[NE + 1] = nh;
}

// 6 * ∫∫ (s - l(x,y)) dx dy over the projection of segment-fan (a, b) from the local origin
template <class T>
PSE_HD T fan_const(const P3<T> &a, const P3<T> &b, T s, T l0, T lx, T ly)
{
    const T fa = s - fmaT(lx, a.x, fmaT(ly, a.y, l0));
    const T fb = s - fmaT(lx, b.x, fmaT(ly, b.y, l0));
    return cross_xy(a, b) * ((s - l0) + fa + fb);
}

// 6 * integral of (z - l(x,y)) over the projection of the fan triangle (o, a, b)
template <class T>
PSE_HD T fan_mid(const P3<T> &a, const P3<T> &b, const P3<T> &o, T fo, T l0, T lx, T ly)
{
    const T fa = a.z - fmaT(lx, a.x, fmaT(ly, a.y, l0));
    const T fb = b.z - fmaT(lx, b.x, fmaT(ly, b.y, l0));
    return cross_xy(sub(a, o), sub(b, o)) * (fo + fa + fb);
}

// Split slots [0, NE) at z = lo and z = hi and integrate all three parts in one pass:
// below lo and above hi the integrands are lo - l and hi - l (fans from the local
// origin); in between it is z - l (fan from o, a point of the face plane).  Returns
// 6 * the whole integral; mag accumulates the magnitudes of the three parts.
template <class T, int NE>
PSE_HD T split_zslab(const P3<T> (&A)[7], const P3<T> (&B)[7], T lo, T hi, T tol, T l0, T lx, T ly,
                     const P3<T> &o, T &mag)
{
    const P3<T> z0 = mk<T>(T(0), T(0), T(0));
    P3<T> xl = z0, nl = z0, xh = z0, nh = z0;
    T below = T(0), above = T(0), mid = T(0);
    const T fo = o.z - fmaT(lx, o.x, fmaT(ly, o.y, l0));
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        const P3<T> a = A[k], b = B[k];
        const bool a_lo = a.z < lo - tol, b_lo = b.z < lo - tol;
        const bool a_hi = a.z >= hi - tol, b_hi = b.z >= hi - tol;
        const T inv = fdiv(T(1), b.z - a.z);
        const P3<T> pl = at_plane(a, b, sat01((lo - a.z) * inv), 2, lo);
        const P3<T> ph = at_plane(a, b, sat01((hi - a.z) * inv), 2, hi);
        // the part below lo: whole edge, or from an endpoint to pl
        const P3<T> ba = a_lo ? a : pl, bb = b_lo ? b : pl;
        below += (a_lo || b_lo) ? fan_const(ba, bb, lo, l0, lx, ly) : T(0);
        const P3<T> ua = a_hi ? a : ph, ub = b_hi ? b : ph;
        above += (a_hi || b_hi) ? fan_const(ua, ub, hi, l0, lx, ly) : T(0);
        // the part in between (an edge wholly below or above is zero-length here and adds 0)
        const P3<T> na = a_lo ? pl : (a_hi ? ph : a);
        const P3<T> nb = b_lo ? pl : (b_hi ? ph : b);
        mid += fan_mid(na, nb, o, fo, l0, lx, ly);
        xl = (!a_lo && b_lo) ? pl : xl;
        nl = (a_lo && !b_lo) ? pl : nl;
        xh = (!a_hi && b_hi) ? ph : xh;
        nh = (a_hi && !b_hi) ? ph : nh;
    }
    // closing edges: of the part below (entry -> exit on lo), above (on hi), and of the
    // part in between (exit -> entry on each plane)
    below += fan_const(nl, xl, lo, l0, lx, ly);
    above += fan_const(nh, xh, hi, l0, lx, ly);
    mid += fan_mid(xl, nl, o, fo, l0, lx, ly) + fan_mid(xh, nh, o, fo, l0, lx, ly);
    mag += fabs(below) + fabs(above) + fabs(mid);
    return below + above + mid;
}

// ---------------------------------------------------------------------------
// Exact overlap volume of a positively oriented tetrahedron p[4] (cell frame:
// the cell is [0,1)^3) with the cell.  n[f]: outward face normals (unnormalised,
// face f opposite vertex f); (lx, ly): slopes of the plane l (0 for a horizontal
// plane).  err receives the sum of the magnitudes of the terms.
// ---------------------------------------------------------------------------
template <class T>
PSE_HD T overlap_volume(const P3<T> (&p)[4], const P3<T> (&n)[4], T lx, T ly, T &err)
{
    // local frame
    const T cx = T(0.25) * ((p[0].x + p[1].x) + (p[2].x + p[3].x));
    const T cy = T(0.25) * ((p[0].y + p[1].y) + (p[2].y + p[3].y));
    const T cz = T(0.25) * ((p[0].z + p[1].z) + (p[2].z + p[3].z));
    const P3<T> q = mk<T>(floor(fmin(fmax(cx, T(0)), T(1)) * T(256) + T(0.5)) * T(1.0 / 256),
                          floor(fmin(fmax(cy, T(0)), T(1)) * T(256) + T(0.5)) * T(1.0 / 256),
                          floor(fmin(fmax(cz, T(0)), T(1)) * T(256) + T(0.5)) * T(1.0 / 256));
    P3<T> pl[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) pl[i] = sub(p[i], q);
    const T xlo = -q.x, xhi = T(1) - q.x, ylo = -q.y, yhi = T(1) - q.y, zlo = -q.z, zhi = T(1) - q.z;
    // reference plane l: slopes (lx, ly), through the centroid, but held inside the cell's
    // z range at the column centre so that its values stay O(1) near the cell
    const T xc = T(0.5) - q.x, yc = T(0.5) - q.y;
    const T lc = fmin(fmax((cz - q.z) + lx * (xc - (cx - q.x)) + ly * (yc - (cy - q.y)), zlo), zhi);
    const T l0 = lc - lx * xc - ly * yc;

    T vol = T(0), mag = T(0);
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        int ia, ib, ic;
        face_vertices(f, ia, ib, ic);
        const P3<T> a = pick4(pl, ia), b = pick4(pl, ib), c = pick4(pl, ic);
        const T mnx = fmin(a.x, fmin(b.x, c.x)), mxx = fmax(a.x, fmax(b.x, c.x));
        const T mny = fmin(a.y, fmin(b.y, c.y)), mxy = fmax(a.y, fmax(b.y, c.y));
        if (mxx < xlo || mnx >= xhi || mxy < ylo || mny >= yhi) continue;  // outside the column
        const P3<T> nf = (f == 0) ? n[0] : (f == 1) ? n[1] : (f == 2) ? n[2] : n[3];
        if (nf.z == T(0)) continue;  // vertical face: no projected area
        const T mnz = fmin(a.z, fmin(b.z, c.z)), mxz = fmax(a.z, fmax(b.z, c.z));
        // classification tolerance: a few units of rounding of this face's coordinates
        const T cmag = fmax(T(1), fmax(fmax(fmax(fabs(mnx), fabs(mxx)), fmax(fabs(mny), fabs(mxy))),
                                       fmax(fabs(mnz), fabs(mxz))));
        const T tol = T(8) * roundoff<T>() * cmag;
        // anchor of the between-planes region: the local origin projected onto the face plane
        const T sc = fdiv(dot(nf, a), dot(nf, nf));
        const P3<T> o = mk<T>(sc * nf.x, sc * nf.y, sc * nf.z);

        P3<T> A[7], B[7];
        A[0] = a; B[0] = b;
        A[1] = b; B[1] = c;
        A[2] = c; B[2] = a;
        A[3] = B[3] = A[4] = B[4] = mk<T>(T(0), T(0), T(0));
        clip_slab<T, 3>(A, B, 0, xlo, xhi, tol);
        clip_slab<T, 5>(A, B, 1, ylo, yhi, tol);
        vol += split_zslab<T, 7>(A, B, zlo, zhi, tol, l0, lx, ly, o, mag);
    }
    err = mag * T(1.0 / 6.0);
    return vol * T(1.0 / 6.0);
}

// Cyclic relabelling of the axes that brings `axis` to z (orientation preserving).
template <class T>
PSE_HD P3<T> to_axis(const P3<T> &a, int axis)
{
    P3<T> r = a;
    r = (axis == 0) ? mk<T>(a.y, a.z, a.x) : r;
    r = (axis == 1) ? mk<T>(a.z, a.x, a.y) : r;
    return r;
}

// The clip in the frame where the tetrahedron's largest face is the most horizontal one:
// p, n as for overlap_volume; lx, ly: reference slopes in that frame (tet_setup).
template <class T>
PSE_HD T overlap_volume_ax(const P3<T> (&p)[4], const P3<T> (&n)[4], int axis, T lx, T ly, T &err)
{
    P3<T> pa[4], na[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        pa[q] = to_axis(p[q], axis);
        na[q] = to_axis(n[q], axis);
    }
    return overlap_volume<T>(pa, na, lx, ly, err);
}

// Slopes of the reference plane l: the plane of the face whose normal is closest to
// the z axis, unless that plane is steeper than 8 (then l is horizontal).
template <class T>
PSE_HD void ref_slopes(const P3<T> (&n)[4], T &lx, T &ly)
{
    int best = 0;
    T bz = T(-1);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const T n2 = dot(n[f], n[f]);
        const T r = (n2 > T(0)) ? n[f].z * n[f].z / n2 : T(0);
        if (r > bz) { bz = r; best = f; }
    }
    const P3<T> nb = pick4(n, best);
    lx = T(0);
    ly = T(0);
    if (nb.z != T(0)) {
        lx = -nb.x / nb.z;
        ly = -nb.y / nb.z;
    }
    if (!(fabs(lx) <= T(8) && fabs(ly) <= T(8))) {
        lx = T(0);
        ly = T(0);
    }
}

// Outward face normals (face f opposite vertex f) of a positively oriented tetrahedron.
template <class T>
PSE_HD void face_normals(const P3<T> (&v)[4], P3<T> (&n)[4])
{
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        int ia, ib, ic;
        face_vertices(f, ia, ib, ic);
        const P3<T> a = pick4(v, ia), b = pick4(v, ib), c = pick4(v, ic);
        n[f] = cross(sub(b, a), sub(c, a));
    }
}

// float64 6 * signed volume of four vertices
PSE_HD double det6(const P3<double> (&p)[4])
{
    const double ax = p[1].x - p[0].x, ay = p[1].y - p[0].y, az = p[1].z - p[0].z;
    const double bx = p[2].x - p[0].x, by = p[2].y - p[0].y, bz = p[2].z - p[0].z;
    const double cx = p[3].x - p[0].x, cy = p[3].y - p[0].y, cz = p[3].z - p[0].z;
    return ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx);
}

// Overlap volume of a tetrahedron (cell frame, float64 vertices, either orientation)
// with the cell, computed in float64: the guarded clip of the cell-by-cell schedules.  The
// vertices must be the exact ones (not the float32-rounded set the FP32 clip used),
// otherwise the float64 clip only reproduces the rounding of the inputs.
PSE_HD double overlap_volume_fp64(P3<double> (&pd)[4])
{
    if (det6(pd) < 0.0) {
        const P3<double> t = pd[1];
        pd[1] = pd[2];
        pd[2] = t;
    }
    P3<double> nd[4];
    face_normals<double>(pd, nd);
    double lx, ly, err;
    ref_slopes<double>(nd, lx, ly);
    return overlap_volume<double>(pd, nd, lx, ly, err);
}

// ---------------------------------------------------------------------------
// Per-tetrahedron set-up in grid units.
// ---------------------------------------------------------------------------
template <class T>
struct TetSetup {
    P3<T> v[4];     // vertices relative to the base cell corner, positively oriented
    P3<T> n[4];     // outward face normals (face f opposite vertex f)
    T e[4];         // n_f . x <= e_f inside (base-cell frame)
    T pos[4], neg[4];  // sum of positive / negative components of n_f (corner extremes)
    int lo[3], dim[3]; // bounding-box cells relative to the base: [lo, lo + dim)
    double vol6;       // |6 V| in grid units (float64)
    float kappa;       // conditioning estimate (surface * extent / volume)
    int axis;          // the clip integrates along this axis (the largest face's dominant normal axis)
    T lx, ly;          // slopes of the reference plane l in the clip's frame (to_axis)
};

// Returns true if v[1] and v[2] were swapped to make the tetrahedron positively oriented.
template <class T>
PSE_HD bool tet_setup(P3<T> (&v)[4], TetSetup<T> &s)
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
    // divergence axis: the dominant component of the largest face's normal, so that this
    // face (and, for a sliver, its near-parallel partner) is close to horizontal in the
    // clip's frame; thin dimensions are then integrated along the axis, not across it
    {
        int fb = 0;
        T best = T(-1);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const T a2 = dot(s.n[f], s.n[f]);
            fb = (a2 > best) ? f : fb;
            best = (a2 > best) ? a2 : best;
        }
        const P3<T> nb = pick4(s.n, fb);
        const T ax = fabs(nb.x), ay = fabs(nb.y), az = fabs(nb.z);
        s.axis = (az >= ax && az >= ay) ? 2 : (ax >= ay ? 0 : 1);
        P3<T> na[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) na[f] = to_axis(s.n[f], s.axis);
        ref_slopes<T>(na, s.lx, s.ly);
    }
    if constexpr (sizeof(T) == 4) {
        // a threshold test only: float is enough (a volume below float's range gives inf: guarded)
        s.kappa = area2 * sqrtf(lmax2) / (float)s.vol6;
    } else {
        const double denom = s.vol6 > 0.0 ? s.vol6 : 1e-300;
        s.kappa = (float)((double)area2 * sqrt((double)lmax2) / denom);
    }
    return d6 < 0.0;
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

// ---------------------------------------------------------------------------
// The FP32 clip of the warp kernels: overlap_volume<float> above, with the polygon's
// edge slots in shared memory instead of registers.  E is this lane's column of a
// [21][32] float2 array; slot k holds a.xyz, b.xyz in rows 3k .. 3k+2.  The arithmetic and
// its order are those of overlap_volume; only the edge loops stay rolled, so that the
// per-edge code exists once per slab pass and once for the z split.  The
// clip dominates the deposit kernel, whose speed is set by instruction fetch as much as
// by issue: the unrolled clip is 15 copies of the per-edge code.
// ---------------------------------------------------------------------------
// A slot row holds two scalars: float2 for float, double2 for double, and this pair for
// any other scalar type (host checks instantiate the clip with counting types).
template <class T>
struct Slot2 {
    T x, y;
};
template <class T>
struct SlotOf {
    using type = Slot2<T>;
};
template <>
struct SlotOf<float> {
    using type = float2;
};
template <>
struct SlotOf<double> {
    using type = double2;
};
template <class T>
using slot2_t = typename SlotOf<T>::type;

template <class T>
PSE_HD void slot_store(slot2_t<T> *E, int k, const P3<T> &a, const P3<T> &b)
{
    slot2_t<T> *r = E + k * (3 * 32);
    r[0].x = a.x; r[0].y = a.y;
    r[32].x = a.z; r[32].y = b.x;
    r[64].x = b.y; r[64].y = b.z;
}

template <class T>
PSE_HD void slot_load(const slot2_t<T> *E, int k, P3<T> &a, P3<T> &b)
{
    const slot2_t<T> *r = E + k * (3 * 32);
    const slot2_t<T> u = r[0], v = r[32], w = r[64];
    a = mk<T>(u.x, u.y, v.x);
    b = mk<T>(v.y, w.x, w.y);
}

// One slab pass of the rolled clip (clip_slab<3 + 2 AX> of geom.cuh on the slots in E):
// clips slots [0, ne) against lo <= c_AX < hi and appends the two new edges.  The axis is
// a template parameter, so the x and y passes each get their own loop body without
// per-edge axis selects (one more copy of the per-edge code, fewer instructions).
template <int AX, class T>
PSE_HD void slab_pass(slot2_t<T> *E, T lo, T hi, T tol)
{
    constexpr int ne = 3 + 2 * AX;
    const P3<T> z0 = mk<T>(T(0), T(0), T(0));
    P3<T> xl = z0, nl = z0, xh = z0, nh = z0;
#pragma unroll 1
    for (int k = 0; k < ne; ++k) {
        P3<T> ea, eb;
        slot_load<T>(E, k, ea, eb);
        const T ca = AX ? ea.y : ea.x, cb = AX ? eb.y : eb.x;
        const bool a_lo = ca < lo - tol, b_lo = cb < lo - tol;
        const bool a_hi = ca >= hi - tol, b_hi = cb >= hi - tol;
        const T inv = fdiv(T(1), cb - ca);
        const P3<T> pa = at_plane(ea, eb, sat01((lo - ca) * inv), AX, lo);
        const P3<T> ph = at_plane(ea, eb, sat01((hi - ca) * inv), AX, hi);
        const P3<T> na = a_lo ? pa : (a_hi ? ph : ea);
        const P3<T> nb = b_lo ? pa : (b_hi ? ph : eb);
        slot_store<T>(E, k, na, nb);
        xl = (!a_lo && b_lo) ? pa : xl;
        nl = (a_lo && !b_lo) ? pa : nl;
        xh = (!a_hi && b_hi) ? ph : xh;
        nh = (a_hi && !b_hi) ? ph : nh;
    }
    slot_store<T>(E, ne, xl, nl);
    slot_store<T>(E, ne + 1, xh, nh);
}

PSE_HD float overlap_volume_rolled(const P3<float> (&p)[4], const P3<float> (&n)[4], float lx,
                                                       float ly, float &err, float2 *E)
{
    using T = float;
    const T cx = T(0.25) * ((p[0].x + p[1].x) + (p[2].x + p[3].x));
    const T cy = T(0.25) * ((p[0].y + p[1].y) + (p[2].y + p[3].y));
    const T cz = T(0.25) * ((p[0].z + p[1].z) + (p[2].z + p[3].z));
    const P3<T> q = mk<T>(floor(fmin(fmax(cx, T(0)), T(1)) * T(256) + T(0.5)) * T(1.0 / 256),
                          floor(fmin(fmax(cy, T(0)), T(1)) * T(256) + T(0.5)) * T(1.0 / 256),
                          floor(fmin(fmax(cz, T(0)), T(1)) * T(256) + T(0.5)) * T(1.0 / 256));
    P3<T> pl[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) pl[i] = sub(p[i], q);
    const T xlo = -q.x, xhi = T(1) - q.x, ylo = -q.y, yhi = T(1) - q.y, zlo = -q.z, zhi = T(1) - q.z;
    const T xc = T(0.5) - q.x, yc = T(0.5) - q.y;
    const T lc = fmin(fmax((cz - q.z) + lx * (xc - (cx - q.x)) + ly * (yc - (cy - q.y)), zlo), zhi);
    const T l0 = lc - lx * xc - ly * yc;
    const P3<T> z0 = mk<T>(T(0), T(0), T(0));

    T vol = T(0), mag = T(0);
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        int ia, ib, ic;
        face_vertices(f, ia, ib, ic);
        const P3<T> a = pick4(pl, ia), b = pick4(pl, ib), c = pick4(pl, ic);
        const T mnx = fmin(a.x, fmin(b.x, c.x)), mxx = fmax(a.x, fmax(b.x, c.x));
        const T mny = fmin(a.y, fmin(b.y, c.y)), mxy = fmax(a.y, fmax(b.y, c.y));
        if (mxx < xlo || mnx >= xhi || mxy < ylo || mny >= yhi) continue;
        const P3<T> nf = (f == 0) ? n[0] : (f == 1) ? n[1] : (f == 2) ? n[2] : n[3];
        if (nf.z == T(0)) continue;
        const T mnz = fmin(a.z, fmin(b.z, c.z)), mxz = fmax(a.z, fmax(b.z, c.z));
        const T cmag = fmax(T(1), fmax(fmax(fmax(fabs(mnx), fabs(mxx)), fmax(fabs(mny), fabs(mxy))),
                                       fmax(fabs(mnz), fabs(mxz))));
        const T tol = T(8) * roundoff<T>() * cmag;
        const T sc = fdiv(dot(nf, a), dot(nf, nf));
        const P3<T> o = mk<T>(sc * nf.x, sc * nf.y, sc * nf.z);

        slot_store<float>(E, 0, a, b);
        slot_store<float>(E, 1, b, c);
        slot_store<float>(E, 2, c, a);
        // the x and y slab passes (clip_slab<3> then clip_slab<5>)
        slab_pass<0, float>(E, xlo, xhi, tol);
        slab_pass<1, float>(E, ylo, yhi, tol);
        // the z split with the three integrals (split_zslab<7>)
        {
            P3<T> xl = z0, nl = z0, xh = z0, nh = z0;
            T below = T(0), above = T(0), mid = T(0);
            const T fo = o.z - fmaT(lx, o.x, fmaT(ly, o.y, l0));
#pragma unroll 1
            for (int k = 0; k < 7; ++k) {
                P3<T> ea, eb;
                slot_load<float>(E, k, ea, eb);
                const bool a_lo = ea.z < zlo - tol, b_lo = eb.z < zlo - tol;
                const bool a_hi = ea.z >= zhi - tol, b_hi = eb.z >= zhi - tol;
                const T inv = fdiv(T(1), eb.z - ea.z);
                const P3<T> pa = at_plane(ea, eb, sat01((zlo - ea.z) * inv), 2, zlo);
                const P3<T> ph = at_plane(ea, eb, sat01((zhi - ea.z) * inv), 2, zhi);
                const P3<T> ba = a_lo ? ea : pa, bb = b_lo ? eb : pa;
                below += (a_lo || b_lo) ? fan_const(ba, bb, zlo, l0, lx, ly) : T(0);
                const P3<T> ua = a_hi ? ea : ph, ub = b_hi ? eb : ph;
                above += (a_hi || b_hi) ? fan_const(ua, ub, zhi, l0, lx, ly) : T(0);
                const P3<T> na = a_lo ? pa : (a_hi ? ph : ea);
                const P3<T> nb = b_lo ? pa : (b_hi ? ph : eb);
                mid += fan_mid(na, nb, o, fo, l0, lx, ly);
                xl = (!a_lo && b_lo) ? pa : xl;
                nl = (a_lo && !b_lo) ? pa : nl;
                xh = (!a_hi && b_hi) ? ph : xh;
                nh = (a_hi && !b_hi) ? ph : nh;
            }
            below += fan_const(nl, xl, zlo, l0, lx, ly);
            above += fan_const(nh, xh, zhi, l0, lx, ly);
            mid += fan_mid(xl, nl, o, fo, l0, lx, ly) + fan_mid(xh, nh, o, fo, l0, lx, ly);
            mag += fabs(below) + fabs(above) + fabs(mid);
            vol += below + above + mid;
        }
    }
    err = mag * T(1.0 / 6.0);
    return vol * T(1.0 / 6.0);
}

}  // namespace pse
