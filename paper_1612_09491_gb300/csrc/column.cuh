// column.cuh -- the column clip of the warp kernels: the overlap volumes of a tetrahedron
// with a run of cells stacked along its divergence axis, from one x/y clip per face
// (geom.cuh holds the per-cell clips it builds on).  Templated on the scalar type: float
// for the FP32 pass, double for guarded tetrahedra (from their exact vertices).
#pragma once

#include "geom.cuh"

namespace pse {

// ---------------------------------------------------------------------------
// Column clip: the overlap volumes of a tetrahedron with a run of up to KW cells stacked
// along the divergence axis (one column of the clip frame), from one x/y clip per face.
//
// With the same field as overlap_volume, the volume of T below a level z = c inside the
// column is
//
//   B(c) = Σ_f  ∫∫_{Q_f} (min(z_f(x,y), c) - l(x,y)) dx dy          (signed per face)
//
// where Q_f is face f's projection clipped to the column; the reference plane l cancels
// over the closed surface for every c, so each level may be evaluated with it.  The cells
// of the column are the slabs between consecutive integer levels, vol_j = B(c_{j+1}) -
// B(c_j), so the x and y slab passes of a face are shared by all cells of the run and
// every interior level serves the two cells beside it.  Per face and level c:
//   * face entirely above c:   ∫(c - l)           = (3c X - Y)/6 with face sums X, Y;
//   * face entirely below c:   ∫(z - l)           = M/6, the face's own moment;
//   * face crossing c:         M/6 - ∫(z - c)_+, the last term a fan of triangles from a
//     point o_c of the face plane on the line z = c, over the parts of the polygon's
//     edges above c.  The fan's triangles along the cut line are degenerate (o_c lies on
//     it), so the cut edge need not be formed, and the sum is continuous in the vertices.
// o_c is the foot of the perpendicular from the local origin onto that line in the xy
// plane; the line crosses the face inside the tetrahedron's bounding box, so o_c stays
// within a few cells of the origin.
// ---------------------------------------------------------------------------
template <class T>
struct FaceSums {
    T m6;          // 6 ∫ (z - l) over the clipped face polygon (signed by orientation)
    T x2;          // Σ cross_xy(a, b) over its edges (twice the signed projected area)
    T y6;          // Σ cross_xy(a, b) (l(0) + l(a) + l(b)): 6 ∫ l = y6, 6 ∫ c = 3 c x2
    T zmin, zmax;  // z range of the polygon's vertices
};

// y slab pass of the column clip: slab_pass<1> on the slots in E, and the face sums of the
// clipped polygon (its surviving edges and the two new ones on the y planes).
template <class T>
PSE_HD void yslab_sums(slot2_t<T> *E, T lo, T hi, T tol, const P3<T> &o, T fo, T l0, T lx, T ly, FaceSums<T> &I)
{
    constexpr int ne = 5;
    const P3<T> z0 = mk<T>(T(0), T(0), T(0));
    P3<T> xl = z0, nl = z0, xh = z0, nh = z0;
    T m6 = T(0), x2 = T(0), y6 = T(0);
    T zmn = T(1e30), zmx = T(-1e30);  // an empty polygon keeps this range
#pragma unroll 1
    for (int k = 0; k < ne; ++k) {
        P3<T> ea, eb;
        slot_load<T>(E, k, ea, eb);
        const bool a_lo = ea.y < lo - tol, b_lo = eb.y < lo - tol;
        const bool a_hi = ea.y >= hi - tol, b_hi = eb.y >= hi - tol;
        const T inv = fdiv(T(1), eb.y - ea.y);
        const P3<T> pa = at_plane(ea, eb, sat01((lo - ea.y) * inv), 1, lo);
        const P3<T> ph = at_plane(ea, eb, sat01((hi - ea.y) * inv), 1, hi);
        const P3<T> na = a_lo ? pa : (a_hi ? ph : ea);
        const P3<T> nb = b_lo ? pa : (b_hi ? ph : eb);
        slot_store<T>(E, k, na, nb);
        xl = (!a_lo && b_lo) ? pa : xl;
        nl = (a_lo && !b_lo) ? pa : nl;
        xh = (!a_hi && b_hi) ? ph : xh;
        nh = (a_hi && !b_hi) ? ph : nh;
        // a dropped edge has zero length: it adds nothing to the sums
        const T cr = cross_xy(na, nb);
        m6 += fan_mid(na, nb, o, fo, l0, lx, ly);
        x2 += cr;
        y6 += cr * fmaT(T(3), l0, fmaT(lx, na.x + nb.x, ly * (na.y + nb.y)));
        // z range over edges of nonzero length (dropped edges carry no vertex of the polygon)
        const bool live = na.x != nb.x || na.y != nb.y || na.z != nb.z;
        zmn = live ? fmin(zmn, fmin(na.z, nb.z)) : zmn;
        zmx = live ? fmax(zmx, fmax(na.z, nb.z)) : zmx;
    }
    slot_store<T>(E, ne, xl, nl);
    slot_store<T>(E, ne + 1, xh, nh);
    // the new edges join points that already bound surviving edges: they change no z range
    {
        const T c1 = cross_xy(xl, nl), c2 = cross_xy(xh, nh);
        m6 += fan_mid(xl, nl, o, fo, l0, lx, ly) + fan_mid(xh, nh, o, fo, l0, lx, ly);
        x2 += c1 + c2;
        y6 += c1 * fmaT(T(3), l0, fmaT(lx, xl.x + nl.x, ly * (xl.y + nl.y))) +
              c2 * fmaT(T(3), l0, fmaT(lx, xh.x + nh.x, ly * (xh.y + nh.y)));
    }
    I.m6 = m6;
    I.x2 = x2;
    I.y6 = y6;
    I.zmin = zmn;
    I.zmax = zmx;
}

// 6 ∫ (z - c)_+ over the polygon in the 7 slots of E: fan from (ox, oy), a point of the face
// plane at height c, over the parts of the edges above c.
template <class T>
PSE_HD T level_fan(const slot2_t<T> *E, T c, T ox, T oy)
{
    T g = T(0);
#pragma unroll 1
    for (int k = 0; k < 7; ++k) {
        P3<T> ea, eb;
        slot_load<T>(E, k, ea, eb);
        const bool a_up = ea.z > c, b_up = eb.z > c;
        const T t = (c - ea.z) * fdiv(T(1), eb.z - ea.z);
        const T px = fmaT(t, eb.x - ea.x, ea.x), py = fmaT(t, eb.y - ea.y, ea.y);
        const T ax = (a_up ? ea.x : px) - ox, ay = (a_up ? ea.y : py) - oy;
        const T bx = (b_up ? eb.x : px) - ox, by = (b_up ? eb.y : py) - oy;
        const T fa = a_up ? ea.z - c : T(0), fb = b_up ? eb.z - c : T(0);
        const T cr = mul_rn(ax, by) - mul_rn(ay, bx);
        g += (a_up || b_up) ? cr * (fa + fb) : T(0);
    }
    return g;
}

// The tetrahedron of a run given as arrays (clip frame, relative to the run's first cell).
template <class T>
struct TetArrays {
    const P3<T> *p, *n;
    PSE_HD P3<T> vtx(int i) const { return p[i]; }
    PSE_HD P3<T> nrm(int f) const { return n[f]; }
};

// The local frame of one run: origin q (the centroid held in the run and rounded to 1/256,
// so the cell planes and the levels c_j = j - q.z stay exact), the reference plane l(x, y) =
// l0 + lx x + ly y held inside the run's z range at the column centre, the run length K and
// the first level evaluated, j0 (0 if the tetrahedron may reach below the run, else 1).
template <class T>
struct RunFrame {
    T qx, qy, qz, l0, lx, ly;
    int K, j0;
};

template <class T, class Src>
PSE_HD RunFrame<T> run_frame(const Src &src, T lx, T ly, int K, bool lo_open)
{
    const P3<T> p0 = src.vtx(0), p1 = src.vtx(1), p2 = src.vtx(2), p3 = src.vtx(3);
    const T cx = T(0.25) * ((p0.x + p1.x) + (p2.x + p3.x));
    const T cy = T(0.25) * ((p0.y + p1.y) + (p2.y + p3.y));
    const T cz = T(0.25) * ((p0.z + p1.z) + (p2.z + p3.z));
    const T kf = (T)K;
    RunFrame<T> F;
    F.qx = floor(fmin(fmax(cx, T(0)), T(1)) * T(256) + T(0.5)) * T(1.0 / 256);
    F.qy = floor(fmin(fmax(cy, T(0)), T(1)) * T(256) + T(0.5)) * T(1.0 / 256);
    F.qz = floor(fmin(fmax(cz, T(0)), kf) * T(256) + T(0.5)) * T(1.0 / 256);
    const T xc = T(0.5) - F.qx, yc = T(0.5) - F.qy;
    const T lc = fmin(fmax((cz - F.qz) + lx * (xc - (cx - F.qx)) + ly * (yc - (cy - F.qy)), -F.qz), kf - F.qz);
    F.l0 = lc - lx * xc - ly * yc;
    F.lx = lx;
    F.ly = ly;
    F.K = K;
    F.j0 = lo_open ? 0 : 1;
    return F;
}

// Whether face f can reach the run's column (its projection's bounding box meets the column
// and it is not vertical).
template <class T, class Src>
PSE_HD bool face_meets_column(const Src &src, int f, const RunFrame<T> &F)
{
    int ia, ib, ic;
    face_vertices(f, ia, ib, ic);
    const P3<T> a = src.vtx(ia), b = src.vtx(ib), c = src.vtx(ic);
    const T mnx = fmin(a.x, fmin(b.x, c.x)) - F.qx, mxx = fmax(a.x, fmax(b.x, c.x)) - F.qx;
    const T mny = fmin(a.y, fmin(b.y, c.y)) - F.qy, mxy = fmax(a.y, fmax(b.y, c.y)) - F.qy;
    if (mxx < -F.qx || mnx >= T(1) - F.qx || mxy < -F.qy || mny >= T(1) - F.qy) return false;
    return src.nrm(f).z != T(0);
}

// One face of a run: the x and y slab passes (the clipped polygon is left in the 7 slots of
// E), then 6 x its term of B(c_j) for the levels j0 .. K by the closed forms (a level the
// face straddles gets the "below" form m6; the fan of its part above the level is subtracted
// afterwards, see level_fan), its z range, its moment, and the straddled levels jlo .. jhi
// (empty when jlo > jhi) with the plane data their fans need.
template <int KW, class T>
struct FaceRun {
    T k6[KW + 1];
    T zmin, zmax, m6;
    int jlo, jhi;
    T nx, ny, nz, ef;  // face plane n . x = ef in the local frame
};

template <int KW, class T, class Src>
PSE_HD void face_run(const Src &src, int f, const RunFrame<T> &F, slot2_t<T> *E, FaceRun<KW, T> &R)
{
    int ia, ib, ic;
    face_vertices(f, ia, ib, ic);
    const P3<T> q = mk<T>(F.qx, F.qy, F.qz);
    const P3<T> a = sub(src.vtx(ia), q), b = sub(src.vtx(ib), q), c = sub(src.vtx(ic), q);
    const P3<T> nf = src.nrm(f);
    const T mnx = fmin(a.x, fmin(b.x, c.x)), mxx = fmax(a.x, fmax(b.x, c.x));
    const T mny = fmin(a.y, fmin(b.y, c.y)), mxy = fmax(a.y, fmax(b.y, c.y));
    const T mnz = fmin(a.z, fmin(b.z, c.z)), mxz = fmax(a.z, fmax(b.z, c.z));
    const T cmag = fmax(T(1), fmax(fmax(fmax(fabs(mnx), fabs(mxx)), fmax(fabs(mny), fabs(mxy))),
                                   fmax(fabs(mnz), fabs(mxz))));
    const T tol = T(8) * roundoff<T>() * cmag;
    const T ef = dot(nf, a);
    const T sc = fdiv(ef, dot(nf, nf));
    const P3<T> o = mk<T>(sc * nf.x, sc * nf.y, sc * nf.z);
    const T fo = o.z - fmaT(F.lx, o.x, fmaT(F.ly, o.y, F.l0));

    slot_store<T>(E, 0, a, b);
    slot_store<T>(E, 1, b, c);
    slot_store<T>(E, 2, c, a);
    slab_pass<0, T>(E, -F.qx, T(1) - F.qx, tol);
    FaceSums<T> I;
    yslab_sums<T>(E, -F.qy, T(1) - F.qy, tol, o, fo, F.l0, F.lx, F.ly, I);

    // levels the polygon straddles: jlo .. jhi (c_j - zmin > 0 and zmax - c_j > 0)
    const T kf = (T)F.K;
    const T flo = fmin(fmax(floor(I.zmin + F.qz) + T(1), T(F.j0)), kf + T(1));
    const T fhi = fmin(fmax(ceil(I.zmax + F.qz) - T(1), T(-1)), kf);
    R.jlo = (int)flo;
    R.jhi = (int)fhi;
    // closed forms: below jlo the face is above the level; from jlo on it is (at first taken
    // as) below it
#pragma unroll
    for (int j = 0; j <= KW; ++j) {
        const T cj = (T)j - F.qz;
        const T v = (j < R.jlo) ? fmaT(T(3) * cj, I.x2, -I.y6) : I.m6;
        R.k6[j] = (j >= F.j0 && j <= F.K) ? v : T(0);
    }
    R.zmin = I.zmin;
    R.zmax = I.zmax;
    R.m6 = I.m6;
    R.nx = nf.x;
    R.ny = nf.y;
    R.nz = nf.z;
    R.ef = ef;
}

// The anchor of a level fan: the point of the face plane at height c nearest the local
// origin in the xy plane.
template <class T>
PSE_HD void fan_anchor(T nx, T ny, T nz, T ef, T c, T &ox, T &oy)
{
    const T s = fmaT(-nz, c, ef) * fdiv(T(1), fmaT(nx, nx, ny * ny));
    ox = s * nx;
    oy = s * ny;
}

// Cell volumes of a run from the level sums S[j] = 6 B(c_j): levels at or below the
// tetrahedron's lowest point in the column hold exactly 0, and levels at or above its highest
// point the column's whole volume, so they are set so rather than left to the rounding of
// terms that cancel; then vol_j = (S[j+1] - S[j]) / 6.
template <int KW, class T>
PSE_HD void column_finish(const RunFrame<T> &F, T (&S)[KW + 1], T colmin, T colmax, T msum, T (&vol)[KW])
{
#pragma unroll
    for (int j = 0; j <= KW; ++j) {
        const T cj = (T)j - F.qz;
        S[j] = (cj <= colmin) ? T(0) : ((cj >= colmax) ? msum : S[j]);
    }
#pragma unroll
    for (int j = 0; j < KW; ++j) vol[j] = (S[j + 1] - S[j]) * T(1.0 / 6.0);
}

// Overlap volumes of a positively oriented tetrahedron (clip frame, relative to the first
// cell of the run: the run is [0,1)^2 x [0,K), K <= KW) with the K cells of the run.  src
// gives vertex i (src.vtx(i)) and the outward normal of face f (src.nrm(f)), read when
// needed; (lx, ly): reference slopes.  lo_open: the tetrahedron may reach below the run (a
// run that starts above its bounding box's first layer); otherwise B(0) is exactly 0.
// E: this lane's edge slots (float2 rows with a stride of 32).
template <int KW, class T, class Src>
PSE_HD void column_volumes(const Src &src, T lx, T ly, int K, bool lo_open, T (&vol)[KW], slot2_t<T> *E)
{
    const RunFrame<T> F = run_frame<T>(src, lx, ly, K, lo_open);
    // S[j]: 6 B(c_j), c_j = j - q.z, j = 0 .. KW (levels past K are unused)
    T S[KW + 1];
#pragma unroll
    for (int j = 0; j <= KW; ++j) S[j] = T(0);
    // the tetrahedron's z range inside the column, and 6 x its volume there
    T colmin = T(1e30), colmax = T(-1e30), msum = T(0);
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        if (!face_meets_column<T>(src, f, F)) continue;
        FaceRun<KW, T> R;
        face_run<KW, T>(src, f, F, E, R);
#pragma unroll 1
        for (int j = R.jlo; j <= R.jhi; ++j) {  // straddled levels: subtract the part above
            const T cj = (T)j - F.qz;
            T ox, oy;
            fan_anchor<T>(R.nx, R.ny, R.nz, R.ef, cj, ox, oy);
            const T g = level_fan<T>(E, cj, ox, oy);
#pragma unroll
            for (int i = 0; i <= KW; ++i) R.k6[i] -= (i == j) ? g : T(0);
        }
#pragma unroll
        for (int j = 0; j <= KW; ++j) S[j] += R.k6[j];
        colmin = fmin(colmin, R.zmin);
        colmax = fmax(colmax, R.zmax);
        msum += R.m6;
    }
    column_finish<KW, T>(F, S, colmin, colmax, msum, vol);
}

}  // namespace pse
