"""Exact rational volumes by Lasserre's facet recursion -- TEST INFRASTRUCTURE ONLY.

Used to pin the C oracle, never by the product.  The algorithm is deliberately
different from the oracle's recursive tetrahedron split (Sec. 6.3): the
polytope {x : a_i . x <= b_i} has volume

    vol_d(P) = (1/d) * sum_i  b_i / |a_ij| * vol_{d-1}(proj_j F_i)

(J.B. Lasserre, "An analytical expression and an algorithm for the volume of a
convex polyhedron in R^n", JOTA 39, 1983): the pyramid decomposition of P from
the origin over its facets F_i, with each facet measured through its projection
along a coordinate j where a_ij != 0, so everything stays rational.  The
recursion bottoms out at intervals in 1D.  With ``fractions.Fraction`` inputs the
result is exact.
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Sequence, Tuple

Constraint = Tuple[List[Fraction], Fraction]  # (a, b) meaning a . x <= b


def _vol(cons: Sequence[Constraint], d: int) -> Fraction:
    # drop constraints with a == 0 (or detect emptiness)
    live: List[Constraint] = []
    for a, b in cons:
        if all(c == 0 for c in a):
            if b < 0:
                return Fraction(0)
            continue
        live.append((list(a), b))
    if d == 1:
        lo, hi = None, None
        for a, b in live:
            x = b / a[0]
            if a[0] > 0:
                hi = x if hi is None or x < hi else hi
            else:
                lo = x if lo is None or x > lo else lo
        if lo is None or hi is None:
            raise ValueError("unbounded polytope")
        return max(Fraction(0), hi - lo)
    total = Fraction(0)
    for i, (ai, bi) in enumerate(live):
        j = max(range(d), key=lambda k: abs(ai[k]))
        aij = ai[j]
        sub: List[Constraint] = []
        empty = False
        for l, (al, bl) in enumerate(live):
            if l == i:
                continue
            f = al[j] / aij
            c = [al[k] - f * ai[k] for k in range(d) if k != j]
            r = bl - f * bi
            if all(x == 0 for x in c):
                if r < 0:
                    empty = True
                    break
                if r == 0 and f > 0 and l < i:
                    # same hyperplane, same orientation: the facet belongs to the first copy
                    empty = True
                    break
                continue
            sub.append((c, r))
        if empty:
            continue
        fv = _vol(sub, d - 1)
        if fv != 0:
            total += bi / abs(aij) * fv
    return total / d


def tet_halfspaces(tet: Sequence[Sequence[Fraction]]) -> List[Constraint]:
    """The four half-spaces n_f . x <= e_f of a non-degenerate tetrahedron."""
    p = [[Fraction(c) for c in v] for v in tet]
    out: List[Constraint] = []
    for f in range(4):
        q = [p[k] for k in range(4) if k != f]
        u = [q[1][k] - q[0][k] for k in range(3)]
        w = [q[2][k] - q[0][k] for k in range(3)]
        n = [u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]]
        e = sum(n[k] * q[0][k] for k in range(3))
        # orient so that the opposite vertex is inside
        if sum(n[k] * p[f][k] for k in range(3)) > e:
            n = [-c for c in n]
            e = -e
        out.append((n, e))
    return out


def box_halfspaces(lo: Sequence[Fraction], hi: Sequence[Fraction]) -> List[Constraint]:
    out: List[Constraint] = []
    for a in range(3):
        e = [Fraction(0)] * 3
        e[a] = Fraction(1)
        out.append((list(e), Fraction(hi[a])))
        m = [Fraction(0)] * 3
        m[a] = Fraction(-1)
        out.append((m, -Fraction(lo[a])))
    return out


def tet_box_volume(tet, lo, hi) -> Fraction:
    """Exact vol(T intersect [lo, hi]) for rational inputs."""
    tet = [[Fraction(c) for c in v] for v in tet]
    return _vol(tet_halfspaces(tet) + box_halfspaces(lo, hi), 3)


def tet_volume(tet) -> Fraction:
    p = [[Fraction(c) for c in v] for v in tet]
    a = [[p[k][c] - p[0][c] for c in range(3)] for k in (1, 2, 3)]
    det = (a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1])
           - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
           + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]))
    return abs(det) / 6
