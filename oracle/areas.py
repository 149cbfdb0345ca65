"""Oracle for the band areas of spherical polygon cells (the zonal-mean step).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
legs may use this module.

What it computes
----------------
A cell is a simple spherical polygon: FP64 vertices v_0 .. v_{m-1} (directions;
|v| need not be 1) joined in order by minor great circle arcs (Sec. 1.2), the
last vertex back to the first, listed counter-clockwise as seen from outside
the sphere (the interior lies to the left of each arc). Ascending latitudes
z_0 < ... < z_{L-1} cut the sphere into bands B_k = {z_k <= z <= z_{k+1}},
k = 0 .. L-2. The band areas are A[k] = area(cell ∩ B_k); parts of the cell
outside [z_0, z_{L-1}] belong to no band. Zonal means (Sec. 1 names them as the
use of arc-latitude intersections) weight a cell field by these areas.

How (the plain definition)
--------------------------
On the unit sphere the area element in longitude and height is dλ dz
(Archimedes: the projection onto the circumscribed cylinder keeps areas). So

    A[k] = integral over z in [z_k, z_{k+1}] of W(z) dz,

with W(z) the total longitude extent of the part of the latitude circle at
height z that lies inside the cell.

W(z) comes from the crossings of that circle with the cell's arcs, i.e. from
Eq. 2.2, taken from oracle.exact in exact integers: the normal, the sign of Q
and the closed on-arc test. Along an arc run from x1 to x2 the direction of
travel at the candidate P(sigma) is n x P, whose z-component is sigma * s
(s = sqrt(Q), after dividing by S2), so sigma = +1 (slot 0) crosses the
circle upwards and sigma = -1 (slot 1) downwards. The interior is on the left
of the direction of travel, so walking east along the circle one enters the
cell at a downward crossing and leaves it at the next upward one; W(z) is the
sum of these eastward stretches. Longitudes are measured from the meridian of
a reference vertex: with P = (U + sigma sqrt(Qi) V) / c exactly, the sine and
cosine of the angle are (alpha + beta sqrt(Qi)) / c for integers alpha, beta,
each correctly rounded by oracle.exact.round_quadratic, so every longitude
difference is accurate relative to itself. A circle that meets no arc is
either wholly inside (the cell contains the pole on the far side of the
circle from the boundary) or wholly outside; the winding number of the
boundary around the z-axis tells which pole, if either, the cell contains.

W is piecewise smooth: it has kinks at the heights of the vertices and
square-root behaviour at the highest or lowest point of an arc, where two
crossings merge. Between consecutive such breakpoints the substitution
z = a + (b - a) sin^2(pi t / 2) makes the integrand smooth in t, and
Gauss-Legendre in t converges quickly (GAUSS_NODES nodes per piece; a piece
is halved until one rule and the rule on the two halves agree to 2^-50).

Conventions (our readings)
--------------------------
* A cell contains at most one pole in its interior; which one is read from the
  winding number of the boundary around the z-axis.
* Degenerate arcs (repeated vertices) and arcs on the equator contribute no
  crossings; W(z) at the finitely many heights where the crossing set changes
  is never evaluated (quadrature nodes lie strictly inside the pieces).

Accuracy: longitudes within a few units of rounding of W(z) itself and an
adaptive quadrature error below 2^-50 relative (checked against rules with
more nodes in the tests), so A[k] is within a few 1e-15 of itself.
"""
from __future__ import annotations

import math

import numpy as np

from . import exact

GAUSS_NODES = 16
TWO_PI = 2.0 * math.pi


def _unit(v):
    v = [float(x) for x in v]
    r = math.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
    return [x / r for x in v]


def _ref_xy(cell):
    """Integer x, y of the first vertex off the poles (the reference meridian)."""
    for v in cell:
        if float(v[0]) != 0.0 or float(v[1]) != 0.0:
            (mx, ex), (my, ey) = exact.dyadic(float(v[0])), exact.dyadic(float(v[1]))
            e = min(x for m, x in ((mx, ex), (my, ey)) if m != 0)
            return ((mx << (ex - e)) if mx else 0, (my << (ey - e)) if my else 0)
    raise ValueError("every vertex of the cell is a pole")


def winding(cell) -> int:
    """Winding number of the boundary around the z-axis (+1: the cell holds the
    north pole, -1: the south pole, 0: neither), from the arcs' longitude steps."""
    tot = 0.0
    m = len(cell)
    for i in range(m):
        a, b = cell[i], cell[(i + 1) % m]
        if (float(a[0]) == 0.0 and float(a[1]) == 0.0) or (float(b[0]) == 0.0 and float(b[1]) == 0.0):
            continue  # a pole has no longitude: an arc from or to it steps none
        cr = float(a[0]) * float(b[1]) - float(a[1]) * float(b[0])
        dt = float(a[0]) * float(b[0]) + float(a[1]) * float(b[1])
        tot += math.atan2(cr, dt)
    return int(round(tot / TWO_PI))


def _crossings(cell, z, R):
    """(longitude from the reference meridian, +1 up / -1 down) of every
    crossing of the circle at height z with the cell's arcs (Eq. 2.2)."""
    out = []
    m = len(cell)
    for i in range(m):
        x1, x2 = cell[i], cell[(i + 1) % m]
        ex = exact.setup(tuple(map(float, x1)), tuple(map(float, x2)), float(z))
        if ex.N == (0, 0, 0) or ex.S2i == 0 or ex.Qi <= 0:
            continue  # degenerate, on the equator, no crossing, or a touch
        for sigma in (1, -1):
            g1, g2 = exact.contained_sign(ex, sigma)
            if g1 < 0 or g2 < 0:
                continue
            # c * (R x P)_z and c * (R . P)_xy as alpha + beta * sqrt(Qi)
            a_s = R[0] * ex.U[1] - R[1] * ex.U[0]
            b_s = R[0] * ex.V[1] - R[1] * ex.V[0]
            a_c = R[0] * ex.U[0] + R[1] * ex.U[1]
            b_c = R[0] * ex.V[0] + R[1] * ex.V[1]
            sn = exact.round_quadratic(a_s, sigma * b_s, ex.Qi, ex.c)
            cs = exact.round_quadratic(a_c, sigma * b_c, ex.Qi, ex.c)
            out.append((math.atan2(sn, cs), sigma))
    return out


def width(cell, z, R=None, w=None, zlo=None, zhi=None) -> float:
    """W(z): longitude extent of the cell's part of the circle at height z."""
    if R is None:
        R = _ref_xy(cell)
    xs = _crossings(cell, z, R)
    if not xs:
        if w is None:
            w = winding(cell)
        if zlo is None or zhi is None:
            bz = breakpoints(cell)
            zlo, zhi = min(bz), max(bz)
        # the boundary lies wholly below (or above) the circle
        if w == 1 and z > zhi:
            return TWO_PI
        if w == -1 and z < zlo:
            return TWO_PI
        return 0.0
    xs.sort()
    n = len(xs)
    total = 0.0
    for j in range(n):
        lam, d = xs[j]
        lam2, d2 = xs[(j + 1) % n]
        if d == d2:
            raise ValueError(f"crossings at height {z!r} do not alternate")
        if d == -1:
            step = lam2 - lam
            if step <= 0.0:
                step += TWO_PI
            total += step
    return total


def breakpoints(cell):
    """Heights where W has a kink or a square-root point: the vertices and the
    highest / lowest points of arcs that pass them (decided exactly)."""
    zs = [_unit(v)[2] for v in cell]
    m = len(cell)
    for i in range(m):
        x1, x2 = cell[i], cell[(i + 1) % m]
        ex = exact.setup(tuple(map(float, x1)), tuple(map(float, x2)), 0.0)
        N = ex.N
        S2 = N[0] * N[0] + N[1] * N[1]
        if N == (0, 0, 0) or S2 == 0:
            continue
        # highest point of the great circle, up to a positive factor
        top = (-N[0] * N[2], -N[1] * N[2], S2)
        for sgn in (1, -1):
            a = tuple(sgn * t for t in top)
            t1 = exact._dot(exact._cross(ex.X1, a), N)
            t2 = exact._dot(exact._cross(a, ex.X2), N)
            if t1 >= 0 and t2 >= 0:
                S3 = S2 + N[2] * N[2]
                zs.append(sgn * math.sqrt(S2 / S3))
    return zs


def _gauss(n):
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def _piece(Wf, a, b, tq, wq, depth=0):
    """Integral of W over [a, b] (no breakpoint inside): Gauss-Legendre after
    z = a + (b - a) sin^2(pi t / 2), accepted when it agrees with the sum over
    the two halves to 2^-50 relative (else each half recursively, depth <= 8)."""

    def gl(lo, hi):
        h = hi - lo
        acc = 0.0
        for t, wt in zip(tq, wq):
            s = math.sin(0.5 * math.pi * t)
            z = lo + h * s * s
            if lo < z < hi:
                acc += wt * Wf(z) * math.sin(math.pi * t)
        return acc * h * 0.5 * math.pi

    m = 0.5 * (a + b)
    whole = gl(a, b)
    halves = gl(a, m) + gl(m, b)
    if depth >= 8 or not (a < m < b) or abs(whole - halves) <= 2.0 ** -50 * abs(halves):
        return halves
    return _piece(Wf, a, m, tq, wq, depth + 1) + _piece(Wf, m, b, tq, wq, depth + 1)


def band_areas(cell, lat_z, nodes: int = GAUSS_NODES):
    """A[k] = area(cell ∩ [z_k, z_{k+1}]) for k = 0 .. L-2 (a list of floats)."""
    lat = [float(z) for z in lat_z]
    R = _ref_xy(cell)
    w = winding(cell)
    bz = breakpoints(cell)
    zlo, zhi = min(bz), max(bz)  # the boundary's z-extent
    bps = sorted(set(bz + [-1.0, 1.0]))
    tq, wq = _gauss(nodes)

    def Wf(z):
        return width(cell, z, R, w, zlo, zhi)

    out = []
    for k in range(len(lat) - 1):
        a0, b0 = lat[k], lat[k + 1]
        cuts = [a0] + [z for z in bps if a0 < z < b0] + [b0]
        total = 0.0
        for a, b in zip(cuts[:-1], cuts[1:]):
            if not b > a:
                continue
            if a >= zhi or b <= zlo:
                # beyond the boundary W is constant: 2 pi inside a polar cap, else 0
                if (w == 1 and a >= zhi) or (w == -1 and b <= zlo):
                    total += TWO_PI * (b - a)
                continue
            total += _piece(Wf, a, b, tq, wq)
        out.append(total)
    return out


def cell_area(cell) -> float:
    """Area of the cell by the triangle fan from v_0 with the Van Oosterom and
    Strackee formula tan(E / 2) = a . (b x c) / (1 + a.b + b.c + c.a) for each
    triangle's spherical excess E (a textbook identity, independent of the
    band integral above). Numerator and denominator are evaluated exactly in
    rationals on the normalised FP64 vertices, so each E is accurate relative
    to itself even for tiny triangles."""
    from fractions import Fraction

    vs = [[Fraction(x) for x in _unit(v)] for v in cell]

    def dot(p, q):
        return p[0] * q[0] + p[1] * q[1] + p[2] * q[2]

    def cross(p, q):
        return (p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2], p[0] * q[1] - p[1] * q[0])

    a = vs[0]
    tot = 0.0
    for i in range(1, len(vs) - 1):
        b, c = vs[i], vs[i + 1]
        num = dot(a, cross(b, c))
        den = 1 + dot(a, b) + dot(b, c) + dot(c, a)
        tot += 2.0 * math.atan2(float(num), float(den))
    return tot


def _batch_worker(args):
    cells, lat = args
    return [band_areas(c, lat) for c in cells]


def band_areas_batch(cells, lat_z, processes: int | None = None):
    """band_areas for a list of cells (a list of lists), optionally in a spawn pool."""
    lat = [float(z) for z in lat_z]
    if processes is None or processes <= 1 or len(cells) < 8:
        return _batch_worker((cells, lat))
    import multiprocessing as mp
    chunk = max(1, (len(cells) + processes * 4 - 1) // (processes * 4))
    jobs = [(cells[i:i + chunk], lat) for i in range(0, len(cells), chunk)]
    with mp.get_context("spawn").Pool(processes) as pool:
        return [r for part in pool.map(_batch_worker, jobs) for r in part]


def zonal_sums(cells, field, lat_z, areas=None):
    """Per band: (sum_c f_c A[c, k], sum_c A[c, k]); the zonal mean is their ratio."""
    if areas is None:
        areas = band_areas_batch(cells, lat_z)
    nb = len(lat_z) - 1
    fa = [0.0] * nb
    aa = [0.0] * nb
    for f, row in zip(field, areas):
        for k in range(nb):
            fa[k] += float(f) * row[k]
            aa[k] += row[k]
    return fa, aa
