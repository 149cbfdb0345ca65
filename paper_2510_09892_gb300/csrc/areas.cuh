// The per-cell geometry of the band-area call (areas.cu): the mesh view, the
// boundary integral over arc pieces (Green's theorem in longitude and height),
// the fan of spherical triangles, and the fan-plus-sliver area of a cell cut
// by one latitude. These functions build for the host too (tests), with the
// status flags set by a plain OR there; the device code is unchanged.
#pragma once
#include <stdint.h>

#include "common.cuh"
#include "intersect.cuh"
#include "ranges.cuh"

namespace sphx {

// status flags: an atomic OR on the device, a plain one in a host build
EFT_HD void flag_status(unsigned *status, unsigned bits) {
#if defined(__CUDA_ARCH__)
    atomicOr(status, bits);
#else
    *status |= bits;
#endif
}

// position of the lowest set bit, 1-based (0 for none)
EFT_HD int ffs_hd(unsigned x) {
#if defined(__CUDA_ARCH__)
    return __ffs(x);
#else
    return __builtin_ffs((int)x);
#endif
}

constexpr double kTwoPi = 6.283185307179586476925286766559;
// a point this close to the z-axis (|xy| < 2^-40) counts as a pole: its
// computed longitude would be rounding noise
constexpr double kPoleRho = 9.094947017729282e-13;

struct Mesh {
    const double *nodes;
    int64_t n_nodes;
    const int64_t *face_offsets;
    const int32_t *face_nodes;
    int64_t n_face_nodes, n_faces;
    const double *lat;
    int64_t L;
    unsigned *status;
    // the nodes normalised by unit(), one vector per node, when the call made
    // that copy (unit_nodes_kernel); else the routines normalise each node of
    // a cell as they read it
    const double *unit_nodes = nullptr;
};

// node range [s, e) of cell f in face_nodes; false (status flagged) if invalid
EFT_HD bool cell_span(const Mesh &m, int64_t f, int64_t &s, int64_t &e) {
    s = m.face_offsets[f];
    e = m.face_offsets[f + 1];
    if (s < 0 || e < s || e > m.n_face_nodes) {
        flag_status(m.status, kStatusInvalid);
        return false;
    }
    return true;
}

// coordinates of node face_nodes[i]; false (status flagged) for an index
// outside the node array
EFT_HD bool node_at(const Mesh &m, int64_t i, double (&v)[3]) {
    const int32_t id = m.face_nodes[i];
    if (id < 0 || (int64_t)id >= m.n_nodes) {
        flag_status(m.status, kStatusInvalid);
        return false;
    }
    const double *p = m.nodes + 3 * (int64_t)id;
    v[0] = p[0];
    v[1] = p[1];
    v[2] = p[2];
    return true;
}

// v / |v|. Mesh nodes are nearly always unit vectors to rounding, q = |v|^2 =
// 1 + d with |d| of a few ulps: then 1 / sqrt(q) = 1 - d/2 + 3 d^2/8 - ..., to
// d^2 (the next term is below 2^-61 for |d| <= 2^-20), takes two FMAs in place
// of the reciprocal square root's sequence on the FP64 pipe
EFT_HD void unit(const double (&v)[3], double (&u)[3]) {
    const double q = fma(v[0], v[0], fma(v[1], v[1], v[2] * v[2]));
    const double d = q - 1.0;
    double r;
    if ((wide::bits_of(d) & 0x7fffffffffffffffull) <= 0x3eb0000000000000ull)  // |d| <= 2^-20
        r = fma(d, fma(0.375, d, -0.5), 1.0);
    else
        r = rsqrt_hd(q);
    u[0] = v[0] * r;
    u[1] = v[1] * r;
    u[2] = v[2] * r;
}

// node face_nodes[i] as a unit vector, given its coordinates `raw` as read
// by node_at (which checked the index): from the normalised copy when there is
// one (the same bits: unit() of the same node), else normalised here
EFT_HD void unit_of(const Mesh &m, int64_t i, const double (&raw)[3], double (&u)[3]) {
    if (m.unit_nodes) {
        const double *p = m.unit_nodes + 3 * (int64_t)m.face_nodes[i];
        u[0] = p[0];
        u[1] = p[1];
        u[2] = p[2];
    } else {
        unit(raw, u);
    }
}

// node face_nodes[i] as a unit vector, for the routines that need no raw
// coordinates (the fans); false (status flagged) for an index outside the
// node array
EFT_HD bool unit_node_at(const Mesh &m, int64_t i, double (&u)[3]) {
    if (m.unit_nodes) {
        const int32_t id = m.face_nodes[i];
        if (id < 0 || (int64_t)id >= m.n_nodes) {
            flag_status(m.status, kStatusInvalid);
            return false;
        }
        const double *p = m.unit_nodes + 3 * (int64_t)id;
        u[0] = p[0];
        u[1] = p[1];
        u[2] = p[2];
        return true;
    }
    double raw[3];
    if (!node_at(m, i, raw)) return false;
    unit(raw, u);
    return true;
}

// a point of an arc with what the boundary integral needs
struct Pt {
    double x, y, z;  // unit vector
    double rho;      // sqrt(x^2 + y^2); 0 at a pole
};

EFT_HD Pt make_pt(double x, double y, double z) {
    Pt p;
    p.x = x;
    p.y = y;
    p.z = z;
    const double r2 = fma(x, x, y * y);
    if (r2 < kPoleRho * kPoleRho)
        p.x = p.y = p.rho = 0.0;
    else
        p.rho = sqrt(r2);
    return p;
}

// a crossing of the latitude z0, whose distance from the axis is
// rho0 = sqrt((1 - z0)(1 + z0)) (per latitude, not per point)
EFT_HD Pt make_pt_at(double x, double y, double z0, double rho0) {
    Pt p;
    p.z = z0;
    if (rho0 < kPoleRho) {
        p.x = p.y = p.rho = 0.0;
    } else {
        p.x = x;
        p.y = y;
        p.rho = rho0;
    }
    return p;
}

EFT_HD double rho_of_lat(double z) { return sqrt((1.0 - z) * (1.0 + z)); }

// angle from the meridian of r to that of p (xy parts of unit vectors), with
// the cross product taken from the differences, r x p = r x (p - r), so that a
// small angle is accurate relative to itself
EFT_HD double delta_lon(double rx, double ry, double x, double y) {
    return atan2(rx * (y - ry) - ry * (x - rx), fma(rx, x, ry * y));
}

// Comparisons of a double with a constant on the integer pipe (GB300 runs
// FP64 instructions, comparisons included, at 2 per SM per clock), each with
// the FP64 comparison's result for every input, NaN and signed zero included.
// x < c for a constant c > 0 (cbits = the bits of c)
EFT_HD bool lt_pos(double x, uint64_t cbits) {
    const uint64_t b = wide::bits_of(x);
    return (b >> 63) ? ((b & 0x7fffffffffffffffull) <= 0x7ff0000000000000ull) : (b < cbits);
}
// |x| <= c for a constant c > 0
EFT_HD bool abs_le(double x, uint64_t cbits) {
    return (wide::bits_of(x) & 0x7fffffffffffffffull) <= cbits;
}
// (x > 0: gt_zero of intersect.cuh)
constexpr uint64_t kBitsHalf = 0x3fe0000000000000ull;    // 0.5
constexpr uint64_t kBitsSeries = 0x3f60000000000000ull;  // 2^-9

// 1 / den for den in [1, 4], the Van Oosterom-Strackee denominators of the
// fan triangles here (both apex dot products at least 1/2): an FP32 seed
// (relative error below 2^-23) and two Newton steps in FP64 (2^-46, then the
// rounding of the last step), four FMAs in place of a division's longer
// sequence on the FP64 pipe
EFT_HD double rcp_den(double den) {
    const double r0 = f64_of_f32_small(wide::rcp32(f32_of(den)));
    const double r1 = fma(r0, fma(-den, r0, 1.0), r0);
    return fma(r1, fma(-den, r1, 1.0), r1);
}

// arctan x by its series x - x^3/3 + x^5/5 - x^7/7, for |x| <= 2^-9 (the
// next term, x^9/9, is below 2^-75 |x|); for |x| <= 2^-18 (the triangles of
// cells below about 0.1 degree) by x - x^3/3 alone (x^5/5 is below 2^-74 |x|)
EFT_HD double atan_small(double x) {
    const double x2 = x * x;
    if ((wide::bits_of(x) & 0x7fffffffffffffffull) <= 0x3ed0000000000000ull)  // |x| <= 2^-18
        return fma(x * x2, -1.0 / 3.0, x);
    return fma(x * x2, fma(x2, fma(x2, -1.0 / 7.0, 1.0 / 5.0), -1.0 / 3.0), x);
}

// Piece p -> q of an arc; the longitude at p is lam + dp. With dl the
// piece's longitude step, h = tan(dl / 2) from the xy cross and dot
// products, and K = (t_p + t_q) / (1 + t_p t_q) for t = tan(latitude / 2)
// = z / (1 + rho), the signed area between the piece and the equator is
// T = 2 atan(K h), and the boundary integral of lambda dz over the piece is
//   (lam + dp) (z_q - z_p) + dl z_q - T,
// added to the band that holds the piece's midpoint. A piece from or to a
// pole runs along a meridian: dl = T = 0. Returns the longitude offset at q.
EFT_HD double add_piece(const Pt &p, const Pt &q, double lam, double dp,
                        const double *lat, int64_t L, int64_t klo,
                        int64_t nb, double *out) {
    if (p.rho == 0.0 && q.rho == 0.0) return dp;
    double dl = 0.0, W = 0.0;  // W = dl z_q - T
    if (p.rho != 0.0 && q.rho != 0.0) {
        const double cr = p.x * (q.y - p.y) - p.y * (q.x - p.x);  // as in delta_lon
        const double den = fma(p.rho, q.rho, fma(p.x, q.x, p.y * q.y));
        const double h = cr / den;
        const double op = 1.0 + p.rho, oq = 1.0 + q.rho;
        const double K = fma(p.z, oq, q.z * op) / fma(op, oq, p.z * q.z);
        if (fabs(h) <= 0.001953125) {
            const double a = atan_small(h);
            dl = 2.0 * a;
            W = 2.0 * fma(q.z, a, -atan_small(K * h));
        } else {
            dl = 2.0 * atan(h);
            W = fma(dl, q.z, -2.0 * atan(K * h));
        }
    }
    const double sx = p.x + q.x, sy = p.y + q.y, sz = p.z + q.z;
    const double zm = sz * rsqrt_hd(fma(sx, sx, fma(sy, sy, sz * sz)));
    const int64_t k = upper_bound_ord(lat, L, ord64(zm)) - 1;
    if (k >= klo && k < klo + nb) out[k - klo] += fma(lam + dp, q.z - p.z, W);
    return dp + dl;
}

// All pieces of the arc a -> b (raw a, b for Eq. 2.2; ua, ub of unit length,
// pa, pb their points) whose longitudes are lam + (offset from a's meridian,
// 0 at a). rho_lat: the latitudes' radii, or null. Returns the offset at b
// (the arc's longitude step).
template <int Mode>
EFT_HD double arc_pieces(const double (&a)[3], const double (&b)[3],
                         const double (&ua)[3], const double (&ub)[3],
                         const Pt &pa, const Pt &pb, double lam,
                         const double *lat, const double *rho_lat, int64_t L,
                         int64_t klo, int64_t nb, double *out) {
    const double nx = ua[1] * ub[2] - ua[2] * ub[1];
    const double ny = ua[2] * ub[0] - ua[0] * ub[2];
    const double nz = ua[0] * ub[1] - ua[1] * ub[0];
    if (nx == 0.0 && ny == 0.0 && nz == 0.0) return 0.0;
    // (n x x)_z, the vertical direction of travel at x: > 0 where the arc rises
    const double ga = nx * ua[1] - ny * ua[0];
    const double gb = nx * ub[1] - ny * ub[0];
    Pt ends[3];
    bool ups[2];
    int nruns;
    ends[0] = pa;
    if ((ga > 0.0 && gb < 0.0) || (ga < 0.0 && gb > 0.0)) {
        // the arc passes the great circle's highest point (rises, then falls)
        // or its lowest; the highest is (-nx nz, -ny nz, nx^2 + ny^2) / (|n| |n_xy|)
        const double S2 = fma(nx, nx, ny * ny);
        const double sc = (ga > 0.0 ? 1.0 : -1.0) / (sqrt(fma(nz, nz, S2)) * sqrt(S2));
        ends[1] = make_pt(-nx * nz * sc, -ny * nz * sc, S2 * sc);
        ends[2] = pb;
        ups[0] = ga > 0.0;
        ups[1] = !ups[0];
        nruns = 2;
    } else {
        ends[1] = pb;
        ups[0] = ub[2] >= ua[2];
        ups[1] = false;
        nruns = 1;
    }
    double d = 0.0;
    for (int r = 0; r < nruns; ++r) {
        const bool up = ups[r];
        const Pt p1 = ends[r + 1];
        const double zl = fmin(ends[r].z, p1.z) - kZWiden, zh = fmax(ends[r].z, p1.z) + kZWiden;
        const int64_t j0 = lower_bound_ord(lat, L, ord64(zl));
        const int64_t j1 = upper_bound_ord_from(lat, L, j0, ord64(zh));
        const int64_t cnt = j1 > j0 ? j1 - j0 : 0;
        const int slot = up ? 0 : 1;
        Pt prev = ends[r];
        for (int64_t i = 0; i <= cnt; ++i) {
            Pt q;
            if (i < cnt) {
                const int64_t j = up ? j0 + i : j1 - 1 - i;
                const double z0 = lat[j];
                PairOut o;
                intersect_pair<Mode>(a, b, z0, o);
                if (!(o.count > 0 && o.hit[slot])) continue;
                q = make_pt_at(o.px[slot], o.py[slot], z0, rho_lat ? rho_lat[j] : rho_of_lat(z0));
            } else {
                q = p1;
            }
            d = add_piece(prev, q, lam, d, lat, L, klo, nb, out);
            prev = q;
        }
    }
    return d;
}

// The area of cell f in each band of its range by the boundary integral
// (Green's theorem in longitude and height, see add_piece and arc_pieces)
template <int Mode>
EFT_HD void green_cell(const Mesh &m, int64_t f,
                       const int32_t *__restrict__ band_lo,
                       const int32_t *__restrict__ band_hi,
                       const long long *__restrict__ offsets,
                       double *__restrict__ areas, int64_t cap,
                       const double *lat, const double *rho_lat) {
    const int64_t klo = band_lo[f];
    const int64_t nb = (int64_t)band_hi[f] - klo;
    if (nb <= 0) return;
    if (klo < 0 || klo + nb > m.L - 1) {
        flag_status(m.status, kStatusInvalid);
        return;
    }
    const long long off = offsets[f];
    if (off < 0 || off + nb > cap) {
        flag_status(m.status, kStatusCapacity);
        return;
    }
    double *out = areas + off;
    for (int64_t j = 0; j < nb; ++j) out[j] = 0.0;
    int64_t s, e;
    if (!cell_span(m, f, s, e) || e - s < 2) return;
    const int64_t nv = e - s;
    // the first node off the poles: lambda = 0 there, and the cut to a
    // pole inside the cell starts there
    int64_t st = -1;
    double a[3], ua[3];
    for (int64_t i = 0; i < nv; ++i) {
        if (!node_at(m, s + i, a)) break;
        unit_of(m, s + i, a, ua);
        if (!(fma(ua[0], ua[0], ua[1] * ua[1]) < kPoleRho * kPoleRho)) {
            st = i;
            break;
        }
    }
    if (st < 0) return;
    Pt pa = make_pt(ua[0], ua[1], ua[2]);
    const double z_st = ua[2];
    double ax = ua[0], ay = ua[1];  // last node off the poles
    double lam_anc = 0.0;           // its unwrapped longitude
    bool ok = true;
    for (int64_t t = 0; t < nv; ++t) {
        int64_t ib = st + t + 1;
        if (ib >= nv) ib -= nv;
        double b[3], ub[3];
        if (!(ok = node_at(m, s + ib, b))) break;
        unit_of(m, s + ib, b, ub);
        const Pt pb = make_pt(ub[0], ub[1], ub[2]);
        const bool a_pole = pa.rho == 0.0, b_pole = pb.rho == 0.0;
        if (a_pole && b_pole) {
            // nothing: a degenerate or pole-to-pole arc
        } else if (a_pole) {
            // a meridian down from the pole: lambda jumps across the pole
            // from the last node off the poles to b's meridian
            const double lam_b = lam_anc + delta_lon(ax, ay, ub[0], ub[1]);
            arc_pieces<Mode>(a, b, ua, ub, pa, pb, lam_b, lat, rho_lat, m.L, klo, nb, out);
            ax = ub[0];
            ay = ub[1];
            lam_anc = lam_b;
        } else {
            const double d =
                arc_pieces<Mode>(a, b, ua, ub, pa, pb, lam_anc, lat, rho_lat, m.L, klo, nb, out);
            if (!b_pole) {
                ax = ub[0];
                ay = ub[1];
                lam_anc += d;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a[c] = b[c];
            ua[c] = ub[c];
        }
        pa = pb;
    }
    if (!ok) return;
    const double w = rint(lam_anc / kTwoPi);
    if (w != 0.0) {
        for (int64_t j = 0; j < nb; ++j) {
            const double zl = lat[klo + j], zh = lat[klo + j + 1];
            const double lo = w > 0.0 ? fmax(zl, z_st) : fmax(zl, -1.0);
            const double hi = w > 0.0 ? fmin(zh, 1.0) : fmin(zh, z_st);
            if (hi > lo) out[j] += kTwoPi * (hi - lo);
        }
    }
}

// The area of a cell that lies inside one band, written to its one band
// entry: the sum of its fan triangles' spherical excesses from node 0, each by
// Van Oosterom and Strackee, tan(E / 2) = a . (b x c) / (1 + a.b + b.c + c.a),
// with the triple product taken as a . ((b - a) x (c - a)) so that small
// triangles keep relative accuracy (atan by its series below 2^-9). Returns
// true, writing nothing, when a node is more than 60 degrees from node 0: the
// fan is not used for such a cell.
EFT_HD bool fan_area(const Mesh &m, int64_t f,
                     const long long *__restrict__ offsets,
                     double *__restrict__ areas, int64_t cap) {
    {
        const long long off = offsets[f];
        if (off < 0 || off + 1 > cap) {
            flag_status(m.status, kStatusCapacity);
            return false;
        }
        int64_t s, e;
        if (!cell_span(m, f, s, e)) return false;
        double v0[3] = {0.0, 0.0, 0.0}, a[3] = {0.0, 0.0, 0.0}, b[3];
        double area = 0.0;
        bool ok = true, far = false;
        if (e - s >= 3) {
            ok = unit_node_at(m, s, v0);
            if (ok) ok = unit_node_at(m, s + 1, a);
            // node 0's dot product with a and the difference a - node 0 carry
            // over from one triangle to the next (b becomes a)
            double oa = fma(v0[0], a[0], fma(v0[1], a[1], v0[2] * a[2]));
            double d1x = a[0] - v0[0], d1y = a[1] - v0[1], d1z = a[2] - v0[2];
            far = lt_pos(oa, kBitsHalf);
            for (int64_t j = s + 2; j < e && ok && !far; ++j) {
                if (!(ok = unit_node_at(m, j, b))) break;
                const double ab = fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
                const double ob = fma(v0[0], b[0], fma(v0[1], b[1], v0[2] * b[2]));
                far = lt_pos(ob, kBitsHalf);
                const double d2x = b[0] - v0[0], d2y = b[1] - v0[1], d2z = b[2] - v0[2];
                const double tri = fma(v0[0], d1y * d2z - d1z * d2y,
                                       fma(v0[1], d1z * d2x - d1x * d2z,
                                           v0[2] * (d1x * d2y - d1y * d2x)));
                const double t = tri * rcp_den(1.0 + oa + ab + ob);
                area += abs_le(t, kBitsSeries) ? atan_small(t) : atan(t);  // half the excess
                a[0] = b[0];
                a[1] = b[1];
                a[2] = b[2];
                oa = ob;
                d1x = d2x;
                d1y = d2y;
                d1z = d2z;
            }
        }
        if (!ok) return false;
        if (far) return true;
        areas[off] = 2.0 * area;  // the doubling is exact: the same as doubling each term
        return false;
    }
}

// Fan area of a sequence of points (unit vectors) from its first, the apex,
// accumulated one point at a time (the points need not sit in an array):
// the same triangles, in the same order and arithmetic, as fan_area's loop.
// ok turns false when a point of a triangle is more than 60 degrees from the
// apex (a sequence of two points has no triangle and no such test).
struct Fan {
    double o[3], a[3];  // the apex and the last point added
    double oa, d1[3];   // the apex's dot product with a, and a - apex
    double half;        // sum of the triangles' half excesses
    int n;              // points added after the apex
    bool ok;
};

EFT_HD void fan_start(Fan &f, const double (&o)[3]) {
    f.o[0] = o[0];
    f.o[1] = o[1];
    f.o[2] = o[2];
    f.half = 0.0;
    f.n = 0;
    f.ok = true;
}

EFT_HD void fan_add(Fan &f, const double (&b)[3]) {
    const double *o = f.o;
    const double ob = fma(o[0], b[0], fma(o[1], b[1], o[2] * b[2]));
    const double d2x = b[0] - o[0], d2y = b[1] - o[1], d2z = b[2] - o[2];
    if (f.n > 0) {
        const double *a = f.a;
        const double ab = fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
        if (lt_pos(f.oa, kBitsHalf) || lt_pos(ob, kBitsHalf)) f.ok = false;
        const double d1x = f.d1[0], d1y = f.d1[1], d1z = f.d1[2];
        const double tri = fma(o[0], d1y * d2z - d1z * d2y,
                               fma(o[1], d1z * d2x - d1x * d2z, o[2] * (d1x * d2y - d1y * d2x)));
        const double t = tri * rcp_den(1.0 + f.oa + ab + ob);
        f.half += abs_le(t, kBitsSeries) ? atan_small(t) : atan(t);
    }
    f.a[0] = b[0];
    f.a[1] = b[1];
    f.a[2] = b[2];
    f.oa = ob;
    f.d1[0] = d2x;
    f.d1[1] = d2y;
    f.d1[2] = d2z;
    ++f.n;
}

// the fan's area (the doubling is exact: the same as doubling each term)
EFT_HD double fan_area_of(const Fan &f) { return 2.0 * f.half; }

constexpr int kPairMaxNodes = 16;  // cells with more nodes take the boundary integral

// A cell in two bands cut by the latitude z_j: with P_u and P_d its upward and
// downward crossings of that latitude (Eq. 2.2 by the chosen mode; slot 0
// crosses upwards along an arc, slot 1 downwards), the part above z_j is
// bounded by the cell's boundary from P_u to P_d and by the latitude arc from
// P_d eastward back to P_u (the interior lies to the left). Its area is the
// fan of (P_u, the nodes between, P_d), closed by the great circle chord from
// P_d to P_u, plus the sliver between that chord and the latitude arc,
//   2 (atan(z tan(dl/2)) - z dl/2) = 2 (atan(z t) - z atan(t)),  t = tan(dl/2),
// whose series for small t is 2 z (1 - z^2) t^3 (1/3 - (1 + z^2) t^2 / 5
// + (1 + z^2 + z^4) t^4 / 7) (next term below 2^-54 of it for t <= 2^-9). The
// part below is the cell's fan area minus that. Returns true, writing nothing,
// for a cell this does not cover (not exactly one upward and one downward
// crossing, more than kPairMaxNodes nodes, a point more than 60 degrees from
// the first): it goes to the boundary integral.
template <int Mode>
EFT_HD bool pair_area(const Mesh &m, int64_t f,
                      const int32_t *__restrict__ band_lo,
                      const long long *__restrict__ offsets,
                      double *__restrict__ areas, int64_t cap,
                      const double *lat) {
    const long long off = offsets[f];
    if (off < 0 || off + 2 > cap) {
        flag_status(m.status, kStatusCapacity);
        return false;
    }
    int64_t s, e;
    if (!cell_span(m, f, s, e)) return false;
    const int nv = (int)(e - s);
    if (nv < 3 || e - s > kPairMaxNodes) return true;
    const double z = lat[band_lo[f] + 1];
    double r[kPairMaxNodes][3];  // the nodes as given
    double v[kPairMaxNodes][3];  // the nodes, unit length
    for (int i = 0; i < nv; ++i) {
        if (!node_at(m, s + i, r[i])) return false;
        unit_of(m, s + i, r[i], v[i]);
    }
    // the arcs whose widened height range reaches z (only they can cross it);
    // evaluated in a loop over this mask, so that a warp runs as many
    // evaluations as its busiest lane needs, not one per arc
    unsigned need = 0u;
    for (int i = 0; i < nv; ++i) {
        const int i1 = i + 1 < nv ? i + 1 : 0;
        double zl, zh;
        const bool ranged = z_range_fp32(r[i], r[i1], zl, zh) || z_range_fp64(r[i], r[i1], zl, zh);
        if (!ranged || (zl <= z && z <= zh)) need |= 1u << i;
    }
    double Pu[3], Pd[3];
    int au = -1, ad = -1, nu = 0, nd = 0;
    bool up_first = false;
    while (need) {
        const int i = ffs_hd(need) - 1;
        need &= need - 1u;
        const int i1 = i + 1 < nv ? i + 1 : 0;
        PairOut o;
        intersect_pair<Mode>(r[i], r[i1], z, o);
        if (o.count > 0) {
            if (o.hit[0]) {
                ++nu;
                au = i;
                Pu[0] = o.px[0];
                Pu[1] = o.py[0];
                Pu[2] = z;
            }
            if (o.hit[1]) {
                ++nd;
                ad = i;
                Pd[0] = o.px[1];
                Pd[1] = o.py[1];
                Pd[2] = z;
            }
            // both on one arc: the one nearer the arc's start comes first
            // (distance from the start grows along a minor arc)
            if (o.hit[0] && o.hit[1]) {
                const double *u = v[i];
                const double du = (Pu[0] - u[0]) * (Pu[0] - u[0]) + (Pu[1] - u[1]) * (Pu[1] - u[1]) +
                                  (z - u[2]) * (z - u[2]);
                const double dd = (Pd[0] - u[0]) * (Pd[0] - u[0]) + (Pd[1] - u[1]) * (Pd[1] - u[1]) +
                                  (z - u[2]) * (z - u[2]);
                up_first = du < dd;
            }
        }
    }
    if (nu != 1 || nd != 1) return true;
    // the cell's own fan area
    Fan fan;
    fan_start(fan, v[0]);
    for (int i = 1; i < nv; ++i) fan_add(fan, v[i]);
    if (!fan.ok) return true;
    const double total = fan_area_of(fan);
    // the part above z: P_u, the nodes after P_u's arc up to P_d's arc, P_d
    fan_start(fan, Pu);
    const int cnt = au == ad ? (up_first ? 0 : nv) : (ad > au ? ad - au : ad - au + nv);
    for (int k = 1; k <= cnt; ++k) {
        const int i = au + k < nv ? au + k : au + k - nv;
        fan_add(fan, v[i]);
    }
    fan_add(fan, Pd);
    if (!fan.ok) return true;
    double above = fan_area_of(fan);
    // the sliver between the chord P_d -> P_u and the latitude arc
    const double cr = Pd[0] * (Pu[1] - Pd[1]) - Pd[1] * (Pu[0] - Pd[0]);
    const double rho2 = (1.0 - z) * (1.0 + z);
    const double den = rho2 + fma(Pd[0], Pu[0], Pd[1] * Pu[1]);
    if (!gt_zero(cr) || !gt_zero(den)) return true;  // P_u must lie east of P_d, within pi
    const double t = cr / den;
    double sliver;
    if (abs_le(t, kBitsSeries)) {  // t > 0 here
        const double z2 = z * z, t2 = t * t;
        // the coefficients' divisions by 7 and 5 as products with the
        // constants' reciprocals (an FP64 division costs several FMAs)
        const double poly = fma(t2, fma(t2, fma(z2, z2, z2 + 1.0) * (1.0 / 7.0),
                                        (1.0 + z2) * (-1.0 / 5.0)),
                                1.0 / 3.0);
        sliver = 2.0 * z * rho2 * (t * t2) * poly;
    } else {
        sliver = 2.0 * (atan(z * t) - z * atan(t));
    }
    above += sliver;
    areas[off] = total - above;
    areas[off + 1] = above;
    return false;
}

// ---- zonal sums in 128-bit fixed point ---------------------------------------------
// a 64-bit integer rounded to the nearest double, and its leading zeros
EFT_HD double f64_of_u64(unsigned long long x) {
#if defined(__CUDA_ARCH__)
    return __ull2double_rn(x);
#else
    return (double)x;
#endif
}

EFT_HD int clz64(unsigned long long x) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

constexpr int kFracBits = 80;  // zonal sums: fixed point with 2^-80 resolution

// x * 2^80 rounded to an integer (halves away from zero) as a 128-bit two's
// complement (hi, lo); false for a non-finite x or |x| >= 2^46
EFT_HD bool to_fixed(double x, unsigned long long &lo, unsigned long long &hi) {
    const unsigned long long bits = (unsigned long long)wide::bits_of(x);
    const int ex = (int)((bits >> 52) & 0x7ff);
    lo = hi = 0ull;
    if (ex == 0) return true;  // zero or subnormal: far below 2^-80
    if (ex == 0x7ff) return false;
    const unsigned long long M = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = ex - 1075 + kFracBits;  // x * 2^80 = M * 2^sh
    if (sh > 73) return false;             // M * 2^sh >= 2^126
    if (sh >= 64) {
        hi = M << (sh - 64);
    } else if (sh > 0) {
        lo = M << sh;
        hi = M >> (64 - sh);
    } else if (sh == 0) {
        lo = M;
    } else if (-sh <= 54) {
        const int r = -sh;
        lo = (M + (1ull << (r - 1))) >> r;
    }
    if (bits >> 63) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    return true;
}

// the 128-bit fixed-point value as the nearest double
EFT_HD double from_fixed(unsigned long long lo, unsigned long long hi) {
    const bool neg = (hi >> 63) != 0ull;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    double v;
    if (hi == 0ull) {
        v = ldexp(f64_of_u64(lo), -kFracBits);
    } else {
        const int c = clz64(hi);
        unsigned long long top = c ? ((hi << c) | (lo >> (64 - c))) : hi;
        const unsigned long long rest = lo << c;
        top |= rest != 0ull ? 1ull : 0ull;  // sticky: below the rounding position
        v = ldexp(f64_of_u64(top), 64 - c - kFracBits);
    }
    return neg ? -v : v;
}

}  // namespace sphx
