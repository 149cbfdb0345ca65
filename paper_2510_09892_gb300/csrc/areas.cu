// Band areas of spherical cells and zonal sums: the zonal-mean step that
// Sec. 1 names as the use of arc-latitude intersections.
//
//  1. band_range_kernel   one thread per cell: the height range of its arcs
//                         (ranges.cuh) and its winding number around the
//                         z-axis give the bands [lo, hi) it can meet; the
//                         ragged call's prefix sum turns the counts into
//                         output offsets.
//  2. band_partition_kernel sorts the cells into three lists, so that every
//     kernel below sees uniform warps:
//     fan_area_kernel     cells inside one band: the band area is the cell's
//                         own area, a fan of spherical triangles (Van
//                         Oosterom and Strackee's excess).
//     pair_area_kernel    cells cut by one latitude: the fan above its two
//                         crossings (Eq. 2.2) plus the sliver between the
//                         closing chord and the latitude arc; the part below
//                         is the cell's fan minus that.
//     band_area_kernel    every other cell, by the boundary integral. In
//                         longitude and height the area element is
//                         dlambda dz, so by Green's theorem a region's area is
//                         the boundary integral of lambda dz; the latitude
//                         pieces of the boundary of (cell ∩ band) have dz = 0.
//                         Each arc is cut at its crossings with the latitudes
//                         (Eq. 2.2 by the chosen mode), and each piece p -> q
//                         adds lambda_p (z_q - z_p) + dl z_q - T to the band
//                         holding its midpoint: dl is its longitude step and
//                         T = 2 atan(K h) the signed area between it and the
//                         equator, with h = tan(dl / 2) from the xy cross and
//                         dot products and K = (t_p + t_q) / (1 + t_p t_q),
//                         t = tan(latitude / 2). lambda is unwrapped along the
//                         cell from its first node off the poles; a cell
//                         around a pole adds 2 pi times each band's share of
//                         the height from that node to the pole (the cut
//                         across which lambda jumps by 2 pi). Crossings come
//                         in order along the arc without a sort: slot 0 of
//                         Eq. 2.2 crosses upwards along the arc and slot 1
//                         downwards, so a rising run takes the slot-0 hits of
//                         ascending latitudes and a falling run the slot-1
//                         hits of descending ones (an arc that passes its
//                         highest or lowest point is split there).
//  3. zonal_sum_kernel    per band, sum of field * area and of area, in
//                         128-bit fixed point with 64-bit integer atomics (per
//                         block in shared memory, then once per block in
//                         global memory), so the result does not depend on the
//                         order of the additions.
#include <cuda_runtime.h>

#include "common.cuh"
#include "intersect.cuh"
#include "ranges.cuh"

namespace sphx {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kAreaThreads = 128;
constexpr int64_t kSmemLat = 2048;  // latitudes (and their radii) staged in shared memory up to this count
constexpr int kFracBits = 80;       // zonal sums: fixed point with 2^-80 resolution
constexpr int kZonalThreads = 256;
constexpr int64_t kSmemBands = 3072;  // bands accumulated in shared memory up to this count
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
};

// node range [s, e) of cell f in face_nodes; false (status flagged) if invalid
__device__ __forceinline__ bool cell_span(const Mesh &m, int64_t f, int64_t &s, int64_t &e) {
    s = m.face_offsets[f];
    e = m.face_offsets[f + 1];
    if (s < 0 || e < s || e > m.n_face_nodes) {
        atomicOr(m.status, kStatusInvalid);
        return false;
    }
    return true;
}

// coordinates of node face_nodes[i]; false (status flagged) for an index
// outside the node array
__device__ __forceinline__ bool node_at(const Mesh &m, int64_t i, double (&v)[3]) {
    const int32_t id = m.face_nodes[i];
    if (id < 0 || (int64_t)id >= m.n_nodes) {
        atomicOr(m.status, kStatusInvalid);
        return false;
    }
    const double *p = m.nodes + 3 * (int64_t)id;
    v[0] = p[0];
    v[1] = p[1];
    v[2] = p[2];
    return true;
}

__device__ __forceinline__ void unit(const double (&v)[3], double (&u)[3]) {
    const double r = rsqrt(fma(v[0], v[0], fma(v[1], v[1], v[2] * v[2])));
    u[0] = v[0] * r;
    u[1] = v[1] * r;
    u[2] = v[2] * r;
}

// a point of an arc with what the boundary integral needs
struct Pt {
    double x, y, z;  // unit vector
    double rho;      // sqrt(x^2 + y^2); 0 at a pole
};

__device__ __forceinline__ Pt make_pt(double x, double y, double z) {
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
__device__ __forceinline__ Pt make_pt_at(double x, double y, double z0, double rho0) {
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

__device__ __forceinline__ double rho_of_lat(double z) { return sqrt((1.0 - z) * (1.0 + z)); }

// angle from the meridian of r to that of p (xy parts of unit vectors), with
// the cross product taken from the differences, r x p = r x (p - r), so that a
// small angle is accurate relative to itself
__device__ __forceinline__ double delta_lon(double rx, double ry, double x, double y) {
    return atan2(rx * (y - ry) - ry * (x - rx), fma(rx, x, ry * y));
}

// arctan x by its series x - x^3/3 + x^5/5 - x^7/7, for |x| <= 2^-9
// (the next term is below 2^-84 |x|)
__device__ __forceinline__ double atan_small(double x) {
    const double x2 = x * x;
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
__device__ __forceinline__ double add_piece(const Pt &p, const Pt &q, double lam, double dp,
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
    const double zm = sz * rsqrt(fma(sx, sx, fma(sy, sy, sz * sz)));
    const int64_t k = upper_bound_ord(lat, L, ord64(zm)) - 1;
    if (k >= klo && k < klo + nb) out[k - klo] += fma(lam + dp, q.z - p.z, W);
    return dp + dl;
}

// All pieces of the arc a -> b (raw a, b for Eq. 2.2; ua, ub of unit length,
// pa, pb their points) whose longitudes are lam + (offset from a's meridian,
// 0 at a). rho_lat: the latitudes' radii, or null. Returns the offset at b
// (the arc's longitude step).
template <int Mode>
__device__ __forceinline__ double arc_pieces(const double (&a)[3], const double (&b)[3],
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

__global__ void band_range_kernel(Mesh m, int32_t *__restrict__ band_lo,
                                  int32_t *__restrict__ band_hi) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < m.n_faces;
         f += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = 0;
        int64_t s, e;
        if (m.L >= 2 && cell_span(m, f, s, e) && e > s) {
            double zmin = 2.0, zmax = -2.0, wind = 0.0;
            bool ok = true, any = false;
            double a[3], b[3];
            ok = node_at(m, s, a);
            for (int64_t i = s; i < e && ok; ++i) {
                if (!(ok = node_at(m, i + 1 < e ? i + 1 : s, b))) break;
                double zl, zh;
                if (z_range_fp32(a, b, zl, zh) || z_range_fp64(a, b, zl, zh)) {
                    zmin = fmin(zmin, zl);
                    zmax = fmax(zmax, zh);
                    any = true;
                }
                // the winding number needs each step only to well within pi:
                // FP32; arcs from or to a pole step no longitude
                const float ax = (float)a[0], ay = (float)a[1], bx = (float)b[0], by = (float)b[1];
                if ((ax != 0.0f || ay != 0.0f) && (bx != 0.0f || by != 0.0f))
                    wind += (double)atan2f(ax * by - ay * bx, ax * bx + ay * by);
                a[0] = b[0];
                a[1] = b[1];
                a[2] = b[2];
            }
            if (ok && any) {
                const double w = rint(wind / kTwoPi);
                if (w >= 1.0) zmax = 1.0;
                if (w <= -1.0) zmin = -1.0;
                if (!(zmax < m.lat[0] || zmin > m.lat[m.L - 1])) {
                    int64_t klo = upper_bound_ord(m.lat, m.L, ord64(zmin)) - 1;
                    int64_t khi = upper_bound_ord_from(m.lat, m.L, klo + 1, ord64(zmax)) - 1;
                    klo = klo < 0 ? 0 : klo;
                    khi = khi > m.L - 2 ? m.L - 2 : khi;
                    if (khi >= klo) {
                        lo = (int32_t)klo;
                        hi = (int32_t)(khi + 1);
                    }
                }
            }
        }
        band_lo[f] = lo;
        band_hi[f] = hi;
    }
}

// The area of cell f in each band of its range by the boundary integral
// (Green's theorem in longitude and height, see add_piece and arc_pieces)
template <int Mode>
__device__ __forceinline__ void green_cell(const Mesh &m, int64_t f,
                                           const int32_t *__restrict__ band_lo,
                                           const int32_t *__restrict__ band_hi,
                                           const long long *__restrict__ offsets,
                                           double *__restrict__ areas, int64_t cap,
                                           const double *lat, const double *rho_lat) {
    const int64_t klo = band_lo[f];
    const int64_t nb = (int64_t)band_hi[f] - klo;
    if (nb <= 0) return;
    if (klo < 0 || klo + nb > m.L - 1) {
        atomicOr(m.status, kStatusInvalid);
        return;
    }
    const long long off = offsets[f];
    if (off < 0 || off + nb > cap) {
        atomicOr(m.status, kStatusCapacity);
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
        unit(a, ua);
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
        unit(b, ub);
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

// Cells are split in three lists (warp-aggregated appends, so warps stay
// uniform): 0, cells that lie inside one band other than the first and the
// last (their widened height range does, so nothing was clamped), whose band
// area is the cell's own area; 2, cells in two such bands, cut by one
// latitude; 1, the others.
__global__ void band_partition_kernel(const int32_t *__restrict__ band_lo,
                                      const int32_t *__restrict__ band_hi, int64_t F, int64_t L,
                                      int32_t *__restrict__ lists, unsigned long long *counts) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; base < F;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = base + lane;
        int64_t klo = 0, nb = 0;
        if (f < F) {
            klo = band_lo[f];
            nb = (int64_t)band_hi[f] - klo;
        }
        const bool one = f < F && nb == 1 && klo > 0 && klo < L - 2;
        const bool two = f < F && nb == 2 && klo > 0 && klo + 1 < L - 2;
        const bool other = f < F && nb > 0 && !one && !two;
#pragma unroll
        for (int w = 0; w < 3; ++w) {
            const bool mine = w == 0 ? one : (w == 1 ? other : two);
            const unsigned bal = __ballot_sync(0xffffffffu, mine);
            if (!bal) continue;
            unsigned long long at = 0;
            if (lane == __ffs(bal) - 1) at = atomicAdd(counts + w, (unsigned long long)__popc(bal));
            at = __shfl_sync(0xffffffffu, at, __ffs(bal) - 1);
            if (mine) lists[w * F + (int64_t)at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)f;
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
__device__ __forceinline__ bool fan_area(const Mesh &m, int64_t f,
                                         const long long *__restrict__ offsets,
                                         double *__restrict__ areas, int64_t cap) {
    {
        const long long off = offsets[f];
        if (off < 0 || off + 1 > cap) {
            atomicOr(m.status, kStatusCapacity);
            return false;
        }
        int64_t s, e;
        if (!cell_span(m, f, s, e)) return false;
        double v0[3], a[3], b[3], u[3];
        double area = 0.0;
        bool ok = true, far = false;
        if (e - s >= 3) {
            ok = node_at(m, s, u);
            unit(u, v0);
            if (ok) ok = node_at(m, s + 1, u);
            unit(u, a);
            far = fma(v0[0], a[0], fma(v0[1], a[1], v0[2] * a[2])) < 0.5;
            for (int64_t j = s + 2; j < e && ok && !far; ++j) {
                if (!(ok = node_at(m, j, u))) break;
                unit(u, b);
                const double ab = fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
                const double ob = fma(v0[0], b[0], fma(v0[1], b[1], v0[2] * b[2]));
                const double oa = fma(v0[0], a[0], fma(v0[1], a[1], v0[2] * a[2]));
                far = ob < 0.5;
                const double d1x = a[0] - v0[0], d1y = a[1] - v0[1], d1z = a[2] - v0[2];
                const double d2x = b[0] - v0[0], d2y = b[1] - v0[1], d2z = b[2] - v0[2];
                const double tri = fma(v0[0], d1y * d2z - d1z * d2y,
                                       fma(v0[1], d1z * d2x - d1x * d2z,
                                           v0[2] * (d1x * d2y - d1y * d2x)));
                const double t = tri / (1.0 + oa + ab + ob);
                area += 2.0 * (fabs(t) <= 0.001953125 ? atan_small(t) : atan(t));
                a[0] = b[0];
                a[1] = b[1];
                a[2] = b[2];
            }
        }
        if (!ok) return false;
        if (far) return true;
        areas[off] = area;
        return false;
    }
}

// fan_area over the one-band list; a cell the fan does not take is appended
// to the other list, which band_area_kernel (launched after this kernel)
// works through
__global__ void __launch_bounds__(kAreaThreads, 8)
    fan_area_kernel(Mesh m, const long long *__restrict__ offsets, double *__restrict__ areas,
                    int64_t cap, int32_t *__restrict__ lists,
                    unsigned long long *__restrict__ counts) {
    const int64_t n = (int64_t)counts[0];
    const int lane = threadIdx.x & 31;
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + lane;
        bool far = false;
        int64_t f = -1;
        if (i < n) {
            f = lists[i];
            far = fan_area(m, f, offsets, areas, cap);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, far);
        if (bal) {
            unsigned long long at = 0;
            if (lane == __ffs(bal) - 1) at = atomicAdd(counts + 1, (unsigned long long)__popc(bal));
            at = __shfl_sync(0xffffffffu, at, __ffs(bal) - 1);
            if (far) lists[m.n_faces + (int64_t)at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)f;
        }
    }
}

// fan area of the points p[0..n) (unit vectors) from p[0]; false when a point
// is more than 60 degrees from p[0]
__device__ __forceinline__ bool fan_of(const double (*p)[3], int n, double &area) {
    area = 0.0;
    for (int i = 1; i + 1 < n; ++i) {
        const double *a = p[i], *b = p[i + 1], *o = p[0];
        const double oa = fma(o[0], a[0], fma(o[1], a[1], o[2] * a[2]));
        const double ob = fma(o[0], b[0], fma(o[1], b[1], o[2] * b[2]));
        const double ab = fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
        if (oa < 0.5 || ob < 0.5) return false;
        const double d1x = a[0] - o[0], d1y = a[1] - o[1], d1z = a[2] - o[2];
        const double d2x = b[0] - o[0], d2y = b[1] - o[1], d2z = b[2] - o[2];
        const double tri = fma(o[0], d1y * d2z - d1z * d2y,
                               fma(o[1], d1z * d2x - d1x * d2z, o[2] * (d1x * d2y - d1y * d2x)));
        const double t = tri / (1.0 + oa + ab + ob);
        area += 2.0 * (fabs(t) <= 0.001953125 ? atan_small(t) : atan(t));
    }
    return true;
}

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
__device__ __forceinline__ bool pair_area(const Mesh &m, int64_t f,
                                          const int32_t *__restrict__ band_lo,
                                          const long long *__restrict__ offsets,
                                          double *__restrict__ areas, int64_t cap,
                                          const double *lat) {
    const long long off = offsets[f];
    if (off < 0 || off + 2 > cap) {
        atomicOr(m.status, kStatusCapacity);
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
        unit(r[i], v[i]);
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
        const int i = __ffs(need) - 1;
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
    double total;
    if (!fan_of(v, nv, total)) return true;
    // the part above z: P_u, the nodes after P_u's arc up to P_d's arc, P_d
    double q[kPairMaxNodes + 2][3];
    int nq = 0;
    q[nq][0] = Pu[0];
    q[nq][1] = Pu[1];
    q[nq][2] = Pu[2];
    ++nq;
    int cnt = au == ad ? (up_first ? 0 : nv) : (ad - au + nv) % nv;
    for (int k = 1; k <= cnt; ++k) {
        const int i = (au + k) % nv;
        q[nq][0] = v[i][0];
        q[nq][1] = v[i][1];
        q[nq][2] = v[i][2];
        ++nq;
    }
    q[nq][0] = Pd[0];
    q[nq][1] = Pd[1];
    q[nq][2] = Pd[2];
    ++nq;
    double above;
    if (!fan_of(q, nq, above)) return true;
    // the sliver between the chord P_d -> P_u and the latitude arc
    const double cr = Pd[0] * (Pu[1] - Pd[1]) - Pd[1] * (Pu[0] - Pd[0]);
    const double rho2 = (1.0 - z) * (1.0 + z);
    const double den = rho2 + fma(Pd[0], Pu[0], Pd[1] * Pu[1]);
    if (!(cr > 0.0) || !(den > 0.0)) return true;  // P_u must lie east of P_d, within pi
    const double t = cr / den;
    double sliver;
    if (t <= 0.001953125) {
        const double z2 = z * z, t2 = t * t;
        const double poly = fma(t2, fma(t2, fma(z2, z2, z2 + 1.0) / 7.0, -(1.0 + z2) / 5.0),
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

// pair_area over the two-band list; a cell it does not cover is appended to
// the other list (taken by band_area_kernel, launched after this kernel)
template <int Mode>
__global__ void __launch_bounds__(kAreaThreads)
    pair_area_kernel(Mesh m, const int32_t *__restrict__ band_lo,
                     const long long *__restrict__ offsets, double *__restrict__ areas, int64_t cap,
                     int32_t *__restrict__ lists, unsigned long long *__restrict__ counts) {
    extern __shared__ double s_lat[];
    const double *lat = m.lat;
    if (m.L <= kSmemLat) {
        for (int64_t i = threadIdx.x; i < m.L; i += blockDim.x) s_lat[i] = m.lat[i];
        __syncthreads();
        lat = s_lat;
    }
    const int64_t n = (int64_t)counts[2];
    const int lane = threadIdx.x & 31;
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + lane;
        bool back = false;
        int64_t f = -1;
        if (i < n) {
            f = lists[2 * m.n_faces + i];
            back = pair_area<Mode>(m, f, band_lo, offsets, areas, cap, lat);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, back);
        if (bal) {
            unsigned long long at = 0;
            if (lane == __ffs(bal) - 1) at = atomicAdd(counts + 1, (unsigned long long)__popc(bal));
            at = __shfl_sync(0xffffffffu, at, __ffs(bal) - 1);
            if (back) lists[m.n_faces + (int64_t)at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)f;
        }
    }
}

template <int Mode>
__global__ void __launch_bounds__(kAreaThreads, 3)
    band_area_kernel(Mesh m, const int32_t *__restrict__ band_lo,
                     const int32_t *__restrict__ band_hi, const long long *__restrict__ offsets,
                     double *__restrict__ areas, int64_t cap, const int32_t *__restrict__ list,
                     const unsigned long long *__restrict__ count) {
    extern __shared__ double s_lat[];  // L latitudes, then their radii
    const double *lat = m.lat, *rho_lat = nullptr;
    if (m.L <= kSmemLat) {
        for (int64_t i = threadIdx.x; i < m.L; i += blockDim.x) {
            const double z = m.lat[i];
            s_lat[i] = z;
            s_lat[m.L + i] = rho_of_lat(z);
        }
        __syncthreads();
        lat = s_lat;
        rho_lat = s_lat + m.L;
    }
    const int64_t n = (int64_t)*count;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        green_cell<Mode>(m, list[i], band_lo, band_hi, offsets, areas, cap, lat, rho_lat);
}

// ---- zonal sums in 128-bit fixed point ---------------------------------------------
// x * 2^80 rounded to an integer (halves away from zero) as a 128-bit two's
// complement (hi, lo); false for a non-finite x or |x| >= 2^46
__device__ __forceinline__ bool to_fixed(double x, unsigned long long &lo,
                                         unsigned long long &hi) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
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

// (hi, lo) += (vhi, vlo) modulo 2^128 with two 64-bit atomics: each wrap of
// the low word carries once into the high word, whatever the order
__device__ __forceinline__ void add128(unsigned long long *acc, unsigned long long vlo,
                                       unsigned long long vhi) {
    if (vlo == 0ull && vhi == 0ull) return;
    const unsigned long long old = atomicAdd(acc, vlo);
    const unsigned long long up = vhi + (old + vlo < old ? 1ull : 0ull);
    if (up) atomicAdd(acc + 1, up);
}

// the 128-bit fixed-point value as the nearest double
__device__ __forceinline__ double from_fixed(unsigned long long lo, unsigned long long hi) {
    const bool neg = (hi >> 63) != 0ull;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    double v;
    if (hi == 0ull) {
        v = ldexp(__ull2double_rn(lo), -kFracBits);
    } else {
        const int c = __clzll((long long)hi);
        unsigned long long top = c ? ((hi << c) | (lo >> (64 - c))) : hi;
        const unsigned long long rest = lo << c;
        top |= rest != 0ull ? 1ull : 0ull;  // sticky: below the rounding position
        v = ldexp(__ull2double_rn(top), 64 - c - kFracBits);
    }
    return neg ? -v : v;
}

__global__ void __launch_bounds__(kZonalThreads)
    zonal_sum_kernel(const int32_t *__restrict__ band_lo, const int32_t *__restrict__ band_hi,
                     const long long *__restrict__ offsets, int64_t F,
                     const double *__restrict__ areas, const double *__restrict__ field,
                     int64_t n_bands, unsigned long long *__restrict__ acc, int use_smem,
                     unsigned *status) {
    extern __shared__ unsigned long long s_acc[];
    unsigned long long *tgt = acc;
    if (use_smem) {
        for (int64_t i = threadIdx.x; i < 4 * n_bands; i += blockDim.x) s_acc[i] = 0ull;
        __syncthreads();
        tgt = s_acc;
    }
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t klo = band_lo[f];
        const int64_t nb = (int64_t)band_hi[f] - klo;
        if (nb <= 0) continue;
        const long long off = offsets[f];
        const double fv = field[f];
        for (int64_t j = 0; j < nb; ++j) {
            const int64_t k = klo + j;
            if (k < 0 || k >= n_bands || off < 0) {
                atomicOr(status, kStatusInvalid);
                break;
            }
            const double A = areas[off + j];
            unsigned long long lo, hi;
            if (to_fixed(fv * A, lo, hi))
                add128(tgt + 4 * k, lo, hi);
            else
                atomicOr(status, kStatusInvalid);
            if (to_fixed(A, lo, hi))
                add128(tgt + 4 * k + 2, lo, hi);
            else
                atomicOr(status, kStatusInvalid);
        }
    }
    if (use_smem) {
        __syncthreads();
        for (int64_t i = threadIdx.x; i < 2 * n_bands; i += blockDim.x)
            add128(acc + 2 * i, s_acc[2 * i], s_acc[2 * i + 1]);
    }
}

__global__ void zonal_finish_kernel(const unsigned long long *__restrict__ acc, int64_t n_bands,
                                    double *__restrict__ out_fa, double *__restrict__ out_a) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_bands;
         k += (int64_t)gridDim.x * blockDim.x) {
        out_fa[k] = from_fixed(acc[4 * k], acc[4 * k + 1]);
        out_a[k] = from_fixed(acc[4 * k + 2], acc[4 * k + 3]);
    }
}

// ---- launchers -------------------------------------------------------------------
template <int Mode>
static cudaError_t launch_areas_mode(const Mesh &m, const int32_t *lo, const int32_t *hi,
                                     const long long *off, double *areas, int64_t cap,
                                     int32_t *lists, unsigned long long *counts, int sm_count,
                                     cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int64_t need = (m.n_faces + 255) / 256;
    band_partition_kernel<<<(unsigned)std::min<int64_t>(need, (int64_t)sm_count * 8), 256, 0, s>>>(
        lo, hi, m.n_faces, m.L, lists, counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fan_area_kernel, kAreaThreads, 0);
    if (e != cudaSuccess) return e;
    int64_t grid = std::min<int64_t>((m.n_faces + kAreaThreads - 1) / kAreaThreads,
                                     (int64_t)std::max(per_sm, 1) * sm_count);
    fan_area_kernel<<<(unsigned)grid, kAreaThreads, 0, s>>>(m, off, areas, cap, lists, counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem1 = m.L <= kSmemLat ? (size_t)m.L * sizeof(double) : 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_area_kernel<Mode>, kAreaThreads,
                                                      smem1);
    if (e != cudaSuccess) return e;
    grid = std::min<int64_t>((m.n_faces + kAreaThreads - 1) / kAreaThreads,
                             (int64_t)std::max(per_sm, 1) * sm_count);
    pair_area_kernel<Mode><<<(unsigned)grid, kAreaThreads, smem1, s>>>(m, lo, off, areas, cap, lists,
                                                                        counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = m.L <= kSmemLat ? 2 * (size_t)m.L * sizeof(double) : 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, band_area_kernel<Mode>, kAreaThreads,
                                                      smem);
    if (e != cudaSuccess) return e;
    grid = std::min<int64_t>((m.n_faces + kAreaThreads - 1) / kAreaThreads,
                             (int64_t)std::max(per_sm, 1) * sm_count);
    band_area_kernel<Mode><<<(unsigned)grid, kAreaThreads, smem, s>>>(
        m, lo, hi, off, areas, cap, lists + m.n_faces, counts + 1);
    return cudaGetLastError();
}

}  // namespace sphx

using namespace sphx;

namespace {

bool valid_mesh(sphx_context *ctx, const double *nodes, int64_t n_nodes,
                const int64_t *face_offsets, const int32_t *face_nodes, int64_t n_face_nodes,
                int64_t n_faces, const double *lat_z, int64_t n_lat) {
    // cells and nodes are indexed by int32 (node indices, the cell lists)
    return ctx && n_faces >= 0 && n_faces <= INT32_MAX && n_nodes >= 0 && n_nodes <= INT32_MAX &&
           n_face_nodes >= 0 && n_lat >= 2 && n_lat <= INT32_MAX &&
           (n_faces == 0 || (nodes && face_offsets && face_nodes)) && lat_z;
}

Mesh make_mesh(sphx_context *ctx, const double *nodes, int64_t n_nodes,
               const int64_t *face_offsets, const int32_t *face_nodes, int64_t n_face_nodes,
               int64_t n_faces, const double *lat_z, int64_t n_lat) {
    Mesh m;
    m.nodes = nodes;
    m.n_nodes = n_nodes;
    m.face_offsets = face_offsets;
    m.face_nodes = face_nodes;
    m.n_face_nodes = n_face_nodes;
    m.n_faces = n_faces;
    m.lat = lat_z;
    m.L = n_lat;
    m.status = ctx->status;
    return m;
}

}  // namespace

extern "C" sphx_status sphx_band_ranges(sphx_context *ctx, const double *nodes, int64_t n_nodes,
                                        const int64_t *face_offsets, const int32_t *face_nodes,
                                        int64_t n_face_nodes, int64_t n_faces,
                                        const double *lat_z, int64_t n_lat, int32_t *band_lo,
                                        int32_t *band_hi, int64_t *area_offsets,
                                        sphx_stream stream) {
    if (!valid_mesh(ctx, nodes, n_nodes, face_offsets, face_nodes, n_face_nodes, n_faces, lat_z,
                    n_lat) ||
        !area_offsets || (n_faces > 0 && (!band_lo || !band_hi)))
        return SPHX_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> g(ctx->mu);
    SPHX_CUDA(cudaSetDevice(ctx->device));
    if (n_faces == 0) {
        SPHX_CUDA(cudaMemsetAsync(area_offsets, 0, sizeof(int64_t), s));
        return SPHX_OK;
    }
    sphx_status st = ensure_band_scratch(ctx, n_faces);
    if (st != SPHX_OK) return st;
    const Mesh m =
        make_mesh(ctx, nodes, n_nodes, face_offsets, face_nodes, n_face_nodes, n_faces, lat_z, n_lat);
    const int64_t grid = std::min<int64_t>((n_faces + 255) / 256, (int64_t)ctx->sm_count * 8);
    band_range_kernel<<<(unsigned)grid, 256, 0, s>>>(m, band_lo, band_hi);
    SPHX_CUDA(cudaGetLastError());
    SPHX_CUDA(launch_scan(band_lo, band_hi, n_faces, ctx->band_block_sums,
                          reinterpret_cast<long long *>(area_offsets), s));
    return SPHX_OK;
}

extern "C" sphx_status sphx_band_areas(sphx_context *ctx, const double *nodes, int64_t n_nodes,
                                       const int64_t *face_offsets, const int32_t *face_nodes,
                                       int64_t n_face_nodes, int64_t n_faces,
                                       const double *lat_z, int64_t n_lat,
                                       const int32_t *band_lo, const int32_t *band_hi,
                                       const int64_t *area_offsets, sphx_mode mode,
                                       double *areas, int64_t areas_cap, sphx_stream stream) {
    if (!valid_mesh(ctx, nodes, n_nodes, face_offsets, face_nodes, n_face_nodes, n_faces, lat_z,
                    n_lat) ||
        areas_cap < 0 || (n_faces > 0 && (!band_lo || !band_hi || !area_offsets)) ||
        (areas_cap > 0 && !areas))
        return SPHX_ERR_INVALID_ARG;
    if (n_faces == 0) return SPHX_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> g(ctx->mu);
    SPHX_CUDA(cudaSetDevice(ctx->device));
    sphx_status st = ensure_band_scratch(ctx, n_faces);
    if (st != SPHX_OK) return st;
    const Mesh m =
        make_mesh(ctx, nodes, n_nodes, face_offsets, face_nodes, n_face_nodes, n_faces, lat_z, n_lat);
    const long long *off = reinterpret_cast<const long long *>(area_offsets);
    cudaError_t e;
    switch (mode) {
        case SPHX_MODE_DIRECT_FP64:
            e = launch_areas_mode<kDirect>(m, band_lo, band_hi, off, areas, areas_cap, ctx->band_lists,
                                 ctx->band_counts, ctx->sm_count, s);
            break;
        case SPHX_MODE_EFT_FP64:
            e = launch_areas_mode<kEftFp64>(m, band_lo, band_hi, off, areas, areas_cap, ctx->band_lists,
                                 ctx->band_counts, ctx->sm_count, s);
            break;
        case SPHX_MODE_EFT_FF32:
            e = launch_areas_mode<kEftFf32>(m, band_lo, band_hi, off, areas, areas_cap, ctx->band_lists,
                                 ctx->band_counts, ctx->sm_count, s);
            break;
        case SPHX_MODE_EFT_FP64_PRINTED:
            e = launch_areas_mode<kEftFp64Printed>(m, band_lo, band_hi, off, areas, areas_cap, ctx->band_lists,
                                 ctx->band_counts, ctx->sm_count, s);
            break;
        case SPHX_MODE_WIDE_INT:
            e = launch_areas_mode<kWideInt>(m, band_lo, band_hi, off, areas, areas_cap, ctx->band_lists,
                                 ctx->band_counts, ctx->sm_count, s);
            break;
        case SPHX_MODE_ADAPTIVE:
            return SPHX_ERR_UNSUPPORTED;
        default:
            return SPHX_ERR_INVALID_ARG;
    }
    SPHX_CUDA(e);
    return SPHX_OK;
}

extern "C" sphx_status sphx_zonal_sums(sphx_context *ctx, const int32_t *band_lo,
                                       const int32_t *band_hi, const int64_t *area_offsets,
                                       int64_t n_faces, const double *areas, const double *field,
                                       int64_t n_lat, double *out_fa, double *out_a,
                                       sphx_stream stream) {
    if (!ctx || n_faces < 0 || n_lat < 2 || !out_fa || !out_a ||
        (n_faces > 0 && (!band_lo || !band_hi || !area_offsets || !areas || !field)))
        return SPHX_ERR_INVALID_ARG;
    const int64_t n_bands = n_lat - 1;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> g(ctx->mu);
    SPHX_CUDA(cudaSetDevice(ctx->device));
    sphx_status st = ensure_zonal_scratch(ctx, n_bands);
    if (st != SPHX_OK) return st;
    unsigned long long *acc = ctx->zonal_acc;
    SPHX_CUDA(cudaMemsetAsync(acc, 0, 4 * n_bands * sizeof(unsigned long long), s));
    if (n_faces > 0) {
        const int use_smem = n_bands <= kSmemBands ? 1 : 0;
        const size_t smem = use_smem ? (size_t)(4 * n_bands) * sizeof(unsigned long long) : 0;
        if (smem > 48 * 1024)
            SPHX_CUDA(cudaFuncSetAttribute(zonal_sum_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int64_t grid =
            std::min<int64_t>((n_faces + kZonalThreads - 1) / kZonalThreads, (int64_t)ctx->sm_count * 2);
        zonal_sum_kernel<<<(unsigned)grid, kZonalThreads, smem, s>>>(
            band_lo, band_hi, reinterpret_cast<const long long *>(area_offsets), n_faces, areas,
            field, n_bands, acc, use_smem, ctx->status);
        SPHX_CUDA(cudaGetLastError());
    }
    const int64_t g2 = std::min<int64_t>((n_bands + 255) / 256, 1024);
    zonal_finish_kernel<<<(unsigned)g2, 256, 0, s>>>(acc, n_bands, out_fa, out_a);
    SPHX_CUDA(cudaGetLastError());
    return SPHX_OK;
}
