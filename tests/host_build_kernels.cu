// Host builds of the kernels' per-pair and per-cell routines, exported for
// tests/test_host_builds.py: pair_wide, pair_ff32, pair_accux and pair_direct
// (paper_2510_09892_gb300/csrc/intersect.cuh), arcs_wide (arcs.cuh), the
// adaptive filter (adaptive.cuh), the band-area routines (areas.cuh) and the
// height ranges and latitude searches (ranges.cuh) are __host__ __device__.
// The same source as the GPU kernels, run on the CPU against the exact
// oracles and the step-by-step FP64 reference. Built with FMA contraction off.
#include "../paper_2510_09892_gb300/csrc/adaptive.cuh"
#include "../paper_2510_09892_gb300/csrc/areas.cuh"
#include "../paper_2510_09892_gb300/csrc/arcs.cuh"

extern "C" void h_pair_wide(const double *A, const double *B, const double *Z, long long n,
                            double *pts, int *cnt) {
    const double nan = __builtin_nan("");
    for (long long i = 0; i < n; ++i) {
        const double x1[3] = {A[3 * i], A[3 * i + 1], A[3 * i + 2]};
        const double x2[3] = {B[3 * i], B[3 * i + 1], B[3 * i + 2]};
        sphx::PairOut o;
        sphx::pair_wide(x1, x2, Z[i], o);
        for (int r = 0; r < 2; ++r) {
            pts[6 * i + 3 * r + 0] = o.hit[r] ? o.px[r] : nan;
            pts[6 * i + 3 * r + 1] = o.hit[r] ? o.py[r] : nan;
            pts[6 * i + 3 * r + 2] = o.hit[r] ? Z[i] : nan;
        }
        cnt[i] = o.count;
    }
}

template <int Which>
static void run_fp64(const double *A, const double *B, const double *Z, long long n,
                     double *pts, int *cnt) {
    const double nan = __builtin_nan("");
    for (long long i = 0; i < n; ++i) {
        const double x1[3] = {A[3 * i], A[3 * i + 1], A[3 * i + 2]};
        const double x2[3] = {B[3 * i], B[3 * i + 1], B[3 * i + 2]};
        sphx::PairOut o;
        if (Which == 0)
            sphx::pair_direct(x1, x2, Z[i], o);
        else if (Which == 1)
            sphx::pair_accux<true>(x1, x2, Z[i], o);
        else
            sphx::pair_accux<false>(x1, x2, Z[i], o);
        for (int r = 0; r < 2; ++r) {
            pts[6 * i + 3 * r + 0] = o.hit[r] ? o.px[r] : nan;
            pts[6 * i + 3 * r + 1] = o.hit[r] ? o.py[r] : nan;
            pts[6 * i + 3 * r + 2] = o.hit[r] ? Z[i] : nan;
        }
        cnt[i] = o.count;
    }
}

extern "C" void h_pair_direct(const double *A, const double *B, const double *Z, long long n,
                              double *pts, int *cnt) {
    run_fp64<0>(A, B, Z, n, pts, cnt);
}

extern "C" void h_pair_accux(const double *A, const double *B, const double *Z, long long n,
                             double *pts, int *cnt) {
    run_fp64<1>(A, B, Z, n, pts, cnt);
}

extern "C" void h_pair_accux_printed(const double *A, const double *B, const double *Z,
                                     long long n, double *pts, int *cnt) {
    run_fp64<2>(A, B, Z, n, pts, cnt);
}

extern "C" void h_pair_ff32(const double *A, const double *B, const double *Z, long long n,
                           double *pts, int *cnt) {
    const double nan = __builtin_nan("");
    for (long long i = 0; i < n; ++i) {
        const double x1[3] = {A[3 * i], A[3 * i + 1], A[3 * i + 2]};
        const double x2[3] = {B[3 * i], B[3 * i + 1], B[3 * i + 2]};
        sphx::PairOut o;
        sphx::pair_ff32(x1, x2, Z[i], o);
        for (int r = 0; r < 2; ++r) {
            pts[6 * i + 3 * r + 0] = o.hit[r] ? o.px[r] : nan;
            pts[6 * i + 3 * r + 1] = o.hit[r] ? o.py[r] : nan;
            pts[6 * i + 3 * r + 2] = o.hit[r] ? Z[i] : nan;
        }
        cnt[i] = o.count;
    }
}

extern "C" void h_arcs_wide(const double *A1, const double *A2, const double *B1,
                            const double *B2, long long n, double *pts, int *cnt) {
    const double nan = __builtin_nan("");
    for (long long i = 0; i < n; ++i) {
        const double a1[3] = {A1[3 * i], A1[3 * i + 1], A1[3 * i + 2]};
        const double a2[3] = {A2[3 * i], A2[3 * i + 1], A2[3 * i + 2]};
        const double b1[3] = {B1[3 * i], B1[3 * i + 1], B1[3 * i + 2]};
        const double b2[3] = {B2[3 * i], B2[3 * i + 1], B2[3 * i + 2]};
        sphx::ArcOut r;
        sphx::arcs_wide(a1, a2, b1, b2, r);
        for (int k = 0; k < 2; ++k) {
            const bool h = r.o.hit[k];
            pts[6 * i + 3 * k + 0] = h ? r.o.px[k] : nan;
            pts[6 * i + 3 * k + 1] = h ? r.o.py[k] : nan;
            pts[6 * i + 3 * k + 2] = h ? (k == 0 ? r.pz : -r.pz) : nan;
        }
        cnt[i] = r.o.count;
    }
}

// the adaptive filter alone: kept[i] = 1 where it vouches for arc i (its
// result in pts and cnt), 0 where the kernel would hand the arc on
extern "C" void h_pair_filtered(const double *A, const double *B, const double *Z, long long n,
                                double gate_ulps, double *pts, int *cnt, int *kept) {
    const double nan = __builtin_nan("");
    for (long long i = 0; i < n; ++i) {
        const double x1[3] = {A[3 * i], A[3 * i + 1], A[3 * i + 2]};
        const double x2[3] = {B[3 * i], B[3 * i + 1], B[3 * i + 2]};
        sphx::PairOut o;
        kept[i] = sphx::filt::pair_filtered(x1, x2, Z[i], 0.975 * gate_ulps, o) ? 1 : 0;
        for (int r = 0; r < 2; ++r) {
            const bool h = kept[i] && o.hit[r];
            pts[6 * i + 3 * r + 0] = h ? o.px[r] : nan;
            pts[6 * i + 3 * r + 1] = h ? o.py[r] : nan;
            pts[6 * i + 3 * r + 2] = h ? Z[i] : nan;
        }
        cnt[i] = kept[i] ? o.count : -9;
    }
}

// the normalised copy of the nodes that sphx_band_areas makes (unit() per
// node), or nullptr: the area routines must give the same bits either way
static double *unit_copy(const double *nodes, long long n_nodes, int pre) {
    if (!pre) return nullptr;
    double *u = new double[3 * (n_nodes > 0 ? n_nodes : 1)];
    for (long long i = 0; i < n_nodes; ++i) {
        const double v[3] = {nodes[3 * i], nodes[3 * i + 1], nodes[3 * i + 2]};
        double w[3];
        sphx::unit(v, w);
        u[3 * i] = w[0];
        u[3 * i + 1] = w[1];
        u[3 * i + 2] = w[2];
    }
    return u;
}

// band areas of every cell with the boundary integral (green_cell, crossings
// in integer limbs), each cell given the full band range: out is n_faces x
// (L - 1), row f the areas of cell f in bands 0 .. L - 2
extern "C" unsigned h_green_cells(const double *nodes, long long n_nodes,
                                  const long long *face_offsets, const int *face_nodes,
                                  long long n_faces, const double *lat, long long L,
                                  double *out, int pre) {
    unsigned status = 0u;
    double *un = unit_copy(nodes, n_nodes, pre);
    sphx::Mesh m{nodes, n_nodes, (const int64_t *)face_offsets, face_nodes,
                 (int64_t)face_offsets[n_faces], n_faces, lat, L, &status, un};
    const long long nb = L - 1;
    int32_t *lo = new int32_t[n_faces], *hi = new int32_t[n_faces];
    long long *off = new long long[n_faces];
    double *rho = new double[L];
    for (long long k = 0; k < L; ++k) rho[k] = sphx::rho_of_lat(lat[k]);
    for (long long f = 0; f < n_faces; ++f) {
        lo[f] = 0;
        hi[f] = (int32_t)nb;
        off[f] = f * nb;
    }
    for (long long f = 0; f < n_faces; ++f)
        sphx::green_cell<sphx::kWideInt>(m, f, lo, hi, off, out, n_faces * nb, lat, rho);
    delete[] un;
    delete[] lo;
    delete[] hi;
    delete[] off;
    delete[] rho;
    return status;
}

// the fan area of every cell (fan_area): area[f], or NaN where the routine
// declines the cell (a node more than 60 degrees from node 0)
extern "C" void h_fan_cells(const double *nodes, long long n_nodes, const long long *face_offsets,
                            const int *face_nodes, long long n_faces, double *area, int pre) {
    unsigned status = 0u;
    double *un = unit_copy(nodes, n_nodes, pre);
    sphx::Mesh m{nodes, n_nodes, (const int64_t *)face_offsets, face_nodes,
                 (int64_t)face_offsets[n_faces], n_faces, nullptr, 0, &status, un};
    long long *off = new long long[n_faces];
    for (long long f = 0; f < n_faces; ++f) {
        off[f] = f;
        area[f] = __builtin_nan("");
    }
    for (long long f = 0; f < n_faces; ++f) sphx::fan_area(m, f, off, area, n_faces);
    delete[] un;
    delete[] off;
}

// the two band areas of each cell cut by the latitude lat[band_lo[f] + 1]
// (pair_area, crossings in integer limbs): out[2 f], out[2 f + 1] for bands
// band_lo[f] and band_lo[f] + 1, NaN where the routine declines the cell
extern "C" void h_pair_cells(const double *nodes, long long n_nodes,
                             const long long *face_offsets, const int *face_nodes,
                             long long n_faces, const double *lat, long long L,
                             const int *band_lo, double *out, int pre) {
    unsigned status = 0u;
    double *un = unit_copy(nodes, n_nodes, pre);
    sphx::Mesh m{nodes, n_nodes, (const int64_t *)face_offsets, face_nodes,
                 (int64_t)face_offsets[n_faces], n_faces, lat, L, &status, un};
    long long *off = new long long[n_faces];
    for (long long f = 0; f < n_faces; ++f) {
        off[f] = 2 * f;
        out[2 * f] = out[2 * f + 1] = __builtin_nan("");
    }
    for (long long f = 0; f < n_faces; ++f)
        sphx::pair_area<sphx::kWideInt>(m, f, band_lo, off, out, 2 * n_faces, lat);
    delete[] un;
    delete[] off;
}

// the candidate kernels' height range of each arc (z_range_fp32, else
// z_range_fp64 for finite endpoints, as in ragged.cu and fused.cu); ok[i] = 0
// where neither gives one. fp32[i] = 1 where the FP32 range alone gives it.
extern "C" void h_z_ranges(const double *A, const double *B, long long n, double *zmin,
                           double *zmax, int *ok, int *fp32) {
    for (long long i = 0; i < n; ++i) {
        const double x1[3] = {A[3 * i], A[3 * i + 1], A[3 * i + 2]};
        const double x2[3] = {B[3 * i], B[3 * i + 1], B[3 * i + 2]};
        double lo = 0.0, hi = 0.0;
        bool finite = true;
        for (int k = 0; k < 3; ++k) finite = finite && sphx::finite_bits(x1[k]) && sphx::finite_bits(x2[k]);
        const bool f32 = sphx::z_range_fp32(x1, x2, lo, hi);
        fp32[i] = f32 ? 1 : 0;
        ok[i] = (f32 || (finite && sphx::z_range_fp64(x1, x2, lo, hi))) ? 1 : 0;
        zmin[i] = lo;
        zmax[i] = hi;
    }
}

// the latitude searches of ranges.cuh over one sorted array: for each key,
// the first index with a[i] >= key, the first with a[i] > key, and the latter
// again by galloping forward from the former
extern "C" void h_searches(const double *a, long long n, const double *keys, long long m,
                           long long *lower, long long *upper, long long *gallop) {
    for (long long i = 0; i < m; ++i) {
        const long long k = sphx::ord64(keys[i]);
        lower[i] = sphx::lower_bound_ord(a, n, k);
        upper[i] = sphx::upper_bound_ord(a, n, k);
        gallop[i] = sphx::upper_bound_ord_from(a, n, lower[i], k);
    }
}

// the zonal sums' fixed point: x * 2^80 rounded (halves away from zero) as a
// 128-bit two's complement (lo, hi) with ok = 0 where out of range, and a
// 128-bit value back as the nearest double
extern "C" void h_to_fixed(const double *x, long long n, unsigned long long *lo,
                           unsigned long long *hi, int *ok) {
    for (long long i = 0; i < n; ++i) ok[i] = sphx::to_fixed(x[i], lo[i], hi[i]) ? 1 : 0;
}

extern "C" void h_from_fixed(const unsigned long long *lo, const unsigned long long *hi,
                             long long n, double *x) {
    for (long long i = 0; i < n; ++i) x[i] = sphx::from_fixed(lo[i], hi[i]);
}

// Algorithm 8's intermediate pairs (App. A) as the intermediates call dumps
// them: 16 doubles per arc
extern "C" void h_accux_mid(const double *A, const double *B, const double *Z, long long n,
                            double *mid) {
    for (long long i = 0; i < n; ++i) {
        const double x1[3] = {A[3 * i], A[3 * i + 1], A[3 * i + 2]};
        const double x2[3] = {B[3 * i], B[3 * i + 1], B[3 * i + 2]};
        sphx::PairOut o;
        sphx::pair_accux<true>(x1, x2, Z[i], o, mid + 16 * i);
    }
}

// the fast FP64 -> FP32 conversion against the general one, on given bit patterns
extern "C" long long h_f32_of_mismatches(const double *x, long long n) {
    long long bad = 0;
    for (long long i = 0; i < n; ++i) {
        const float a = sphx::f32_of(x[i]), b = sphx::f32_scaled(x[i], 0);
        if (sphx::wide::fbits_of(a) != sphx::wide::fbits_of(b)) ++bad;
    }
    return bad;
}

// the fan triangles' reciprocal (areas.cuh) and the nodes' normalisation
extern "C" void h_rcp_den(const double *x, long long n, double *out) {
    for (long long i = 0; i < n; ++i) out[i] = sphx::rcp_den(x[i]);
}

extern "C" void h_unit(const double *v, long long n, double *out) {
    for (long long i = 0; i < n; ++i) {
        const double a[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
        double u[3];
        sphx::unit(a, u);
        out[3 * i] = u[0];
        out[3 * i + 1] = u[1];
        out[3 * i + 2] = u[2];
    }
}

// the integer-pipe tests of doubles: bit 0 lt_pos(x, 0.5), bit 1
// abs_le(x, 2^-9), bit 2 gt_zero(x), bit 3 ge_zero(x), bit 4 eq_zero(x),
// bit 5 finite_bits(x), bit 6 le_zero(x)
extern "C" void h_compares(const double *x, long long n, int *out) {
    for (long long i = 0; i < n; ++i)
        out[i] = (sphx::lt_pos(x[i], sphx::kBitsHalf) ? 1 : 0) |
                 (sphx::abs_le(x[i], sphx::kBitsSeries) ? 2 : 0) | (sphx::gt_zero(x[i]) ? 4 : 0) |
                 (sphx::ge_zero(x[i]) ? 8 : 0) | (sphx::eq_zero(x[i]) ? 16 : 0) |
                 (sphx::finite_bits(x[i]) ? 32 : 0) | (sphx::le_zero(x[i]) ? 64 : 0);
}

// the FP64 TwoSum the kernels use (magnitude-ordered FastTwoSum)
extern "C" void h_two_sum(const double *a, const double *b, long long n, double *s, double *e) {
    for (long long i = 0; i < n; ++i) sphx::two_sum<double>(a[i], b[i], s[i], e[i]);
}
