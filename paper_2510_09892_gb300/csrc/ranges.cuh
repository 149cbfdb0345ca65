// Height ranges of arcs and searches in sorted latitude arrays, shared by the
// ragged call (candidate latitudes per edge) and the band-area call (bands
// per cell, latitudes per arc piece).
#pragma once
#include "intersect.cuh"

namespace sphx {

// three device intrinsics with host equivalents, so that the functions below
// also build for the host (tests); the device code is unchanged
EFT_HD double rsqrt_hd(double x) {
#if defined(__CUDA_ARCH__)
    return rsqrt(x);
#else
    return 1.0 / sqrt(x);
#endif
}

EFT_HD float rsqrtf_hd(float x) {
#if defined(__CUDA_ARCH__)
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}

EFT_HD int hi_word(double v) {
#if defined(__CUDA_ARCH__)
    return __double2hiint(v);
#else
    return (int)(wide::bits_of(v) >> 32);
#endif
}

// first index i in [0, n) with a[i] > key (n if none)
template <typename T>
EFT_HD int64_t upper_bound_dev(const T *a, int64_t n, T key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] > key)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}
// An order-preserving integer image of a double (not NaN): comparing the
// images compares the values, with no FP64 instruction (GB300 issues FP64
// comparisons at 2 per SM per clock, 64-bit integer ones far faster).
// -0.0 maps just below +0.0, which only matters for keys that widen a range.
EFT_HD long long ord64(double x) {
    const long long b = (long long)wide::bits_of(x);
    return b < 0 ? (b ^ 0x7fffffffffffffffLL) : b;
}

// first index i in [0, n) with a[i] >= key (by ord64)
EFT_HD int64_t lower_bound_ord(const double *a, int64_t n, long long key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (ord64(a[mid]) >= key)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// first index i in [0, n) with a[i] > key (by ord64)
EFT_HD int64_t upper_bound_ord(const double *a, int64_t n, long long key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (ord64(a[mid]) > key)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// first index i in [from, n) with a[i] > key (by ord64), found by galloping
// forward from `from` (steps 1, 2, 4, ... then a binary search): a few loads
// when the answer is near `from`, as for the short ranges of latitudes an arc
// spans
EFT_HD int64_t upper_bound_ord_from(const double *a, int64_t n, int64_t from,
                                    long long key) {
    int64_t lo = from, hi = from, step = 1;
    while (hi < n && ord64(a[hi]) <= key) {
        lo = hi + 1;
        hi += step;
        step <<= 1;
    }
    if (hi > n) hi = n;
    while (lo < hi) {  // a[lo - 1] <= key (or lo == from); a[hi] > key or hi == n
        const int64_t mid = (lo + hi) >> 1;
        if (ord64(a[mid]) > key)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// a float in [-2, 2] as a double, by its bits (values below 2^-126 become +-0)
EFT_HD double f64_of_f32_small(float f) {
    const uint32_t b = wide::fbits_of(f);
    const uint32_t fe = (b >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    if (fe == 0) return wide::double_of(sign);
    return wide::double_of(sign | ((uint64_t)(fe - 127u + 1023u) << 52) |
                           ((uint64_t)(b & 0x7fffffu) << 29));
}

constexpr double kZWiden = 1e-13;

// binary exponent of |v| for a finite nonzero double (floor(log2 |v|))
EFT_HD int exponent_of(double v) {
    int hi = hi_word(v);
    int ex = (hi >> 20) & 0x7ff;
    if (ex == 0) return ilogb(v);  // subnormal
    return ex - 1023;
}

// z-range of the minor arc x1 -> x2 in FP64: the endpoints' z and, when the
// arc passes it, the great circle's highest (or lowest) point +-|n_xy| / |n|,
// widened by 1e-13; false for a degenerate or non-finite arc
EFT_HD bool z_range_fp64(const double (&x1)[3], const double (&x2)[3],
                         double &zmin, double &zmax) {
    double n[3], en[3];
    accu_dop<double, true>(x1[1], x1[2], x2[1], x2[2], n[0], en[0]);
    accu_dop<double, true>(x1[2], x1[0], x2[2], x2[0], n[1], en[1]);
    accu_dop<double, true>(x1[0], x1[1], x2[0], x2[1], n[2], en[2]);
    if (!finite7(x1, x2, 0.0) || (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0)) return false;
    const double z1 = x1[2] * rsqrt_hd(x1[0] * x1[0] + x1[1] * x1[1] + x1[2] * x1[2]);
    const double z2 = x2[2] * rsqrt_hd(x2[0] * x2[0] + x2[1] * x2[1] + x2[2] * x2[2]);
    zmin = fmin(z1, z2);
    zmax = fmax(z1, z2);
    // scale n to avoid underflow in the squares of very short arcs
    const double amax = fmax(fabs(n[0]), fmax(fabs(n[1]), fabs(n[2])));
    const double sc = ldexp(1.0, -exponent_of(amax));
    const double nx = n[0] * sc, ny = n[1] * sc, nz = n[2] * sc;
    const double S2 = nx * nx + ny * ny, S3 = S2 + nz * nz;
    // highest point of the great circle: a = (-nx nz, -ny nz, S2); it is on
    // the arc iff a . (n x x1) >= 0 and a . (x2 x n) >= 0 (the lowest is -a)
    const double ax = -nx * nz, ay = -ny * nz, az = S2;
    const double m1x = ny * x1[2] - nz * x1[1], m1y = nz * x1[0] - nx * x1[2],
                 m1z = nx * x1[1] - ny * x1[0];
    const double m2x = x2[1] * nz - x2[2] * ny, m2y = x2[2] * nx - x2[0] * nz,
                 m2z = x2[0] * ny - x2[1] * nx;
    const double t1 = ax * m1x + ay * m1y + az * m1z;
    const double t2 = ax * m2x + ay * m2y + az * m2z;
    const double zap = sqrt(S2 / S3);
    if (t1 >= 0.0 && t2 >= 0.0) zmax = zap;
    if (t1 <= 0.0 && t2 <= 0.0) zmin = -zap;
    zmin -= kZWiden;
    zmax += kZWiden;
    return true;
}

// The same z-range in FP32 for endpoints of unit norm (to 2^-20), widened by
// kZWiden32. With d = x2 - x1 (or x2 + x1 when x1 . x2 < 0) from one FP64
// subtraction per component, n = x1 x d equals x1 x x2 and stays
// well-conditioned for short and for nearly antipodal arcs (d makes an angle
// of at least 45 degrees with x1), so every FP32 quantity below -- the
// endpoints' z, n, |n_xy|^2, |n|^2 and the apex height |n_xy| / |n| -- is
// within a few units of 2^-24 of its exact value: at most about 6e-7 in z,
// three times below the widening. A wrong apex decision needs the apex within
// about 1e-6 rad of an endpoint, where the two heights differ by ~1e-12.
// Returns false when the fast path does not apply (non-unit or non-finite
// endpoints, or |n| below the FP32 range).
constexpr float kZWiden32 = 1.0f / (1 << 19);

//
// Short arcs take a shorter path: a circular arc stays within its sagitta
// 1 - cos(L/2) <= L^2 / 8 of its chord, so its heights exceed the endpoints'
// by at most that; with the chord |x2 - x1| <= 2^-9 (from FP32 differences,
// within 2.2e-6 of the exact one for endpoints of norm 1 +- 1e-6), L^2 / 8 <=
// 0.31 |x2 - x1|^2 < 1.2e-6, and with the endpoints' FP32 heights (error below
// 2.5e-7) the same widening 2^-19 = 1.9e-6 covers it: no cross product, no
// apex test and no FP64 difference are needed.
constexpr float kShortChord2 = 1.0f / (1 << 18);

EFT_HD bool z_range_fp32(const double (&x1)[3], const double (&x2)[3],
                         double &zmin, double &zmax) {
    float p1[3], p2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        p1[i] = f32_of(x1[i]);
        p2[i] = f32_of(x2[i]);
    }
    const float q1 = p1[0] * p1[0] + p1[1] * p1[1] + p1[2] * p1[2];
    const float q2 = p2[0] * p2[0] + p2[1] * p2[1] + p2[2] * p2[2];
    if (!(fabsf(q1 - 1.0f) < 1e-6f && fabsf(q2 - 1.0f) < 1e-6f)) return false;
    {
        const float dx = p2[0] - p1[0], dy = p2[1] - p1[1], dz = p2[2] - p1[2];
        if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= kShortChord2) {
            const float z1 = p1[2] * rsqrtf_hd(q1), z2 = p2[2] * rsqrtf_hd(q2);
            zmin = f64_of_f32_small(fminf(z1, z2) - kZWiden32);
            zmax = f64_of_f32_small(fmaxf(z1, z2) + kZWiden32);
            return true;
        }
    }
    const double sg = (p1[0] * p2[0] + p1[1] * p2[1] + p1[2] * p2[2] >= 0.0f) ? 1.0 : -1.0;
    float d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = f32_of(x2[i] - sg * x1[i]);
    const float nx = fmaf(p1[1], d[2], -p1[2] * d[1]);
    const float ny = fmaf(p1[2], d[0], -p1[0] * d[2]);
    const float nz = fmaf(p1[0], d[1], -p1[1] * d[0]);
    const float S2 = fmaf(nx, nx, ny * ny), S3 = fmaf(nz, nz, S2);
    if (!(S3 > 1e-30f)) return false;
    const float z1 = p1[2] * rsqrtf_hd(q1), z2 = p2[2] * rsqrtf_hd(q2);
    float lo = fminf(z1, z2), hi = fmaxf(z1, z2);
    const float ax = -nx * nz, ay = -ny * nz, az = S2;
    const float m1x = fmaf(ny, p1[2], -nz * p1[1]), m1y = fmaf(nz, p1[0], -nx * p1[2]),
                m1z = fmaf(nx, p1[1], -ny * p1[0]);
    const float m2x = fmaf(p2[1], nz, -p2[2] * ny), m2y = fmaf(p2[2], nx, -p2[0] * nz),
                m2z = fmaf(p2[0], ny, -p2[1] * nx);
    const float t1 = fmaf(ax, m1x, fmaf(ay, m1y, az * m1z));
    const float t2 = fmaf(ax, m2x, fmaf(ay, m2y, az * m2z));
    const float zap = sqrtf(S2 / S3);
    if (t1 >= 0.0f && t2 >= 0.0f) hi = zap;
    if (t1 <= 0.0f && t2 <= 0.0f) lo = -zap;
    zmin = f64_of_f32_small(lo - kZWiden32);
    zmax = f64_of_f32_small(hi + kZWiden32);
    return true;
}

}  // namespace sphx
