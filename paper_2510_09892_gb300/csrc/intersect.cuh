// Per-pair intersection of one great circle arc (x1, x2) with one latitude
// z = z0: Eq. 2.2 of arXiv 2510.09892 evaluated four ways (direct FP64,
// AccuX in FP64, float-float, integer limbs), followed by the on-arc test.
//
// Conventions (shared by every mode):
//   count = -1  computed n = 0 (x1 parallel to x2), or n_xy = 0 and z0 = 0
//               (the arc lies on the equator: coincident circles);
//   count = 0   no hit, also for any non-finite input and for n_xy = 0,
//               z0 != 0 (parallel planes);
//   slot 0      the upper sign of Eq. 2.2 (the alpha* <= 0 root that
//               Algorithm 8 returns), slot 1 the lower sign;
//   tangency    computed s^2 == 0 gives one candidate, in slot 0;
//   on-arc      with m1 = n x x1 and m2 = x2 x n, a candidate P is kept iff
//               P . m1 >= 0 and P . m2 >= 0 (that is (x1 x P).n >= 0 and
//               (P x x2).n >= 0: P between x1 and x2 on the minor arc).
#pragma once
#include "eft.cuh"
#include "ff.cuh"
#include "wide.cuh"

namespace sphx {

enum : int { kDirect = 0, kEftFp64 = 1, kEftFf32 = 2, kEftFp64Printed = 3, kWideInt = 4 };

struct PairOut {
    int count;      // -1, 0, 1, 2
    bool hit[2];    // slot r holds a hit
    double px[2], py[2];
};

// Tests of doubles on the integer pipe (GB300 issues FP64 instructions,
// comparisons included, at 2 per SM per clock), each with the FP64 test's
// result for every input: NaN compares false, -0 equals +0.
SPHX_HD bool finite_bits(double x) {  // isfinite(x)
    return ((wide::bits_of(x) >> 52) & 0x7ff) != 0x7ff;
}
SPHX_HD bool eq_zero(double x) { return (wide::bits_of(x) << 1) == 0; }  // x == 0
SPHX_HD bool ge_zero(double x) {                                          // x >= 0
    const uint64_t b = wide::bits_of(x);
    return b <= 0x7ff0000000000000ull || b == 0x8000000000000000ull;
}
SPHX_HD bool gt_zero(double x) { return wide::bits_of(x) - 1u < 0x7ff0000000000000ull; }  // x > 0
SPHX_HD bool le_zero(double x) {                                          // x <= 0
    const uint64_t b = wide::bits_of(x);
    return b == 0u || (b >= 0x8000000000000000ull && b <= 0xfff0000000000000ull);
}

EFT_HD bool finite7(const double (&x1)[3], const double (&x2)[3], double z0) {
    // bitwise &: one test of the seven exponent fields, no branch per value
    return finite_bits(x1[0]) & finite_bits(x1[1]) & finite_bits(x1[2]) & finite_bits(x2[0]) &
           finite_bits(x2[1]) & finite_bits(x2[2]) & finite_bits(z0);
}

SPHX_HD void clear(PairOut &o, int count) {
    o.count = count;
    o.hit[0] = o.hit[1] = false;
    o.px[0] = o.px[1] = o.py[0] = o.py[1] = 0.0;
}

// ---- Sec. 4: direct FP64 translation of Eq. 2.2 (no FMA anywhere) -----------
EFT_HD void pair_direct(const double (&x1)[3], const double (&x2)[3],
                                            double z0, PairOut &o) {
    if (!finite7(x1, x2, z0)) return clear(o, 0);
    double nx = sub(mul(x1[1], x2[2]), mul(x1[2], x2[1]));
    double ny = sub(mul(x1[2], x2[0]), mul(x1[0], x2[2]));
    double nz = sub(mul(x1[0], x2[1]), mul(x1[1], x2[0]));
    double S2 = add(mul(nx, nx), mul(ny, ny));
    double S3 = add(S2, mul(nz, nz));
    if (eq_zero(S3)) return clear(o, -1);
    if (eq_zero(S2)) return clear(o, eq_zero(z0) ? -1 : 0);
    double s2 = sub(S2, mul(S3, mul(z0, z0)));
    if (!ge_zero(s2)) return clear(o, 0);
    double s = sqrt_(s2);
    double a = mul(mul(z0, nx), nz);
    double b = mul(mul(z0, ny), nz);
    double sny = mul(s, ny), snx = mul(s, nx);
    double m1x = sub(mul(ny, x1[2]), mul(nz, x1[1]));
    double m1y = sub(mul(nz, x1[0]), mul(nx, x1[2]));
    double m1z = sub(mul(nx, x1[1]), mul(ny, x1[0]));
    double m2x = sub(mul(x2[1], nz), mul(x2[2], ny));
    double m2y = sub(mul(x2[2], nx), mul(x2[0], nz));
    double m2z = sub(mul(x2[0], ny), mul(x2[1], nx));
    const int nroots = gt_zero(s2) ? 2 : 1;
    o.count = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        o.hit[r] = false;
        if (r >= nroots) continue;
        double X = r == 0 ? add(a, sny) : sub(a, sny);
        double Y = r == 0 ? sub(b, snx) : add(b, snx);
        double Px = -div_(X, S2);
        double Py = -div_(Y, S2);
        double t1 = add(add(mul(Px, m1x), mul(Py, m1y)), mul(z0, m1z));
        double t2 = add(add(mul(Px, m2x), mul(Py, m2y)), mul(z0, m2z));
        o.px[r] = Px;
        o.py[r] = Py;
        if (ge_zero(t1) && ge_zero(t2)) {
            o.hit[r] = true;
            ++o.count;
        }
    }
}

// ---- Algorithm 8 (AccuX) in FP64, both roots --------------------------------
// mid (optional): Algorithm 8's pairs for the intermediate-error analysis of
// App. A, 16 doubles: n[3], en[3], S2, s2, S3, s3, ss, ess, sb, es, X (root
// 0's x-coordinate numerator), 0 -- zeros past the point where the arc stops
template <bool Renorm>
EFT_HD void pair_accux(const double (&x1)[3], const double (&x2)[3],
                                           double z0, PairOut &o, double *mid = nullptr) {
    if (mid) {
#pragma unroll
        for (int k = 0; k < 16; ++k) mid[k] = 0.0;
    }
    if (!finite7(x1, x2, z0)) return clear(o, 0);
    // n = x1 x x2 as three compensated pairs
    double n[3], en[3];
    accu_dop<double, Renorm>(x1[1], x1[2], x2[1], x2[2], n[0], en[0]);  // y1 z2 - z1 y2
    accu_dop<double, Renorm>(x1[2], x1[0], x2[2], x2[0], n[1], en[1]);  // z1 x2 - x1 z2
    accu_dop<double, Renorm>(x1[0], x1[1], x2[0], x2[1], n[2], en[2]);  // x1 y2 - y1 x2
    double S2, s2, S3, s3;
    {
        const double nxy[2] = {n[0], n[1]}, exy[2] = {en[0], en[1]};
        sum_of_squares_c<double, 2>(nxy, exy, S2, s2);
        sum_of_squares_c<double, 3>(n, en, S3, s3);
    }
    if (mid) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            mid[k] = n[k];
            mid[3 + k] = en[k];
        }
        mid[6] = S2;
        mid[7] = s2;
        mid[8] = S3;
        mid[9] = s3;
    }
    if (eq_zero(S3)) return clear(o, -1);
    if (eq_zero(S2)) return clear(o, eq_zero(z0) ? -1 : 0);
    // s^2 = |n_xy|^2 - |n|^2 z0^2 as a pair
    double C, eC, D, eD, E, eE;
    two_prod(z0, z0, C, eC);
    {
        const double xs[4] = {S3, S3, s3, s3}, ys[4] = {C, eC, C, eC};
        comp_dot_c<double, 4>(xs, ys, D, eD);
    }
    two_sum(S2, -D, E, eE);
    double e = add(sub(s2, eD), eE);
    double ss, ess;
    fast_two_sum(E, e, ss, ess);
    if (mid) {
        mid[10] = ss;
        mid[11] = ess;
    }
    if (!ge_zero(ss)) return clear(o, 0);
    double sb, es;
    acc_sqrt(ss, ess, sb, es);
    if (mid) {
        mid[12] = sb;
        mid[13] = es;
    }
    // F = n_x n_z and n_y n_z with their first-order compensation terms
    double Fx, eFx, Fy, eFy;
    two_prod(n[0], n[2], Fx, eFx);
    eFx = add(add(eFx, mul(n[0], en[2])), mul(n[2], en[0]));
    two_prod(n[1], n[2], Fy, eFy);
    eFy = add(add(eFy, mul(n[1], en[2])), mul(n[2], en[1]));
    // containment vectors from the leading parts of n
    double m1x = fma_(n[1], x1[2], -mul(n[2], x1[1]));
    double m1y = fma_(n[2], x1[0], -mul(n[0], x1[2]));
    double m1z = fma_(n[0], x1[1], -mul(n[1], x1[0]));
    double m2x = fma_(x2[1], n[2], -mul(x2[2], n[1]));
    double m2y = fma_(x2[2], n[0], -mul(x2[0], n[2]));
    double m2z = fma_(x2[0], n[1], -mul(x2[1], n[0]));
    const int nroots = gt_zero(ss) ? 2 : 1;
    o.count = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        o.hit[r] = false;
        if (r >= nroots) continue;
        const double sg = r == 0 ? sb : -sb;
        const double eg = r == 0 ? es : -es;
        const double xa[6] = {Fx, eFx, n[1], en[1], n[1], en[1]};
        const double yy[6] = {z0, z0, sg, sg, eg, eg};
        const double xb[6] = {Fy, eFy, -n[0], -en[0], -n[0], -en[0]};
        double X = comp_dot<double, 6>(xa, yy);
        double Y = comp_dot<double, 6>(xb, yy);
        if (mid && r == 0) mid[14] = X;
        double Px = -div_(X, S2);
        double Py = -div_(Y, S2);
        double t1 = fma_(Px, m1x, fma_(Py, m1y, mul(z0, m1z)));
        double t2 = fma_(Px, m2x, fma_(Py, m2y, mul(z0, m2z)));
        o.px[r] = Px;
        o.py[r] = Py;
        if (ge_zero(t1) && ge_zero(t2)) {
            o.hit[r] = true;
            ++o.count;
        }
    }
}

// ---- Eq. 2.2 in multi-limb integer arithmetic (wide.cuh) ----------------------
// The normal n = x1 x x2 is formed from exact 106-bit products of the FP64
// inputs and carried with 128-bit mantissas through |n_xy|^2, |n|^2 and
// s^2 = |n_xy|^2 - |n|^2 z0^2, the steps whose cancellation the paper's error
// analysis is about (Sec. 4, 6.1); the square root, the numerators
// z0 n_x n_z +- s n_y, z0 n_y n_z -+ s n_x and the division by |n_xy|^2 follow
// with 96-bit mantissas (every numerator term is at most sqrt(1 - z0^2)
// |n_xy|^2 in magnitude, so 96 bits leave each coordinate within a fraction
// of an ulp). The square root and the reciprocal start from FP32 seeds and
// are refined by fixed-point Newton steps on the limbs (recip_int, sqrt_int).
// The only FP64 arithmetic left is the on-arc offsets; everything else runs
// on the 32-bit integer pipe.
//
// On-arc test: t1 = (x1 x P).n = d1 . m1 with m1 = n x x1 and
// d1 = P - l x1, l = +-1/|x1| (the sign of P . x1): x1 . m1 = 0, so any l
// gives the same value, and this choice keeps |d1| |m1| within a factor
// sqrt(2) of |t1| wherever t1 is small, so m1 and d1 in FP32 (d1 from one
// FP64 FMA per component) decide its sign correctly except within an angle
// of about 2^-40 of the endpoint (the oracle's near-endpoint flag).
// Likewise t2 = (P x x2).n = d2 . m2.

SPHX_HD int exponent_bits(double x) {  // unbiased; very small for 0
    const int ex = (int)((wide::bits_of(x) >> 52) & 0x7ff);
    return ex ? ex - 1023 : -2000;
}

// x 2^-sc as a float (mantissa truncated; 0 below the float range)
SPHX_HD float f32_scaled(double x, int sc) {
    const uint64_t b = wide::bits_of(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    const int fe = ex - 1023 + 127 - sc;
    if (ex == 0 || fe <= 0) return 0.0f;
    return wide::float_of(((uint32_t)(b >> 63) << 31) | ((uint32_t)(fe > 254 ? 254 : fe) << 23) |
                          (uint32_t)((b >> 29) & 0x7fffffu));
}

// f32_scaled(x, 0) in fewer instructions, bit for bit for every input: a
// funnel shift brings the double's low 9 exponent bits and top 23 mantissa
// bits into place, and keeping 8 bits of (exponent - 384) gives the float's
// exponent field (1023 - 127 = 896 = 512 + 384) over the whole float range
SPHX_HD float f32_of(double x) {
    const uint64_t b = wide::bits_of(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t f = wide::funnel_l(lo, hi, 3), sign = hi & 0x80000000u, e2 = hi << 1;
    const uint32_t v = e2 >= (1151u << 21) ? (sign | (254u << 23) | (f & 0x7fffffu))
                                           : (((f - (384u << 23)) & 0x7fffffffu) | sign);
    return e2 >= (897u << 21) ? wide::float_of(v) : 0.0f;
}

// 0.M 2^(e - emax) of a W<4> as a float
SPHX_HD float f32_rel(const wide::W<4> &a, int emax) {
    const int fe = a.e - emax + 126;
    if (wide::is_zero(a) || fe <= 0) return 0.0f;
    return wide::float_of((a.neg << 31) | ((uint32_t)fe << 23) | ((a.m[3] >> 8) & 0x7fffffu));
}

// a positive normal float times 2^-sc, as a double (exact)
SPHX_HD double f64_of_f32_scaled(float f, int sc) {
    const uint32_t b = wide::fbits_of(f);
    const int fe = (int)((b >> 23) & 0xff);
    return wide::double_of(((uint64_t)(fe - 127 + 1023 - sc) << 52) | ((uint64_t)(b & 0x7fffffu) << 29));
}

// The exact and 128-bit part of the integer-limb evaluation: n, |n_xy|^2 and
// s^2 = |n_xy|^2 - |n|^2 z0^2, the quantities whose cancellation the paper's
// error analysis is about. Returns false after filling `o` for the cases that
// end here (non-finite input, degenerate arc, no candidate).
struct WideCore {
    wide::W<4> n[3], S2, s2;
    bool tangent;
};

SPHX_HD bool wide_core(const double (&x1)[3], const double (&x2)[3], double z0, WideCore &c,
                       PairOut &o) {
    using namespace wide;
    if (!(finite_bits(x1[0]) && finite_bits(x1[1]) && finite_bits(x1[2]) && finite_bits(x2[0]) &&
          finite_bits(x2[1]) && finite_bits(x2[2]) && finite_bits(z0))) {
        clear(o, 0);
        return false;
    }
    W<2> a[3], b[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        a[i] = from_double<2>(x1[i]);
        b[i] = from_double<2>(x2[i]);
    }
    c.n[0] = sub<4>(mul_exact(a[1], b[2]), mul_exact(a[2], b[1]));  // y1 z2 - z1 y2
    c.n[1] = sub<4>(mul_exact(a[2], b[0]), mul_exact(a[0], b[2]));  // z1 x2 - x1 z2
    c.n[2] = sub<4>(mul_exact(a[0], b[1]), mul_exact(a[1], b[0]));  // x1 y2 - y1 x2
    if (is_zero(c.n[0]) && is_zero(c.n[1]) && is_zero(c.n[2])) {
        clear(o, -1);
        return false;
    }
    const bool z0_zero = (bits_of(z0) << 1) == 0;
    if (is_zero(c.n[0]) && is_zero(c.n[1])) {
        clear(o, z0_zero ? -1 : 0);
        return false;
    }
    c.S2 = add_same<4>(sqr<4>(c.n[0]), sqr<4>(c.n[1]));
    const W<4> S3 = add_same<4>(c.S2, sqr<4>(c.n[2]));
    const W<2> zz = from_double<2>(z0);
    c.s2 = sub<4>(c.S2, mul<4>(S3, mul_exact(zz, zz)));
    if (c.s2.neg && !is_zero(c.s2)) {
        clear(o, 0);
        return false;
    }
    c.tangent = is_zero(c.s2);
    return true;
}

// Set-up of the on-arc test (FP32 normals and endpoints, scaled by powers of
// two), placed before the root computation so that its latency overlaps that
// work.
struct OnArc {
    float p1[3], p2[3], m1[3], m2[3], zf;
    double inv1, inv2;
};

SPHX_HD void onarc_setup(const double (&x1)[3], const double (&x2)[3], double z0,
                         const WideCore &c, OnArc &q) {
    using namespace wide;
    int emax = c.n[0].e;
    emax = c.n[1].e > emax ? c.n[1].e : emax;
    emax = c.n[2].e > emax ? c.n[2].e : emax;
    const float nf[3] = {f32_rel(c.n[0], emax), f32_rel(c.n[1], emax), f32_rel(c.n[2], emax)};
    int sc1 = exponent_bits(x1[0]), sc2 = exponent_bits(x2[0]);
#pragma unroll
    for (int i = 1; i < 3; ++i) {
        const int e1 = exponent_bits(x1[i]), e2 = exponent_bits(x2[i]);
        sc1 = e1 > sc1 ? e1 : sc1;
        sc2 = e2 > sc2 ? e2 : sc2;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        q.p1[i] = f32_scaled(x1[i], sc1);
        q.p2[i] = f32_scaled(x2[i], sc2);
    }
    const float *p1 = q.p1, *p2 = q.p2;
    q.m1[0] = wide::fma32(nf[1], p1[2], -nf[2] * p1[1]);
    q.m1[1] = wide::fma32(nf[2], p1[0], -nf[0] * p1[2]);
    q.m1[2] = wide::fma32(nf[0], p1[1], -nf[1] * p1[0]);
    q.m2[0] = wide::fma32(p2[1], nf[2], -p2[2] * nf[1]);
    q.m2[1] = wide::fma32(p2[2], nf[0], -p2[0] * nf[2]);
    q.m2[2] = wide::fma32(p2[0], nf[1], -p2[1] * nf[0]);
    // l = 1 / |x| in FP32, except that endpoints of unit norm (to FP32
    // resolution) take l = 1 exactly: then d = P -+ x is exact near x
    const float r1 = wide::rsqrt_approx(p1[0] * p1[0] + p1[1] * p1[1] + p1[2] * p1[2]);
    const float r2 = wide::rsqrt_approx(p2[0] * p2[0] + p2[1] * p2[1] + p2[2] * p2[2]);
    const bool unit1 = (sc1 == -1 || sc1 == 0) && fabsf(r1 * (sc1 ? 2.0f : 1.0f) - 1.0f) < 1e-6f;
    const bool unit2 = (sc2 == -1 || sc2 == 0) && fabsf(r2 * (sc2 ? 2.0f : 1.0f) - 1.0f) < 1e-6f;
    q.inv1 = unit1 ? 1.0 : f64_of_f32_scaled(r1, sc1);
    q.inv2 = unit2 ? 1.0 : f64_of_f32_scaled(r2, sc2);
    q.zf = f32_scaled(z0, 0);
}

// the on-arc decision for the candidate (Px, Py, z0)
SPHX_HD bool onarc_test(const double (&x1)[3], const double (&x2)[3], double z0, const OnArc &q,
                        double Px, double Py) {
    const float pf[3] = {f32_scaled(Px, 0), f32_scaled(Py, 0), q.zf};
    const double l1 = (pf[0] * q.p1[0] + pf[1] * q.p1[1] + pf[2] * q.p1[2] >= 0.0f) ? q.inv1 : -q.inv1;
    const double l2 = (pf[0] * q.p2[0] + pf[1] * q.p2[1] + pf[2] * q.p2[2] >= 0.0f) ? q.inv2 : -q.inv2;
    const float d1[3] = {f32_scaled(wide::fma64(-l1, x1[0], Px), 0),
                         f32_scaled(wide::fma64(-l1, x1[1], Py), 0),
                         f32_scaled(wide::fma64(-l1, x1[2], z0), 0)};
    const float d2[3] = {f32_scaled(wide::fma64(-l2, x2[0], Px), 0),
                         f32_scaled(wide::fma64(-l2, x2[1], Py), 0),
                         f32_scaled(wide::fma64(-l2, x2[2], z0), 0)};
    const float t1 = wide::fma32(d1[0], q.m1[0], wide::fma32(d1[1], q.m1[1], d1[2] * q.m1[2]));
    const float t2 = wide::fma32(d2[0], q.m2[0], wide::fma32(d2[1], q.m2[1], d2[2] * q.m2[2]));
    return t1 >= 0.0f && t2 >= 0.0f;
}

SPHX_HD void pair_wide(const double (&x1)[3], const double (&x2)[3], double z0,
                                          PairOut &o) {
    using namespace wide;
    WideCore c;
    if (!wide_core(x1, x2, z0, c, o)) return;
    OnArc q;
    onarc_setup(x1, x2, z0, c, q);
    // P_xy = g n_xy + sigma h (n_y, -n_x) with g = -z0 n_z / |n_xy|^2 and
    // h = -s / |n_xy|^2: Eq. 2.2 with the division distributed
    const W<3> nx = narrow<4, 3>(c.n[0]), ny = narrow<4, 3>(c.n[1]), nz = narrow<4, 3>(c.n[2]);
    const W<3> rS2 = negate<3>(recip_int<3>(narrow<4, 3>(c.S2)));  // -1 / |n_xy|^2
    const W<3> g = mul<3>(mul<3>(from_double<3>(z0), nz), rS2);
    const W<3> h = c.tangent ? zero<3>() : mul<3>(sqrt_int<3>(narrow<4, 3>(c.s2)), rS2);
    const W<3> gx = mul<3>(g, nx), gy = mul<3>(g, ny);
    const W<3> hx = mul<3>(h, nx), hy = mul<3>(h, ny);
    W<3> Px_lin[2], Py_lin[2];  // both roots: g n_x +- h n_y and g n_y -+ h n_x
    add_sub<3>(gx, hy, Px_lin[0], Px_lin[1]);
    add_sub<3>(gy, hx, Py_lin[1], Py_lin[0]);

    const int nroots = c.tangent ? 1 : 2;
    o.count = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        o.hit[r] = false;
        if (r >= nroots) continue;
        const double Px = to_double<3>(Px_lin[r]);
        const double Py = to_double<3>(Py_lin[r]);
        o.px[r] = Px;
        o.py[r] = Py;
        if (onarc_test(x1, x2, z0, q, Px, Py)) {
            o.hit[r] = true;
            ++o.count;
        }
    }
}

// ---- float-float tail on the exact core --------------------------------------
// The cancelling steps stay exact or 128-bit on the integer limbs (wide_core:
// the cross product of nearly coincident or nearly antipodal endpoints and
// s^2 = |n_xy|^2 - |n|^2 z0^2, whose sign decides whether the circles meet);
// everything after them runs in float-float on the FP32 pipe: with F the
// exponent of the larger of |n_x|, |n_y|, the quantities b = n_xy 2^-F,
// T = |n_xy|^2 2^-2F in [1/4, 2), sigma = s^2 2^-2F <= T and Z = z0 n_z 2^-F
// (|Z| <= sqrt(T) whenever s^2 >= 0) are rounded to pairs (2^-49), and
//
//     P_x = G b_x +- H b_y,  P_y = G b_y -+ H b_x,
//     G = -Z / T,  H = -sqrt(sigma) / T
//
// (Eq. 2.2: g n_x = G b_x with g = -z0 n_z / |n_xy|^2, h n_y = H b_y with
// h = -s / |n_xy|^2). With eps = 2^-48 and the pair operations' relative
// errors (products <= 3 eps, reciprocal and square root <= 3 eps, sums of
// pairs <= 2 eps of the operands' magnitudes), each term G b and H b is within
// 13 eps of its value and each coordinate within 15 eps (|g n_x| + |h n_y|),
// so |dP| <= 15 eps sqrt(2) sqrt(1 - z0^2) < 2^-44 sqrt(1 - z0^2) (the terms
// are bounded by sqrt(1 - z0^2), |g n_xy|^2 + |h n_xy|^2 = 1 - z0^2). The
// hit count follows the exact sign of s^2 and the on-arc test of pair_wide
// (P within 2^-44 moves no decision outside the oracle's 2^-40 endpoint
// flag).
SPHX_HD void pair_ff32(const double (&x1)[3], const double (&x2)[3], double z0, PairOut &o) {
    using namespace wide;
    using namespace ffa;
    WideCore c;
    if (!wide_core(x1, x2, z0, c, o)) return;
    OnArc q;
    onarc_setup(x1, x2, z0, c, q);
    const int F = c.n[0].e > c.n[1].e ? c.n[0].e : c.n[1].e;
    const F2 bx = ff_of<4>(c.n[0], F), by = ff_of<4>(c.n[1], F);
    const F2 T = ff_of<4>(c.S2, 2 * F);
    const F2 sig = c.tangent ? F2{0.0f, 0.0f} : ff_of<4>(c.s2, 2 * F);
    const F2 Z = ff_of<3>(mul<3>(from_double<3>(z0), narrow<4, 3>(c.n[2])), F);
    const F2 iT = rcp2(T);
    const F2 G = neg(mul2(Z, iT));
    const F2 H = neg(mul2(sqrt2(sig), iT));
    const F2 gx = mul2(G, bx), gy = mul2(G, by), hx = mul2(H, bx), hy = mul2(H, by);
    const int nroots = c.tangent ? 1 : 2;
    o.count = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        o.hit[r] = false;
        if (r >= nroots) continue;
        const F2 X = add2(gx, r == 0 ? hy : neg(hy));
        const F2 Y = add2(gy, r == 0 ? neg(hx) : hx);
        const double Px = to_f64(X.hi) + to_f64(X.lo);
        const double Py = to_f64(Y.hi) + to_f64(Y.lo);
        o.px[r] = Px;
        o.py[r] = Py;
        if (onarc_test(x1, x2, z0, q, Px, Py)) {
            o.hit[r] = true;
            ++o.count;
        }
    }
}

template <int Mode>
EFT_HD void intersect_pair(const double (&x1)[3], const double (&x2)[3], double z0, PairOut &o) {
    if (Mode == kDirect)
        pair_direct(x1, x2, z0, o);
    else if (Mode == kEftFp64)
        pair_accux<true>(x1, x2, z0, o);
    else if (Mode == kEftFp64Printed)
        pair_accux<false>(x1, x2, z0, o);
    else if (Mode == kWideInt)
        pair_wide(x1, x2, z0, o);
    else
        pair_ff32(x1, x2, z0, o);
}

}  // namespace sphx
