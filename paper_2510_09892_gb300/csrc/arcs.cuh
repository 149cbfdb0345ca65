// Per-pair intersection of two great circle arcs a = (a1, a2), b = (b1, b2):
// three cross products followed by a normalisation (Sec. 1 of arXiv 2510.09892;
// Sec. 9 names it as a use of the accurate cross product). The great circles
// meet at +-v / |v|, v = n_a x n_b with n_a = a1 x a2, n_b = b1 x b2; slot 0
// holds +v / |v|, slot 1 -v / |v|; a slot is a hit iff the point lies on both
// closed minor arcs, (x1 x p) . n >= 0 and (p x x2) . n >= 0 for each arc.
//   count = -1  an arc's normal is 0, or both arcs lie on one great circle
//   count = 0   no hit; also for non-finite inputs
#pragma once
#include "intersect.cuh"

namespace sphx {

// On-arc test values of +p for the four endpoints (those of -p are their
// negatives). As in pair_wide: t = (p - l x) . m with m = n x x1 or x2 x n in
// FP32 and l = +-1/|x| (the sign of p . x; exactly +-1 for unit endpoints),
// p - l x by one FP64 FMA per component, which keeps |p - l x| |m| within a
// factor sqrt(2) of |t| where t is small.
struct ArcEnds {
    float p[3];     // the endpoint in FP32, scaled by a power of two
    float m[3];     // n x x for a first endpoint, x x n for a second one
    double inv;     // l magnitude: 1 / |x| (exactly 1 for unit endpoints)
};

SPHX_HD void arc_end(const double (&x)[3], const float (&nf)[3], bool first, ArcEnds &e) {
    int sc = exponent_bits(x[0]);
#pragma unroll
    for (int i = 1; i < 3; ++i) sc = exponent_bits(x[i]) > sc ? exponent_bits(x[i]) : sc;
#pragma unroll
    for (int i = 0; i < 3; ++i) e.p[i] = f32_scaled(x[i], sc);
    const float *a = first ? nf : e.p;
    const float *b = first ? e.p : nf;
    e.m[0] = wide::fma32(a[1], b[2], -a[2] * b[1]);
    e.m[1] = wide::fma32(a[2], b[0], -a[0] * b[2]);
    e.m[2] = wide::fma32(a[0], b[1], -a[1] * b[0]);
    const float r = wide::rsqrt_approx(e.p[0] * e.p[0] + e.p[1] * e.p[1] + e.p[2] * e.p[2]);
    const bool unit = (sc == -1 || sc == 0) && fabsf(r * (sc ? 2.0f : 1.0f) - 1.0f) < 1e-6f;
    e.inv = unit ? 1.0 : f64_of_f32_scaled(r, sc);
}

SPHX_HD float arc_end_t(const ArcEnds &e, const double (&x)[3], const double (&p)[3]) {
    const float pf[3] = {f32_scaled(p[0], 0), f32_scaled(p[1], 0), f32_scaled(p[2], 0)};
    const double l = (pf[0] * e.p[0] + pf[1] * e.p[1] + pf[2] * e.p[2] >= 0.0f) ? e.inv : -e.inv;
    const float d[3] = {f32_scaled(wide::fma64(-l, x[0], p[0]), 0),
                        f32_scaled(wide::fma64(-l, x[1], p[1]), 0),
                        f32_scaled(wide::fma64(-l, x[2], p[2]), 0)};
    return wide::fma32(d[0], e.m[0], wide::fma32(d[1], e.m[1], d[2] * e.m[2]));
}

// both slots from the unit point p = v / |v| and FP32 copies of the normals
SPHX_HD void arcs_finish(const double (&a1)[3], const double (&a2)[3], const double (&b1)[3],
                         const double (&b2)[3], const float (&na)[3], const float (&nb)[3],
                         const double (&p)[3], PairOut &o) {
    ArcEnds e[4];
    arc_end(a1, na, true, e[0]);
    arc_end(a2, na, false, e[1]);
    arc_end(b1, nb, true, e[2]);
    arc_end(b2, nb, false, e[3]);
    const float t0 = arc_end_t(e[0], a1, p), t1 = arc_end_t(e[1], a2, p);
    const float t2 = arc_end_t(e[2], b1, p), t3 = arc_end_t(e[3], b2, p);
    o.hit[0] = t0 >= 0.0f && t1 >= 0.0f && t2 >= 0.0f && t3 >= 0.0f;
    o.hit[1] = t0 <= 0.0f && t1 <= 0.0f && t2 <= 0.0f && t3 <= 0.0f;
    o.count = (int)o.hit[0] + (int)o.hit[1];
    o.px[0] = p[0];
    o.py[0] = p[1];
    o.px[1] = -p[0];
    o.py[1] = -p[1];
}

// the outputs of an arc pair: the point's z is not fixed, so PairOut's
// (px, py) carry x, y and pz the z of slot 0 (slot 1 is the antipode)
struct ArcOut {
    PairOut o;
    double pz;
};

SPHX_HD bool finite12(const double (&a1)[3], const double (&a2)[3], const double (&b1)[3],
                      const double (&b2)[3]) {
    bool ok = true;  // bitwise &: one test of the twelve exponent fields
#pragma unroll
    for (int i = 0; i < 3; ++i)
        ok = ok & finite_bits(a1[i]) & finite_bits(a2[i]) & finite_bits(b1[i]) & finite_bits(b2[i]);
    return ok;
}

// ---- integer limbs -------------------------------------------------------------
// n_a, n_b exact (106-bit products, 128-bit differences), v = n_a x n_b and
// |v|^2 with 128-bit mantissas, 1 / |v| from the integer-limb square root and
// reciprocal (96 bits), p_i = v_i / |v| rounded to nearest
SPHX_HD void arcs_wide(const double (&a1)[3], const double (&a2)[3], const double (&b1)[3],
                       const double (&b2)[3], ArcOut &r) {
    using namespace wide;
    if (!finite12(a1, a2, b1, b2)) {
        clear(r.o, 0);
        return;
    }
    W<2> A1[3], A2[3], B1[3], B2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        A1[i] = from_double<2>(a1[i]);
        A2[i] = from_double<2>(a2[i]);
        B1[i] = from_double<2>(b1[i]);
        B2[i] = from_double<2>(b2[i]);
    }
    W<4> na[3], nb[3], v[3];
    na[0] = sub<4>(mul_exact(A1[1], A2[2]), mul_exact(A1[2], A2[1]));
    na[1] = sub<4>(mul_exact(A1[2], A2[0]), mul_exact(A1[0], A2[2]));
    na[2] = sub<4>(mul_exact(A1[0], A2[1]), mul_exact(A1[1], A2[0]));
    nb[0] = sub<4>(mul_exact(B1[1], B2[2]), mul_exact(B1[2], B2[1]));
    nb[1] = sub<4>(mul_exact(B1[2], B2[0]), mul_exact(B1[0], B2[2]));
    nb[2] = sub<4>(mul_exact(B1[0], B2[1]), mul_exact(B1[1], B2[0]));
    if ((is_zero(na[0]) && is_zero(na[1]) && is_zero(na[2])) ||
        (is_zero(nb[0]) && is_zero(nb[1]) && is_zero(nb[2]))) {
        clear(r.o, -1);
        return;
    }
    v[0] = sub<4>(mul<4>(na[1], nb[2]), mul<4>(na[2], nb[1]));
    v[1] = sub<4>(mul<4>(na[2], nb[0]), mul<4>(na[0], nb[2]));
    v[2] = sub<4>(mul<4>(na[0], nb[1]), mul<4>(na[1], nb[0]));
    if (is_zero(v[0]) && is_zero(v[1]) && is_zero(v[2])) {
        clear(r.o, -1);
        return;
    }
    const W<4> S = add_same<4>(add_same<4>(sqr<4>(v[0]), sqr<4>(v[1])), sqr<4>(v[2]));
    const W<3> inv = recip_int<3>(sqrt_int<3>(narrow<4, 3>(S)));
    const double p[3] = {to_double<3>(mul<3>(narrow<4, 3>(v[0]), inv)),
                         to_double<3>(mul<3>(narrow<4, 3>(v[1]), inv)),
                         to_double<3>(mul<3>(narrow<4, 3>(v[2]), inv))};
    int ea = na[0].e, eb = nb[0].e;
#pragma unroll
    for (int i = 1; i < 3; ++i) {
        ea = na[i].e > ea ? na[i].e : ea;
        eb = nb[i].e > eb ? nb[i].e : eb;
    }
    const float naf[3] = {f32_rel(na[0], ea), f32_rel(na[1], ea), f32_rel(na[2], ea)};
    const float nbf[3] = {f32_rel(nb[0], eb), f32_rel(nb[1], eb), f32_rel(nb[2], eb)};
    arcs_finish(a1, a2, b1, b2, naf, nbf, p, r.o);
    r.pz = p[2];
}

// ---- FP64 with error-free transformations ---------------------------------------
// n_a, n_b by three renormalised AccuDOPs each (Alg. 4, pairs n + e), each
// v_i = (n_a + e_a) x (n_b + e_b) as one 6-term CompDot (Alg. 2), then the
// plain FP64 normalisation
__device__ __forceinline__ void arcs_eft(const double (&a1)[3], const double (&a2)[3],
                                         const double (&b1)[3], const double (&b2)[3],
                                         ArcOut &r) {
    if (!finite12(a1, a2, b1, b2)) {
        clear(r.o, 0);
        return;
    }
    double na[3], ea[3], nb[3], eb[3];
    accu_dop<double, true>(a1[1], a1[2], a2[1], a2[2], na[0], ea[0]);
    accu_dop<double, true>(a1[2], a1[0], a2[2], a2[0], na[1], ea[1]);
    accu_dop<double, true>(a1[0], a1[1], a2[0], a2[1], na[2], ea[2]);
    accu_dop<double, true>(b1[1], b1[2], b2[1], b2[2], nb[0], eb[0]);
    accu_dop<double, true>(b1[2], b1[0], b2[2], b2[0], nb[1], eb[1]);
    accu_dop<double, true>(b1[0], b1[1], b2[0], b2[1], nb[2], eb[2]);
    if ((eq_zero(na[0]) && eq_zero(na[1]) && eq_zero(na[2])) ||
        (eq_zero(nb[0]) && eq_zero(nb[1]) && eq_zero(nb[2]))) {
        clear(r.o, -1);
        return;
    }
    double v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        const double xs[6] = {na[j], na[j], ea[j], -na[k], -na[k], -ea[k]};
        const double ys[6] = {nb[k], eb[k], nb[k], nb[j], eb[j], nb[j]};
        v[i] = comp_dot<double, 6>(xs, ys);
    }
    if (eq_zero(v[0]) && eq_zero(v[1]) && eq_zero(v[2])) {
        clear(r.o, -1);
        return;
    }
    const double nrm = sqrt_(fma_(v[0], v[0], fma_(v[1], v[1], mul(v[2], v[2]))));
    const double p[3] = {div_(v[0], nrm), div_(v[1], nrm), div_(v[2], nrm)};
    const float naf[3] = {(float)na[0], (float)na[1], (float)na[2]};
    const float nbf[3] = {(float)nb[0], (float)nb[1], (float)nb[2]};
    float sa = fmaxf(fabsf(naf[0]), fmaxf(fabsf(naf[1]), fabsf(naf[2])));
    float sb = fmaxf(fabsf(nbf[0]), fmaxf(fabsf(nbf[1]), fabsf(nbf[2])));
    const float naf2[3] = {naf[0] / sa, naf[1] / sa, naf[2] / sa};
    const float nbf2[3] = {nbf[0] / sb, nbf[1] / sb, nbf[2] / sb};
    arcs_finish(a1, a2, b1, b2, naf2, nbf2, p, r.o);
    r.pz = p[2];
}

// ---- direct FP64 -------------------------------------------------------------------
__device__ __forceinline__ void arcs_direct(const double (&a1)[3], const double (&a2)[3],
                                            const double (&b1)[3], const double (&b2)[3],
                                            ArcOut &r) {
    if (!finite12(a1, a2, b1, b2)) {
        clear(r.o, 0);
        return;
    }
    const double na[3] = {sub(mul(a1[1], a2[2]), mul(a1[2], a2[1])),
                          sub(mul(a1[2], a2[0]), mul(a1[0], a2[2])),
                          sub(mul(a1[0], a2[1]), mul(a1[1], a2[0]))};
    const double nb[3] = {sub(mul(b1[1], b2[2]), mul(b1[2], b2[1])),
                          sub(mul(b1[2], b2[0]), mul(b1[0], b2[2])),
                          sub(mul(b1[0], b2[1]), mul(b1[1], b2[0]))};
    if ((eq_zero(na[0]) && eq_zero(na[1]) && eq_zero(na[2])) ||
        (eq_zero(nb[0]) && eq_zero(nb[1]) && eq_zero(nb[2]))) {
        clear(r.o, -1);
        return;
    }
    const double v[3] = {sub(mul(na[1], nb[2]), mul(na[2], nb[1])),
                         sub(mul(na[2], nb[0]), mul(na[0], nb[2])),
                         sub(mul(na[0], nb[1]), mul(na[1], nb[0]))};
    if (eq_zero(v[0]) && eq_zero(v[1]) && eq_zero(v[2])) {
        clear(r.o, -1);
        return;
    }
    const double nrm = sqrt_(add(add(mul(v[0], v[0]), mul(v[1], v[1])), mul(v[2], v[2])));
    const double p[3] = {div_(v[0], nrm), div_(v[1], nrm), div_(v[2], nrm)};
    // plain on-arc test: t = p . m in FP64, m = n x x1 or x2 x n
    const double *xs[4] = {a1, a2, b1, b2};
    double t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double *n = k < 2 ? na : nb;
        const double *x = xs[k];
        const bool first = (k & 1) == 0;
        const double *u = first ? n : x;
        const double *w = first ? x : n;
        const double m0 = sub(mul(u[1], w[2]), mul(u[2], w[1]));
        const double m1 = sub(mul(u[2], w[0]), mul(u[0], w[2]));
        const double m2 = sub(mul(u[0], w[1]), mul(u[1], w[0]));
        t[k] = add(add(mul(p[0], m0), mul(p[1], m1)), mul(p[2], m2));
    }
    r.o.hit[0] = ge_zero(t[0]) && ge_zero(t[1]) && ge_zero(t[2]) && ge_zero(t[3]);
    r.o.hit[1] = le_zero(t[0]) && le_zero(t[1]) && le_zero(t[2]) && le_zero(t[3]);
    r.o.count = (int)r.o.hit[0] + (int)r.o.hit[1];
    r.o.px[0] = p[0];
    r.o.py[0] = p[1];
    r.o.px[1] = -p[0];
    r.o.py[1] = -p[1];
    r.pz = p[2];
}

template <int Mode>
__device__ __forceinline__ void intersect_arcs(const double (&a1)[3], const double (&a2)[3],
                                               const double (&b1)[3], const double (&b2)[3],
                                               ArcOut &r) {
    if (Mode == kWideInt)
        arcs_wide(a1, a2, b1, b2, r);
    else if (Mode == kEftFp64)
        arcs_eft(a1, a2, b1, b2, r);
    else
        arcs_direct(a1, a2, b1, b2, r);
}

}  // namespace sphx
