// The adaptive variant (the filter of Sec. 9): Eq. 2.2 evaluated in plain FP64
// together with a running forward error bound, accepted only where the bound
// proves the result good, and otherwise re-evaluated by the integer-limb form
// (correctly rounded). The paper names the idea (a cheap evaluation first,
// the accurate one only where an error estimate says it is needed) without
// fixing the estimate; this one is a rigorous first-principles bound.
//
// Bound model: every FP64 operation returns the exact result times (1 + d),
// |d| <= u = 2^-53, plus an absolute term below 2^-1074 where a product may
// underflow. Inputs are exact. Each quantity q~ carries e_q >= |q~ - q|, with
// q the exact real value of the same expression on the exact inputs:
//   n = x1 x x2, one FMA per component:  e_n = u (|p| + |n~|), p the rounded product
//   S2 = n_x^2 + n_y^2, S3 = S2 + n_z^2:  rounding + e_n (2 |n~| + e_n) per square
//   Q = S2 - S3 z0^2 (one FMA):           e_Q = u |Q~| + e_S2 + S3~ e_c + e_S3 (c + e_c)
//   s = sqrt(Q):                          e_s = u s~ + e_Q / s~      (|sqrt a - sqrt b| <= |a - b| / sqrt a)
//   X = z0 n_z n_x +- s n_y (FMA):        e_X = u |X~| + e_{z0 n_z n_x} + e_s |n_y~| + (s~ + e_s) e_{n_y}
//   P_x = -X / S2:                        e_P = u |P~| + (e_X + |P~| e_S2) / (S2~ - e_S2)
// and the on-arc values t1 = P . (n x x1), t2 = P . (x2 x n) likewise. The
// bounds are computed in FP64 themselves; their own relative rounding error
// (a few hundred u at most along the chain) is covered by one factor
// 1 + 2^-40 applied wherever a bound is compared.
//
// A lane is accepted when the bound decides everything the output depends on:
//   * the sign of Q (|Q~| > e_Q): no candidate when Q < 0; tangency and
//     near-tangency (|Q~| <= e_Q) go to the accurate form;
//   * n_xy != 0 (S2~ > e_S2), which also rules out n = 0;
//   * for each candidate, the signs of t1 and t2 (a certain negative one
//     rejects it; otherwise both must be certainly positive);
//   * for each hit, both point components within the gate of G ulp (G = 4
//     in the mode's contract, a caller's choice >= 1 in the extended call):
//     G ulp of the correctly rounded exact value where
//     |P_c| >= 2^-20 sqrt(1 - z0^2), else G u sqrt(1 - z0^2) absolute.
// Inputs whose magnitudes leave [2^-100, 2^100] (zeros aside) are not
// filtered, which keeps every intermediate far from overflow and from
// gradual underflow (except in the last products, whose absolute error the
// 2^-1074 terms cover).
#pragma once
#include "intersect.cuh"

namespace sphx {
namespace filt {

constexpr double kU = 1.1102230246251565e-16;  // 2^-53
constexpr double kEta = 4.9406564584124654e-324;  // 2^-1074
constexpr double kSafe = 1.0 + 9.094947017729282e-13;  // 1 + 2^-40

// ulp of a positive double: 2^(exponent - 52), never below 2^-1074
EFT_HD double ulp_pos(double x) {
    const uint64_t e = (wide::bits_of(x) >> 52) & 0x7ff;
    return e > 52 ? wide::double_of((e - 52) << 52) : kEta;
}

// the accepted range of input magnitudes
EFT_HD bool in_range(double v) {
    const double a = fabs(v);
    return a == 0.0 || (a >= 7.888609052210118e-31 && a <= 1.2676506002282294e30);  // 2^-100, 2^100
}

// Is a component p~ with error bound B (already inflated) within a gate of G
// ulp (G = 4: the mode's contract)? Large exact values are gated on G ulp of
// their rounding, which is at least G ulp of any double below the exact
// value; small ones on G u rho. rho~ has a relative error below 3u, so
// 0.975 G u rho~ < G u rho, and the class boundary 2^-20 rho is tested with a
// 2^-40 margin on either side. gate = 0.975 G.
EFT_HD bool within_gate(double p, double B, double rho, double gate) {
    const double a = fabs(p);
    const double thr = 9.5367431640625e-07 * rho;  // 2^-20 rho
    const double lo = (a - B) * (1.0 - 8.881784197001252e-16);  // below a - B (1 - 2^-50)
    const bool surely_large = lo >= thr * kSafe;
    const bool surely_small = (a + B) * (1.0 + 8.881784197001252e-16) < thr * (2.0 - kSafe);
    const bool ok_large = lo > 0.0 && B <= gate * ulp_pos(lo);
    const bool ok_small = B <= gate * kU * rho;
    return (surely_small || ok_large) && (surely_large || ok_small);
}

// One arc against one latitude. Returns true with o filled (the same
// conventions as the other modes) when the bound vouches for the result
// within gate / 0.975 ulp per component, false when the lane must be
// re-evaluated.
EFT_HD bool pair_filtered(const double (&x1)[3], const double (&x2)[3],
                                              double z0, double gate, PairOut &o) {
    if (!(in_range(x1[0]) && in_range(x1[1]) && in_range(x1[2]) && in_range(x2[0]) &&
          in_range(x2[1]) && in_range(x2[2]) && in_range(z0)))
        return false;  // also every non-finite input
    const double a0 = x1[0], a1 = x1[1], a2 = x1[2];
    const double b0 = x2[0], b1 = x2[1], b2 = x2[2];

    // n = x1 x x2
    const double qx = mul(a2, b1), qy = mul(a0, b2), qz = mul(a1, b0);
    const double nx = fma_(a1, b2, -qx), ny = fma_(a2, b0, -qy), nz = fma_(a0, b1, -qz);
    const double ex = kU * (fabs(qx) + fabs(nx));
    const double ey = kU * (fabs(qy) + fabs(ny));
    const double ez = kU * (fabs(qz) + fabs(nz));

    // |n_xy|^2, |n|^2 and Q = S2 - S3 z0^2
    const double yy = mul(ny, ny);
    const double S2 = fma_(nx, nx, yy);
    const double eS2 = kU * (yy + S2) + ex * (2.0 * fabs(nx) + ex) + ey * (2.0 * fabs(ny) + ey);
    if (!(S2 > eS2 * kSafe)) return false;  // n_xy may vanish (n = 0 included)
    const double S3 = fma_(nz, nz, S2);
    const double eS3 = kU * S3 + eS2 + ez * (2.0 * fabs(nz) + ez);
    const double c = mul(z0, z0);
    const double ec = kU * c + kEta;
    const double Q = fma_(-S3, c, S2);
    const double eQ = (kU * fabs(Q) + eS2 + S3 * ec + eS3 * (c + ec)) * kSafe;
    if (Q < -eQ) {  // certainly no candidate
        clear(o, 0);
        return true;
    }
    if (!(Q > eQ)) return false;  // tangency not decided

    const double s = sqrt_(Q);
    const double es = kU * s + eQ / s;

    // numerators of both roots: X = z0 n_z n_x +- s n_y, Y = z0 n_z n_y -+ s n_x
    const double g = mul(z0, nz);
    const double eg = fabs(z0) * ez + kU * fabs(g) + kEta;
    const double ax = mul(g, nx), ay = mul(g, ny);
    const double eax = kU * fabs(ax) + kEta + eg * fabs(nx) + (fabs(g) + eg) * ex;
    const double eay = kU * fabs(ay) + kEta + eg * fabs(ny) + (fabs(g) + eg) * ey;
    const double e_sny = es * fabs(ny) + (s + es) * ey;
    const double e_snx = es * fabs(nx) + (s + es) * ex;

    // on-arc directions m1 = n x x1, m2 = x2 x n (t1 = P . m1, t2 = P . m2)
    const double r1x = mul(nz, a1), r1y = mul(nx, a2), r1z = mul(ny, a0);
    const double m1x = fma_(ny, a2, -r1x), m1y = fma_(nz, a0, -r1y), m1z = fma_(nx, a1, -r1z);
    const double r2x = mul(b2, ny), r2y = mul(b0, nz), r2z = mul(b1, nx);
    const double m2x = fma_(b1, nz, -r2x), m2y = fma_(b2, nx, -r2y), m2z = fma_(b0, ny, -r2z);
    const double em1x = kU * (fabs(r1x) + fabs(m1x)) + 2.0 * kEta + ey * fabs(a2) + ez * fabs(a1);
    const double em1y = kU * (fabs(r1y) + fabs(m1y)) + 2.0 * kEta + ez * fabs(a0) + ex * fabs(a2);
    const double em1z = kU * (fabs(r1z) + fabs(m1z)) + 2.0 * kEta + ex * fabs(a1) + ey * fabs(a0);
    const double em2x = kU * (fabs(r2x) + fabs(m2x)) + 2.0 * kEta + ez * fabs(b1) + ey * fabs(b2);
    const double em2y = kU * (fabs(r2y) + fabs(m2y)) + 2.0 * kEta + ex * fabs(b2) + ez * fabs(b0);
    const double em2z = kU * (fabs(r2z) + fabs(m2z)) + 2.0 * kEta + ey * fabs(b0) + ex * fabs(b1);

    const double rho = sqrt_(mul(1.0 - z0, 1.0 + z0));
    const double S2lo = S2 - eS2 * kSafe;
    o.count = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        o.hit[r] = false;
        const double sg = r == 0 ? 1.0 : -1.0;
        const double X = fma_(sg * s, ny, ax);
        const double Y = fma_(-sg * s, nx, ay);
        const double eX = kU * fabs(X) + kEta + eax + e_sny;
        const double eY = kU * fabs(Y) + kEta + eay + e_snx;
        const double Px = -div_(X, S2), Py = -div_(Y, S2);
        const double ePx = kU * fabs(Px) + kEta + (eX + fabs(Px) * eS2) / S2lo;
        const double ePy = kU * fabs(Py) + kEta + (eY + fabs(Py) * eS2) / S2lo;
        // t1 = z0 m1z + Py m1y + Px m1x by two FMAs after one product
        const double u1 = mul(z0, m1z), v1 = fma_(Py, m1y, u1), t1 = fma_(Px, m1x, v1);
        const double u2 = mul(z0, m2z), v2 = fma_(Py, m2y, u2), t2 = fma_(Px, m2x, v2);
        const double e1 = (kU * (fabs(u1) + fabs(v1) + fabs(t1)) + 3.0 * kEta +
                           ePx * fabs(m1x) + (fabs(Px) + ePx) * em1x +
                           ePy * fabs(m1y) + (fabs(Py) + ePy) * em1y + fabs(z0) * em1z) * kSafe;
        const double e2 = (kU * (fabs(u2) + fabs(v2) + fabs(t2)) + 3.0 * kEta +
                           ePx * fabs(m2x) + (fabs(Px) + ePx) * em2x +
                           ePy * fabs(m2y) + (fabs(Py) + ePy) * em2y + fabs(z0) * em2z) * kSafe;
        if (t1 < -e1 || t2 < -e2) continue;        // certainly off the arc
        if (!(t1 > e1 && t2 > e2)) return false;   // near an endpoint
        if (!(within_gate(Px, ePx * kSafe, rho, gate) && within_gate(Py, ePy * kSafe, rho, gate)))
            return false;
        o.hit[r] = true;
        o.px[r] = Px;
        o.py[r] = Py;
        ++o.count;
    }
    return true;
}

}  // namespace filt
}  // namespace sphx
