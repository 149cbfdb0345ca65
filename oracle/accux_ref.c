/*
 * Step-by-step FP64 reference of the paper's algorithms: TEST INFRASTRUCTURE.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may load it.
 * It shares no code with the CUDA library.
 *
 * Every operation is one IEEE-754 binary64 operation rounded to nearest even:
 * '+', '-', '*', '/', sqrt() and the C99 fma() are all correctly rounded, and
 * the file is compiled with -ffp-contract=off so the compiler fuses nothing
 * (as the paper's own build did, Sec. 7.2). fl(a*b - c) in the paper's
 * notation (Sec. 3) is written fma(a, b, -c).
 *
 * Readings of the paper (where it is silent, garbled or inconsistent):
 *  R1 AccuDOP (Algorithm 4) returns err = fl(s + fl(r1 - r2)): with
 *     [p1,r1] = a*d and [p2,r2] = b*c exactly, ad - bc = (p1 - p2) + (r1 - r2).
 *     The printed '+' is kept behind variant bit SPHX_ORACLE_LITERAL_DOP so a
 *     test can show it breaks the bound of Sec. 5.2.
 *  R2 Algorithm 8 lists AccuDOP arguments in an order that only yields the
 *     normal if the routine is read as first-pair minus second-pair; we compute
 *     the standard n = x1 x x2 (Sec. 1.2): nx = y1 z2 - z1 y2, etc.
 *  R3 AccSqrt is not printed (Sec. 6 cites Rump 2023 and a Taylor expansion):
 *     sbar = fl(sqrt(S)); r = fl(S - sbar*sbar) by one FMA (exact for a
 *     correctly rounded square root); e_s = fl(fl(r + e) / fl(2 sbar)).
 *     S == 0 gives (0, 0).
 *  R4 The second root flips the sign of s in Eq. 2.2 (slot 1); the CompDot
 *     of Algorithm 8 then takes -sbar, -e_s in place of sbar, e_s.
 *  R5 Containment (Sec. 2 asks only that the point lie between the
 *     endpoints): with the computed point P and m1 = n x x1, m2 = x2 x n, a
 *     candidate is a hit iff P.m1 >= 0 and P.m2 >= 0 (equal to
 *     (x1 x P).n >= 0, (P x x2).n >= 0).
 *     The EFT path forms m1, m2 from the leading parts nbar with FMAs; the
 *     direct path uses its plainly computed n without FMAs.
 *  R6 Existence (Sec. 2): candidates exist iff the computed s^2 >= 0; s^2 == 0
 *     is one tangent point (slot 0).
 *  R7 Degenerate: computed S3 == 0 -> count -1; S2 == 0 -> count -1 if
 *     z0 == 0 else 0; any non-finite input -> count 0. Unused slots are NaN.
 *  R8 SumOfSquaresC (Algorithm 7) drops the e_i^2 terms, which is harmless
 *     only while |e_i| <= u |nbar_i|. AccuDOP's pair is not normalised: when
 *     |n_i| is far below |ad| + |bc| (short or near-antipodal arcs) its err is
 *     up to u (|ad| + |bc|), and the dropped e_i^2 costs relative accuracy
 *     (e_i/n_i)^2 in S2 and S3 -- the absolute u^2 terms of the bounds in the
 *     supplement (S2). Variant bit SPHX_ORACLE_RENORM_DOP renormalises each
 *     AccuDOP output with one TwoSum (exact, so n is unchanged), which restores
 *     |e_i| <= u |nbar_i|. Variant 0 is Algorithm 8 as printed.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define SPHX_ORACLE_LITERAL_DOP 1
#define SPHX_ORACLE_RENORM_DOP 2

/* ---- error-free transformations (Sec. 5) -------------------------------- */

/* TwoSum (Knuth): s = fl(a+b), a + b = s + e exactly. */
static void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    double br = b - bv;
    double ar = a - av;
    *s = x;
    *e = ar + br;
}

/* FastTwoSum (Dekker): exact when the exponent of a is >= that of b. */
static void fast_two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double z = x - a;
    *s = x;
    *e = b - z;
}

/* TwoProd with FMA: p = fl(a*b), e = a*b - p exactly. */
static void two_prod(double a, double b, double *p, double *e) {
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

/* Algorithm 1, CompDotC: dot product as an unevaluated pair (p, s). */
static void comp_dot_c(const double *x, const double *y, int n, double *p_out, double *s_out) {
    double p, s, h, r, q;
    two_prod(x[0], y[0], &p, &s);
    for (int i = 1; i < n; ++i) {
        two_prod(x[i], y[i], &h, &r);
        two_sum(p, h, &p, &q);
        s = s + (q + r);
    }
    *p_out = p;
    *s_out = s;
}

/* Algorithm 2, CompDot: fl(p + s) of CompDotC. */
static double comp_dot(const double *x, const double *y, int n) {
    double p, s;
    comp_dot_c(x, y, n, &p, &s);
    return p + s;
}

/* Algorithm 4, AccuDOP: a*d - b*c as the pair (dop, err); reading R1. */
static void accu_dop(double a, double b, double c, double d, int variant,
                     double *dop, double *err) {
    double p1, r1, p2, r2, s;
    two_prod(a, d, &p1, &r1);
    two_prod(b, c, &p2, &r2);
    two_sum(p1, -p2, dop, &s);
    if (variant & SPHX_ORACLE_LITERAL_DOP)
        *err = s + (r1 + r2);
    else
        *err = s + (r1 - r2);
    if (variant & SPHX_ORACLE_RENORM_DOP) /* reading R8 */
        two_sum(*dop, *err, dop, err);
}

/* Algorithm 6, SumNonNeg: [A,a] + [B,b] for non-negative pairs. */
static void sum_non_neg(double A, double a, double B, double b, double *S, double *s) {
    double H, h, c, d;
    two_sum(A, B, &H, &h);
    c = a + b;
    d = h + c;
    fast_two_sum(H, d, S, s);
}

/* Algorithm 5, SumOfSquares: squared norm as a pair, starting from (0, 0). */
static void sum_of_squares(const double *x, int n, double *S, double *s) {
    double Sa = 0.0, sa = 0.0, P, p;
    for (int j = 0; j < n; ++j) {
        two_prod(x[j], x[j], &P, &p);
        sum_non_neg(Sa, sa, P, p, &Sa, &sa);
    }
    *S = Sa;
    *s = sa;
}

/* Algorithm 7, SumOfSquaresC: squared norm of the compensated vector x + e. */
static void sum_of_squares_c(const double *x, const double *e, int n, double *S, double *s) {
    double Ss, ss, Rs, R;
    sum_of_squares(x, n, &Ss, &ss);
    Rs = comp_dot(x, e, n);
    R = fma(2.0, Rs, ss);
    fast_two_sum(Ss, R, S, s);
}

/* AccSqrt, reading R3: sqrt of the pair (S, e) as a pair. */
static void acc_sqrt(double S, double e, double *r_out, double *er_out) {
    if (S == 0.0) {
        *r_out = 0.0;
        *er_out = 0.0;
        return;
    }
    double r = sqrt(S);
    double rem = fma(-r, r, S);
    *r_out = r;
    *er_out = (rem + e) / (2.0 * r);
}

/* ---- Algorithm 8 (AccuX), both roots, with intermediates ----------------- */

typedef struct {
    double n[3], en[3];
    double S2, s2, S3, s3;
    double ss2, ess2; /* [s^2 bar, e] after FastTwoSum */
    double sb, es;    /* AccSqrt */
    double X;         /* root 0's x-coordinate numerator (CompDot), P_x = -X / S2 */
} accux_mid;

static int all_finite(const double *a, const double *b, double z0) {
    return isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]) && isfinite(b[0]) &&
           isfinite(b[1]) && isfinite(b[2]) && isfinite(z0);
}

static void set_nan(double *pts) {
    for (int k = 0; k < 6; ++k) pts[k] = NAN;
}

/* one coordinate numerator, Algorithm 8 lines for x (ysign=+1) or y (-1) */
static double accux_numerator(double F, double eF, double nb, double enb, double z0, double sb,
                              double es) {
    double xs[6] = {F, eF, nb, enb, nb, enb};
    double ys[6] = {z0, z0, sb, sb, es, es};
    return comp_dot(xs, ys, 6);
}

static void accux_one(const double *x1, const double *x2, double z0, int variant, double *pts,
                      int *count, accux_mid *mid) {
    set_nan(pts);
    if (!all_finite(x1, x2, z0)) {
        *count = 0;
        return;
    }
    accux_mid m;
    /* normal n = x1 x x2 by three AccuDOPs (reading R2) */
    accu_dop(x1[1], x1[2], x2[1], x2[2], variant, &m.n[0], &m.en[0]); /* y1 z2 - z1 y2 */
    accu_dop(x1[2], x1[0], x2[2], x2[0], variant, &m.n[1], &m.en[1]); /* z1 x2 - x1 z2 */
    accu_dop(x1[0], x1[1], x2[0], x2[1], variant, &m.n[2], &m.en[2]); /* x1 y2 - y1 x2 */
    sum_of_squares_c(m.n, m.en, 2, &m.S2, &m.s2);
    sum_of_squares_c(m.n, m.en, 3, &m.S3, &m.s3);
    double C, eC, D, eD, E, eE, e;
    two_prod(z0, z0, &C, &eC);
    {
        double xs[4] = {m.S3, m.S3, m.s3, m.s3};
        double ys[4] = {C, eC, C, eC};
        comp_dot_c(xs, ys, 4, &D, &eD);
    }
    two_sum(m.S2, -D, &E, &eE);
    e = (m.s2 - eD) + eE;
    fast_two_sum(E, e, &m.ss2, &m.ess2);
    m.sb = 0.0;
    m.es = 0.0;
    m.X = 0.0;
    if (m.ss2 >= 0.0) acc_sqrt(m.ss2, m.ess2, &m.sb, &m.es);
    if (mid) *mid = m;

    if (m.S3 == 0.0) { /* R7 */
        *count = -1;
        return;
    }
    if (m.S2 == 0.0) {
        *count = (z0 == 0.0) ? -1 : 0;
        return;
    }
    if (!(m.ss2 >= 0.0)) {
        *count = 0;
        return;
    }
    /* F_x, F_y with their compensation terms (shared by both roots) */
    double Fx, eFx1, Fy, eFy1;
    two_prod(m.n[0], m.n[2], &Fx, &eFx1);
    double eFx2 = m.n[0] * m.en[2];
    double eFx3 = m.n[2] * m.en[0];
    double eFx = (eFx1 + eFx2) + eFx3;
    two_prod(m.n[1], m.n[2], &Fy, &eFy1);
    double eFy2 = m.n[1] * m.en[2];
    double eFy3 = m.n[2] * m.en[1];
    double eFy = (eFy1 + eFy2) + eFy3;

    /* containment vectors from the leading parts (reading R5) */
    double m1[3], m2[3];
    m1[0] = fma(m.n[1], x1[2], -(m.n[2] * x1[1]));
    m1[1] = fma(m.n[2], x1[0], -(m.n[0] * x1[2]));
    m1[2] = fma(m.n[0], x1[1], -(m.n[1] * x1[0]));
    m2[0] = fma(x2[1], m.n[2], -(x2[2] * m.n[1]));
    m2[1] = fma(x2[2], m.n[0], -(x2[0] * m.n[2]));
    m2[2] = fma(x2[0], m.n[1], -(x2[1] * m.n[0]));

    int nroots = (m.ss2 > 0.0) ? 2 : 1;
    int c = 0;
    for (int slot = 0; slot < nroots; ++slot) {
        double sg = slot == 0 ? 1.0 : -1.0;
        double xnum = accux_numerator(Fx, eFx, m.n[1], m.en[1], z0, sg * m.sb, sg * m.es);
        if (mid && slot == 0) mid->X = xnum;
        double ynum = accux_numerator(Fy, eFy, -m.n[0], -m.en[0], z0, sg * m.sb, sg * m.es);
        double Px = -(xnum / m.S2);
        double Py = -(ynum / m.S2);
        double t1 = fma(Px, m1[0], fma(Py, m1[1], z0 * m1[2]));
        double t2 = fma(Px, m2[0], fma(Py, m2[1], z0 * m2[2]));
        if (t1 >= 0.0 && t2 >= 0.0) {
            pts[3 * slot + 0] = Px;
            pts[3 * slot + 1] = Py;
            pts[3 * slot + 2] = z0;
            ++c;
        }
    }
    *count = c;
}

/* ---- direct FP64 evaluation of Eq. 2.2 (Sec. 4), no FMA anywhere ---------- */

static void direct_one(const double *x1, const double *x2, double z0, double *pts, int *count) {
    set_nan(pts);
    if (!all_finite(x1, x2, z0)) {
        *count = 0;
        return;
    }
    double nx = x1[1] * x2[2] - x1[2] * x2[1];
    double ny = x1[2] * x2[0] - x1[0] * x2[2];
    double nz = x1[0] * x2[1] - x1[1] * x2[0];
    double S2 = nx * nx + ny * ny;
    double S3 = S2 + nz * nz;
    if (S3 == 0.0) {
        *count = -1;
        return;
    }
    if (S2 == 0.0) {
        *count = (z0 == 0.0) ? -1 : 0;
        return;
    }
    double zz = z0 * z0;
    double s2 = S2 - S3 * zz;
    if (!(s2 >= 0.0)) {
        *count = 0;
        return;
    }
    double s = sqrt(s2);
    double a = (z0 * nx) * nz;
    double b = (z0 * ny) * nz;
    double sny = s * ny;
    double snx = s * nx;
    double m1[3], m2[3];
    m1[0] = ny * x1[2] - nz * x1[1];
    m1[1] = nz * x1[0] - nx * x1[2];
    m1[2] = nx * x1[1] - ny * x1[0];
    m2[0] = x2[1] * nz - x2[2] * ny;
    m2[1] = x2[2] * nx - x2[0] * nz;
    m2[2] = x2[0] * ny - x2[1] * nx;
    int nroots = (s2 > 0.0) ? 2 : 1;
    int c = 0;
    for (int slot = 0; slot < nroots; ++slot) {
        double Px, Py;
        if (slot == 0) {
            Px = -((a + sny) / S2);
            Py = -((b - snx) / S2);
        } else {
            Px = -((a - sny) / S2);
            Py = -((b + snx) / S2);
        }
        double t1 = (Px * m1[0] + Py * m1[1]) + z0 * m1[2];
        double t2 = (Px * m2[0] + Py * m2[1]) + z0 * m2[2];
        if (t1 >= 0.0 && t2 >= 0.0) {
            pts[3 * slot + 0] = Px;
            pts[3 * slot + 1] = Py;
            pts[3 * slot + 2] = z0;
            ++c;
        }
    }
    *count = c;
}

/* ---- exported entry points (ctypes) -------------------------------------- */

void oracle_accux(const double *A, const double *B, const double *z0, int64_t n, int variant,
                  double *pts, int32_t *count) {
    for (int64_t i = 0; i < n; ++i) {
        int c;
        accux_one(A + 3 * i, B + 3 * i, z0[i], variant, pts + 6 * i, &c, NULL);
        count[i] = c;
    }
}

void oracle_direct(const double *A, const double *B, const double *z0, int64_t n, double *pts,
                   int32_t *count) {
    for (int64_t i = 0; i < n; ++i) {
        int c;
        direct_one(A + 3 * i, B + 3 * i, z0[i], pts + 6 * i, &c);
        count[i] = c;
    }
}

/* intermediates of Algorithm 8 (App. A): 16 doubles per arc in the order
   n[3], en[3], S2, s2, S3, s3, ss2, ess2, sb, es, X, pad (X: root 0's
   x-coordinate numerator, 0 when the arc has no candidate) */
void oracle_accux_intermediates(const double *A, const double *B, const double *z0, int64_t n,
                                int variant, double *mid) {
    for (int64_t i = 0; i < n; ++i) {
        double pts[6];
        int c;
        accux_mid m;
        accux_one(A + 3 * i, B + 3 * i, z0[i], variant, pts, &c, &m);
        double *o = mid + 16 * i;
        for (int k = 0; k < 3; ++k) {
            o[k] = m.n[k];
            o[3 + k] = m.en[k];
        }
        o[6] = m.S2; o[7] = m.s2; o[8] = m.S3; o[9] = m.s3;
        o[10] = m.ss2; o[11] = m.ess2; o[12] = m.sb; o[13] = m.es;
        o[14] = m.X; o[15] = 0.0;
    }
}

/* building blocks, one call per element, for the per-algorithm pins */
void oracle_two_prod(const double *a, const double *b, int64_t n, double *p, double *e) {
    for (int64_t i = 0; i < n; ++i) two_prod(a[i], b[i], p + i, e + i);
}
void oracle_two_sum(const double *a, const double *b, int64_t n, double *s, double *e) {
    for (int64_t i = 0; i < n; ++i) two_sum(a[i], b[i], s + i, e + i);
}
void oracle_accu_dop(const double *abcd, int64_t n, int variant, double *dop, double *err) {
    for (int64_t i = 0; i < n; ++i)
        accu_dop(abcd[4 * i], abcd[4 * i + 1], abcd[4 * i + 2], abcd[4 * i + 3], variant, dop + i,
                 err + i);
}
void oracle_comp_dot_c(const double *x, const double *y, int64_t n, int len, double *p,
                       double *s) {
    for (int64_t i = 0; i < n; ++i) comp_dot_c(x + len * i, y + len * i, len, p + i, s + i);
}
void oracle_sum_non_neg(const double *AaBb, int64_t n, double *S, double *s) {
    for (int64_t i = 0; i < n; ++i)
        sum_non_neg(AaBb[4 * i], AaBb[4 * i + 1], AaBb[4 * i + 2], AaBb[4 * i + 3], S + i, s + i);
}
void oracle_sum_of_squares_c(const double *x, const double *e, int64_t n, int len, double *S,
                             double *s) {
    for (int64_t i = 0; i < n; ++i) sum_of_squares_c(x + len * i, e + len * i, len, S + i, s + i);
}
void oracle_acc_sqrt(const double *S, const double *e, int64_t n, double *r, double *er) {
    for (int64_t i = 0; i < n; ++i) acc_sqrt(S[i], e[i], r + i, er + i);
}
