// Error-free transformations and compensated operators (Sec. 5 of Chen,
// Ullrich, Panetta, arXiv 2510.09892), for FP64 and FP32.
//
// Every step is one correctly rounded IEEE operation written with an explicit
// rounding intrinsic on the device (__dadd_rn, __dmul_rn, __fma_rn, ...), so
// nvcc can never contract a product and a sum into an FMA and change a
// rounding: the same discipline the paper gets from -ffp-contract=off
// (Sec. 7.2). The functions also build for the host (plain IEEE operations,
// fma and sqrt, all correctly rounded; the host build of a caller must not
// contract), so the kernels' source can be checked on the CPU.
#pragma once
#include <math.h>

#if defined(__CUDACC__)
#define EFT_HD __host__ __device__ __forceinline__
#else
#define EFT_HD inline
#endif

namespace sphx {

// ---- rounding-explicit scalar operations ------------------------------------
#if defined(__CUDA_ARCH__)
EFT_HD double add(double a, double b) { return __dadd_rn(a, b); }
EFT_HD double sub(double a, double b) { return __dsub_rn(a, b); }
EFT_HD double mul(double a, double b) { return __dmul_rn(a, b); }
EFT_HD double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
EFT_HD double div_(double a, double b) { return __ddiv_rn(a, b); }
EFT_HD double sqrt_(double a) { return __dsqrt_rn(a); }

EFT_HD float add(float a, float b) { return __fadd_rn(a, b); }
EFT_HD float sub(float a, float b) { return __fsub_rn(a, b); }
EFT_HD float mul(float a, float b) { return __fmul_rn(a, b); }
EFT_HD float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
EFT_HD float div_(float a, float b) { return __fdiv_rn(a, b); }
EFT_HD float sqrt_(float a) { return __fsqrt_rn(a); }
#else
EFT_HD double add(double a, double b) { return a + b; }
EFT_HD double sub(double a, double b) { return a - b; }
EFT_HD double mul(double a, double b) { return a * b; }
EFT_HD double fma_(double a, double b, double c) { return ::fma(a, b, c); }
EFT_HD double div_(double a, double b) { return a / b; }
EFT_HD double sqrt_(double a) { return ::sqrt(a); }

EFT_HD float add(float a, float b) { return a + b; }
EFT_HD float sub(float a, float b) { return a - b; }
EFT_HD float mul(float a, float b) { return a * b; }
EFT_HD float fma_(float a, float b, float c) { return ::fmaf(a, b, c); }
EFT_HD float div_(float a, float b) { return a / b; }
EFT_HD float sqrt_(float a) { return ::sqrtf(a); }
#endif

template <typename T>
struct Pair {  // unevaluated sum hi + lo
    T hi, lo;
};

// FastTwoSum (Dekker): exact when exponent(a) >= exponent(b).
template <typename T>
EFT_HD void fast_two_sum(T a, T b, T &s, T &e) {
    T x = add(a, b);
    T z = sub(x, a);
    s = x;
    e = sub(b, z);
}

// TwoSum (Knuth): s = fl(a + b) and a + b = s + e exactly; no precondition.
template <typename T>
EFT_HD void two_sum(T a, T b, T &s, T &e) {
    T x = add(a, b);
    T bv = sub(x, a);
    T av = sub(x, bv);
    T br = sub(b, bv);
    T ar = sub(a, av);
    s = x;
    e = add(ar, br);
}

// The bits of a double (on the integer pipe)
EFT_HD unsigned long long eft_bits(double x) {
#if defined(__CUDA_ARCH__)
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    __builtin_memcpy(&b, &x, sizeof b);
    return b;
#endif
}

// TwoSum of doubles in three FP64 operations instead of six: the operands
// ordered by magnitude on the integer pipe, then FastTwoSum, whose condition
// that ordering meets. s = fl(a + b) either way, and both give the exact
// error a + b - s, so the pair is the same; the one difference, FastTwoSum's
// -0 error for b = -0 where TwoSum gives +0, is mapped to +0 on the integer
// pipe as well. (On GB300 an FP64 operation costs as much issue time as about
// 32 integer ones; on a CPU the branch-free six-operation form is the cheaper.)
template <>
EFT_HD void two_sum<double>(double a, double b, double &s, double &e) {
    const unsigned long long ma = eft_bits(a) & 0x7fffffffffffffffull;
    const unsigned long long mb = eft_bits(b) & 0x7fffffffffffffffull;
    const double x = mb > ma ? b : a, y = mb > ma ? a : b;
    const double t = add(x, y);
    const double z = sub(t, x);
    const double r = sub(y, z);
    s = t;
    e = eft_bits(r) == 0x8000000000000000ull ? 0.0 : r;
}

// TwoProd with FMA: p = fl(a b) and a b = p + e exactly.
template <typename T>
EFT_HD void two_prod(T a, T b, T &p, T &e) {
    T x = mul(a, b);
    p = x;
    e = fma_(a, b, -x);
}

// Algorithm 1, CompDotC: x . y as the pair (p, s), n >= 1 terms.
template <typename T, int N>
EFT_HD void comp_dot_c(const T (&x)[N], const T (&y)[N], T &p_out, T &s_out) {
    T p, s;
    two_prod(x[0], y[0], p, s);
#pragma unroll
    for (int i = 1; i < N; ++i) {
        T h, r, q;
        two_prod(x[i], y[i], h, r);
        two_sum(p, h, p, q);
        s = add(s, add(q, r));
    }
    p_out = p;
    s_out = s;
}

// Algorithm 2, CompDot: fl(p + s) of CompDotC.
template <typename T, int N>
EFT_HD T comp_dot(const T (&x)[N], const T (&y)[N]) {
    T p, s;
    comp_dot_c<T, N>(x, y, p, s);
    return add(p, s);
}

// Algorithm 4, AccuDOP: a d - b c as the pair (dop, err). The compensation is
// s + (r1 - r2): a d - b c = (p1 - p2) + (r1 - r2) exactly; the printed '+'
// would add the two product errors with the wrong sign. With renorm, one more
// TwoSum makes |err| <= u |dop| (the pair's value is unchanged).
template <typename T, bool Renorm>
EFT_HD void accu_dop(T a, T b, T c, T d, T &dop, T &err) {
    T p1, r1, p2, r2, s;
    two_prod(a, d, p1, r1);
    two_prod(b, c, p2, r2);
    two_sum(p1, -p2, dop, s);
    err = add(s, sub(r1, r2));
    if (Renorm) two_sum(dop, err, dop, err);
}

// Algorithm 6, SumNonNeg: [A, a] + [B, b] for non-negative pairs.
template <typename T>
EFT_HD void sum_non_neg(T A, T a, T B, T b, T &S, T &s) {
    T H, h;
    two_sum(A, B, H, h);
    T c = add(a, b);
    T d = add(h, c);
    fast_two_sum(H, d, S, s);
}

// Algorithm 5, SumOfSquares: |x|^2 as a pair (starting from the pair (0, 0)).
template <typename T, int N>
EFT_HD void sum_of_squares(const T (&x)[N], T &S, T &s) {
    T Sa = T(0), sa = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        T P, p;
        two_prod(x[j], x[j], P, p);
        sum_non_neg(Sa, sa, P, p, Sa, sa);
    }
    S = Sa;
    s = sa;
}

// Algorithm 7, SumOfSquaresC: |x + e|^2 as a pair, dropping the e^2 terms.
template <typename T, int N>
EFT_HD void sum_of_squares_c(const T (&x)[N], const T (&e)[N], T &S, T &s) {
    T Ss, ss;
    sum_of_squares<T, N>(x, Ss, ss);
    T Rs = comp_dot<T, N>(x, e);
    T R = fma_(T(2), Rs, ss);
    fast_two_sum(Ss, R, S, s);
}

// AccSqrt: sqrt of the pair (S, e), |e| <= u S, as a pair. The paper cites
// Rump (2023) and a Taylor expansion without printing the routine; this is
// the double-word square root: r = RN(sqrt S), the remainder S - r^2 is exact
// by one FMA for a correctly rounded r, and the first-order Taylor term gives
// er = (S - r^2 + e) / (2 r). S == 0 gives (0, 0).
template <typename T>
EFT_HD void acc_sqrt(T S, T e, T &r_out, T &er_out) {
    if (S == T(0)) {
        r_out = T(0);
        er_out = T(0);
        return;
    }
    T r = sqrt_(S);
    T rem = fma_(-r, r, S);
    r_out = r;
    er_out = div_(add(rem, e), mul(T(2), r));
}

}  // namespace sphx
