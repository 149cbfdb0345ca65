// Software floating point with multi-limb integer mantissas, for the 32-bit
// integer pipe.
//
// GB300 issues 32-bit integer multiply-adds, adds and funnel shifts at 64 per
// SM per clock but FP64 operations at 2, so extended precision is far cheaper
// on integer limbs than as FP64 error-free transformations. W<K> holds
//
//     value = (-1)^neg * 0.M * 2^e,   M = m[K-1] .. m[0] (32-bit limbs),
//
// normalised so that bit 31 of m[K-1] is set (0.M in [1/2, 1)), or zero
// (all limbs 0, e = kZeroExp). Products keep the top K limbs of the 2K-limb
// product (the partial products of the lowest K - 1 columns are dropped: a
// relative error below 2^(6 - 32K)); sums align the smaller operand by a
// truncating shift. Every operation is therefore correct to a few units of
// 2^(-32K) relative to its operands, which is all the intersection formula
// needs: K = 4 (128 bits) for the cancelling terms n, |n_xy|^2, |n|^2, s^2,
// and K = 3 (96 bits) afterwards.
//
// The functions are __host__ __device__ so that the arithmetic is identical
// wherever it is compiled; the device intrinsics have exact host equivalents.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define SPHX_HD __host__ __device__ __forceinline__
#else
#define SPHX_HD inline
#endif

namespace sphx {
namespace wide {

constexpr int kZeroExp = -(1 << 28);

SPHX_HD int clz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return __clz(x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

// low 32 bits of (hi:lo) >> r, 0 <= r < 32
SPHX_HD uint32_t funnel_r(uint32_t lo, uint32_t hi, int r) {
#if defined(__CUDA_ARCH__)
    return __funnelshift_r(lo, hi, r);
#else
    return (uint32_t)(((((uint64_t)hi) << 32) | lo) >> (r & 31));
#endif
}

// high 32 bits of (hi:lo) << r, 0 <= r < 32
SPHX_HD uint32_t funnel_l(uint32_t lo, uint32_t hi, int r) {
#if defined(__CUDA_ARCH__)
    return __funnelshift_l(lo, hi, r);
#else
    return (uint32_t)((((((uint64_t)hi) << 32) | lo) << (r & 31)) >> 32);
#endif
}

SPHX_HD uint64_t bits_of(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}

SPHX_HD double double_of(uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, 8);
    return x;
#endif
}

SPHX_HD uint32_t fbits_of(float x) {
#if defined(__CUDA_ARCH__)
    return (uint32_t)__float_as_uint(x);
#else
    uint32_t b;
    memcpy(&b, &x, 4);
    return b;
#endif
}

SPHX_HD float float_of(uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float x;
    memcpy(&x, &b, 4);
    return x;
#endif
}

// r = a + b over K limbs; returns the carry out (0 or 1)
template <int K>
SPHX_HD uint32_t add_limbs(uint32_t (&r)[K], const uint32_t (&a)[K], const uint32_t (&b)[K]) {
#if defined(__CUDA_ARCH__)
    uint32_t c;
    if (K == 2) {
        asm("add.cc.u32 %0, %3, %5;\n\taddc.cc.u32 %1, %4, %6;\n\taddc.u32 %2, 0, 0;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(b[0]), "r"(b[1]));
    } else if (K == 3) {
        asm("add.cc.u32 %0, %4, %7;\n\taddc.cc.u32 %1, %5, %8;\n\taddc.cc.u32 %2, %6, %9;\n\t"
            "addc.u32 %3, 0, 0;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]));
    } else {
        asm("add.cc.u32 %0, %5, %9;\n\taddc.cc.u32 %1, %6, %10;\n\taddc.cc.u32 %2, %7, %11;\n\t"
            "addc.cc.u32 %3, %8, %12;\n\taddc.u32 %4, 0, 0;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]),
              "r"(b[3]));
    }
    return c;
#else
    uint32_t c = 0u;
    for (int i = 0; i < K; ++i) {
        const uint64_t t = (uint64_t)a[i] + b[i] + c;
        r[i] = (uint32_t)t;
        c = (uint32_t)(t >> 32);
    }
    return c;
#endif
}

// r = a - b over K limbs; returns the borrow out (0 or 1)
template <int K>
SPHX_HD uint32_t sub_limbs(uint32_t (&r)[K], const uint32_t (&a)[K], const uint32_t (&b)[K]) {
#if defined(__CUDA_ARCH__)
    uint32_t c;
    if (K == 2) {
        asm("sub.cc.u32 %0, %3, %5;\n\tsubc.cc.u32 %1, %4, %6;\n\tsubc.u32 %2, 0, 0;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(b[0]), "r"(b[1]));
    } else if (K == 3) {
        asm("sub.cc.u32 %0, %4, %7;\n\tsubc.cc.u32 %1, %5, %8;\n\tsubc.cc.u32 %2, %6, %9;\n\t"
            "subc.u32 %3, 0, 0;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]));
    } else {
        asm("sub.cc.u32 %0, %5, %9;\n\tsubc.cc.u32 %1, %6, %10;\n\tsubc.cc.u32 %2, %7, %11;\n\t"
            "subc.cc.u32 %3, %8, %12;\n\tsubc.u32 %4, 0, 0;"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(c)
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]),
              "r"(b[3]));
    }
    return c & 1u;
#else
    uint32_t bw = 0u;
    for (int i = 0; i < K; ++i) {
        const uint64_t t = (uint64_t)a[i] - b[i] - bw;
        r[i] = (uint32_t)t;
        bw = (uint32_t)(t >> 63);
    }
    return bw;
#endif
}

// three-word accumulator (t0, t1, t2) += x * y (product scanning)
SPHX_HD void mac3(uint32_t &t0, uint32_t &t1, uint32_t &t2, uint32_t x, uint32_t y) {
#if defined(__CUDA_ARCH__)
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;"
        : "+r"(t0), "+r"(t1), "+r"(t2)
        : "r"(x), "r"(y));
#else
    const uint64_t p = (uint64_t)x * y;
    const uint64_t lo = (uint64_t)t0 + (uint32_t)p;
    const uint64_t hi = (uint64_t)t1 + (p >> 32) + (lo >> 32);
    t0 = (uint32_t)lo;
    t1 = (uint32_t)hi;
    t2 += (uint32_t)(hi >> 32);
#endif
}

template <int K>
struct W {
    uint32_t m[K];
    int e;
    uint32_t neg;
};

template <int K>
SPHX_HD W<K> zero() {
    W<K> r;
#pragma unroll
    for (int i = 0; i < K; ++i) r.m[i] = 0u;
    r.e = kZeroExp;
    r.neg = 0u;
    return r;
}

template <int K>
SPHX_HD bool is_zero(const W<K> &a) {
    return a.m[K - 1] == 0u;  // normalised values have the top bit set
}

template <int K>
SPHX_HD W<K> negate(W<K> a) {
    a.neg ^= 1u;
    return a;
}

// m >>= d (d >= 0), truncating
template <int K>
SPHX_HD void shr(uint32_t (&m)[K], int d) {
    if (d < 32) {  // the common alignment: funnel shifts only
#pragma unroll
        for (int i = 0; i < K - 1; ++i) m[i] = funnel_r(m[i], m[i + 1], d);
        m[K - 1] = d ? (m[K - 1] >> d) : m[K - 1];
        return;
    }
    if (d >= 32 * K) {
#pragma unroll
        for (int i = 0; i < K; ++i) m[i] = 0u;
        return;
    }
    const int q = d >> 5;
#pragma unroll
    for (int b = 1; b < K; b <<= 1) {
        if (q & b) {
#pragma unroll
            for (int i = 0; i < K; ++i) m[i] = (i + b < K) ? m[i + b] : 0u;
        }
    }
    const int r = d & 31;
#pragma unroll
    for (int i = 0; i < K - 1; ++i) m[i] = funnel_r(m[i], m[i + 1], r);
    m[K - 1] = r ? (m[K - 1] >> r) : m[K - 1];
}

// bring the top set bit to bit 31 of m[K-1]; returns the shift applied (or -1 for zero)
template <int K>
SPHX_HD int normalize_mant(uint32_t (&m)[K]) {
    int sh = 0;
    if (m[K - 1] == 0u) {  // cancellation of 32 bits or more: move whole limbs first
#pragma unroll
        for (int step = 0; step < K - 1; ++step) {
            if (m[K - 1] == 0u) {
#pragma unroll
                for (int i = K - 1; i > 0; --i) m[i] = m[i - 1];
                m[0] = 0u;
                sh += 32;
            }
        }
        if (m[K - 1] == 0u) return -1;
    }
    const int c = clz32(m[K - 1]);
#pragma unroll
    for (int i = K - 1; i > 0; --i) m[i] = funnel_l(m[i - 1], m[i], c);
    m[0] <<= c;
    return sh + c;
}


template <int K>
SPHX_HD void normalize(W<K> &a) {
    const int sh = normalize_mant<K>(a.m);
    if (sh < 0) {
        a.e = kZeroExp;
        a.neg = 0u;
    } else {
        a.e -= sh;
    }
}

// exact conversion of a finite double (K >= 2)
template <int K>
SPHX_HD W<K> from_double(double x) {
    const uint64_t b = bits_of(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int ex = (int)((hi >> 20) & 0x7ffu);
    W<K> r;
#pragma unroll
    for (int i = 0; i < K - 2; ++i) r.m[i] = 0u;
    r.neg = hi >> 31;
    // normal numbers: the implicit bit and 52 fraction bits, moved to the top
    r.m[K - 1] = funnel_l(lo, (hi & 0xfffffu) | 0x100000u, 11);
    r.m[K - 2] = lo << 11;
    r.e = ex - 1022;
    if (ex == 0) {  // zero or subnormal (value = fraction 2^-1074)
        r.m[K - 1] = funnel_l(lo, hi & 0xfffffu, 11);
        r.e = -1021;
        normalize<K>(r);
    }
    return r;
}

// nearest double (ties to even on the K-limb value); exponents outside the
// normal range are handled by the (rare) subnormal / overflow branch
template <int K>
SPHX_HD double to_double(const W<K> &a) {
    if (is_zero(a)) return a.neg ? -0.0 : 0.0;
    const uint64_t t = ((uint64_t)a.m[K - 1] << 32) | a.m[K - 2];
    uint64_t mant = t >> 11;
    const uint32_t rbit = (uint32_t)(t >> 10) & 1u;
    uint32_t sticky = (uint32_t)(t & 0x3ffu);
#pragma unroll
    for (int i = 0; i < K - 2; ++i) sticky |= a.m[i];
    int e = a.e;
    if (rbit && (sticky || (mant & 1u))) {
        ++mant;
        if (mant >> 53) {
            mant >>= 1;
            ++e;
        }
    }
    const int be = e + 1022;
    const uint64_t sign = (uint64_t)a.neg << 63;
    if (be >= 1 && be <= 2046) return double_of(sign | ((uint64_t)be << 52) | (mant & ((1ull << 52) - 1)));
    if (be > 2046) return double_of(sign | (0x7ffull << 52));
    // subnormal result: round the 53-bit mantissa again at the 2^-1074 grid
    const int sh = 1 - be;  // >= 1
    if (sh > 53) return a.neg ? -0.0 : 0.0;
    const uint64_t q = mant >> sh;
    const uint64_t rem = mant & ((1ull << sh) - 1);
    const uint64_t half = 1ull << (sh - 1);
    const uint64_t qq = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
    return double_of(sign | qq);
}

// product scanning over columns K-1 .. 2K-1 of the 2K-limb product (the
// lower columns' partial products are dropped, see the header comment);
// returns the top K limbs normalised, exponent ea + eb (or one less)
template <int K, bool Square>
SPHX_HD W<K> mul_scan(const W<K> &a, const W<K> &b) {
    uint32_t out[K + 1];
    uint32_t t0 = 0u, t1 = 0u, t2 = 0u;
#pragma unroll
    for (int c = K - 1; c < 2 * K; ++c) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int j = c - i;
            if (j < 0 || j >= K) continue;
            if (Square && i > j) continue;
            mac3(t0, t1, t2, a.m[i], b.m[j]);
            if (Square && i < j) mac3(t0, t1, t2, a.m[i], b.m[j]);
        }
        out[c - (K - 1)] = t0;
        t0 = t1;
        t1 = t2;
        t2 = 0u;
    }
    W<K> r;
    r.neg = a.neg ^ b.neg;
    r.e = a.e + b.e;
    if (out[K] >> 31) {
#pragma unroll
        for (int i = 0; i < K; ++i) r.m[i] = out[i + 1];
    } else {  // product in [1/4, 1/2): one bit up, taking the guard limb's top bit
#pragma unroll
        for (int i = 0; i < K; ++i) r.m[i] = funnel_l(out[i], out[i + 1], 1);
        r.e -= 1;
    }
    if (is_zero(a) || is_zero(b)) return zero<K>();
    return r;
}

// top K limbs of a * b
template <int K>
SPHX_HD W<K> mul(const W<K> &a, const W<K> &b) {
    return mul_scan<K, false>(a, b);
}

// top K limbs of a * a (off-diagonal partial products counted twice)
template <int K>
SPHX_HD W<K> sqr(const W<K> &a) {
    return mul_scan<K, true>(a, a);
}

// exact product of two 2-limb values as a 4-limb value
SPHX_HD W<4> mul_exact(const W<2> &a, const W<2> &b) {
    uint32_t p[4];
    uint32_t t0 = 0u, t1 = 0u, t2 = 0u;
    mac3(t0, t1, t2, a.m[0], b.m[0]);
    p[0] = t0;
    t0 = t1;
    t1 = t2;
    t2 = 0u;
    mac3(t0, t1, t2, a.m[0], b.m[1]);
    mac3(t0, t1, t2, a.m[1], b.m[0]);
    p[1] = t0;
    t0 = t1;
    t1 = t2;
    t2 = 0u;
    mac3(t0, t1, t2, a.m[1], b.m[1]);
    p[2] = t0;
    p[3] = t1;
    W<4> r;
    r.neg = a.neg ^ b.neg;
    r.e = a.e + b.e;
    if (p[3] >> 31) {
#pragma unroll
        for (int i = 0; i < 4; ++i) r.m[i] = p[i];
    } else {
#pragma unroll
        for (int i = 3; i > 0; --i) r.m[i] = funnel_l(p[i - 1], p[i], 1);
        r.m[0] = p[0] << 1;
        r.e -= 1;
    }
    if (is_zero(a) || is_zero(b)) return zero<4>();
    return r;
}

// a + b
template <int K>
SPHX_HD W<K> add(W<K> a, W<K> b) {
    if (a.e < b.e) {
        const W<K> t = a;
        a = b;
        b = t;
    }
    shr<K>(b.m, a.e - b.e);
    W<K> r;
    r.e = a.e;
    r.neg = a.neg;
    if (a.neg == b.neg) {
        if (add_limbs<K>(r.m, a.m, b.m)) {  // carry into a new top bit
#pragma unroll
            for (int i = 0; i < K - 1; ++i) r.m[i] = funnel_r(r.m[i], r.m[i + 1], 1);
            r.m[K - 1] = (r.m[K - 1] >> 1) | 0x80000000u;
            r.e += 1;
        }
        if (is_zero(r)) r.e = kZeroExp;
        return r;
    }
    if (sub_limbs<K>(r.m, a.m, b.m)) {  // |b| > |a| (equal exponents): negate the difference
        uint32_t z[K];
#pragma unroll
        for (int i = 0; i < K; ++i) z[i] = 0u;
        sub_limbs<K>(r.m, z, r.m);
        r.neg ^= 1u;
    }
    normalize<K>(r);
    return r;
}

// a + b for operands of the same sign (sums of squares)
template <int K>
SPHX_HD W<K> add_same(W<K> a, W<K> b) {
    if (a.e < b.e) {
        const W<K> t = a;
        a = b;
        b = t;
    }
    shr<K>(b.m, a.e - b.e);
    W<K> r;
    r.e = a.e;
    r.neg = a.neg;
    if (add_limbs<K>(r.m, a.m, b.m)) {
#pragma unroll
        for (int i = 0; i < K - 1; ++i) r.m[i] = funnel_r(r.m[i], r.m[i + 1], 1);
        r.m[K - 1] = (r.m[K - 1] >> 1) | 0x80000000u;
        r.e += 1;
    }
    if (is_zero(r)) r.e = kZeroExp;
    return r;
}

template <int K>
SPHX_HD W<K> sub(const W<K> &a, const W<K> &b) {
    return add<K>(a, negate<K>(b));
}

// drop (truncate) low limbs
template <int K, int J>
SPHX_HD W<J> narrow(const W<K> &a) {
    static_assert(J <= K, "narrow to fewer limbs");
    W<J> r;
#pragma unroll
    for (int i = 0; i < J; ++i) r.m[i] = a.m[K - J + i];
    r.e = a.e;
    r.neg = a.neg;
    return r;
}

SPHX_HD double fma64(double a, double b, double c) {
#if defined(__CUDA_ARCH__)
    return __fma_rn(a, b, c);
#else
    return __builtin_fma(a, b, c);
#endif
}

SPHX_HD float fma32(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return __builtin_fmaf(a, b, c);
#endif
}

// approximate 1 / sqrt(x) for a positive normal float (about 2^-22)
SPHX_HD float rsqrt_approx(float x) {
#if defined(__CUDA_ARCH__)
    return rsqrtf(x);
#else
    return 1.0f / __builtin_sqrtf(x);
#endif
}

// correctly rounded FP32 reciprocal and reciprocal square root (about 2^-24),
// the seeds of the FP64 steps below; the host computes the same roundings
SPHX_HD float rcp32(float x) {
#if defined(__CUDA_ARCH__)
    return __frcp_rn(x);
#else
    return (float)(1.0 / (double)x);
#endif
}

SPHX_HD float rsqrt32(float x) {
#if defined(__CUDA_ARCH__)
    return __frsqrt_rn(x);
#else
    return (float)(1.0 / __builtin_sqrt((double)x));
#endif
}

// high 64 bits of the 128-bit product a * b
SPHX_HD uint64_t umul64hi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// a 32-bit unsigned integer rounded to the nearest float
SPHX_HD float f32_of_u32(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return __uint2float_rn(x);
#else
    return (float)x;
#endif
}

// R = r 2^31 for an FP32 r in [1, 2] (2 itself saturates to 2^32 - 1)
SPHX_HD uint32_t fixed31_of(float r) {
    const uint32_t b = fbits_of(r);
    return (b >> 23) == 127u ? (((b & 0x7fffffu) | 0x800000u) << 8) : 0xffffffffu;
}

// R r / 2^32 for a signed residual r (|r| < 2^63) and R < 2^32, truncated toward 0
SPHX_HD int64_t mul_fixed31(uint32_t R, int64_t r) {
    const uint64_t m = r < 0 ? (uint64_t)0 - (uint64_t)r : (uint64_t)r;
    const uint64_t p = (uint64_t)R * (uint32_t)(m >> 32) + (((uint64_t)R * (uint32_t)m) >> 32);
    return r < 0 ? -(int64_t)p : (int64_t)p;
}

// the 96-bit value (hi:lo64) plus a signed 64-bit amount, as limbs; the
// result is clamped to 2^96 - 1 on a carry out (callers' values stay below 2^96
// except by rounding-size amounts)
SPHX_HD void add_signed96(uint32_t (&m)[3], uint32_t hi, uint64_t lo, int64_t d) {
    uint64_t l2 = lo + (uint64_t)d;
    uint32_t h2 = hi;
    if (d >= 0) {
        if (l2 < lo) {
            if (++h2 == 0u) {
                m[0] = m[1] = m[2] = 0xffffffffu;
                return;
            }
        }
    } else if (l2 > lo) {
        --h2;
    }
    m[0] = (uint32_t)l2;
    m[1] = (uint32_t)(l2 >> 32);
    m[2] = h2;
}

// 1 / a for a != 0 to about 2^-91, on the integer pipe. With f = 0.M in
// [1/2, 1) the mantissa of a (M = m2 m1 m0): an FP32 seed r0 ~ 1/f from f
// rounded to 24 bits (1 - f r0 within 2^-23), then two Newton steps
// r <- r + r (1 - f r) in fixed point (r0 2^31, r1 2^62, r2 2^94). Each
// residual 1 - f r is small, so it is read from the middle limbs of f r: the
// bits of 2^k - f r 2^k above a limb boundary, taken modulo 2^64, are the
// residual as a signed 64-bit number (the borrow from the dropped low limbs
// is below one unit). Relative error: the second residual squared
// (<= 2^-92) plus truncations of a few units of 2^-94.
template <int K>
SPHX_HD W<K> recip_int(const W<K> &a) {
    static_assert(K == 3, "recip_int works on 96-bit mantissas");
    const uint32_t m0 = a.m[0], m1 = a.m[1], m2 = a.m[2];
    W<3> q;
    q.neg = a.neg;
    if (m2 == 0x80000000u && (m1 | m0) == 0u) {  // f = 1/2: 1/f = 2 exactly
        q.m[0] = q.m[1] = 0u;
        q.m[2] = 0x80000000u;
        q.e = 2 - a.e;
        return q;
    }
    // seed: f rounded to 24 bits, t in [2^23, 2^24], as the float t 2^-24
    const uint32_t t = (m2 >> 8) + ((m2 >> 7) & 1u);
    const uint32_t R0 = fixed31_of(rcp32(float_of(0x3e800000u + t)));  // r0 2^31
    // step 1: f r0 = M R0 2^-127; bits 64.. of 2^127 - M R0 give e0 2^63
    const uint64_t p0 = (uint64_t)m0 * R0, p1 = (uint64_t)m1 * R0, p2 = (uint64_t)m2 * R0;
    const uint64_t mid = (p0 >> 32) + (uint32_t)p1;
    const uint64_t T1 = p2 + (p1 >> 32) + (mid >> 32);
    const int64_t e0 = (int64_t)(0x8000000000000000ull - T1);
    const uint64_t R1 = ((uint64_t)R0 << 31) + (uint64_t)mul_fixed31(R0, e0);  // r1 2^62
    // step 2: f r1 = M R1 2^-158; bits 64..127 of 2^158 - M R1 give e1 2^94
    const uint32_t rl = (uint32_t)R1, rh = (uint32_t)(R1 >> 32);
    const uint64_t a0 = (uint64_t)m0 * rl, a1 = (uint64_t)m0 * rh, b0 = (uint64_t)m1 * rl;
    const uint64_t b1 = (uint64_t)m1 * rh, c0 = (uint64_t)m2 * rl, c1 = (uint64_t)m2 * rh;
    const uint64_t col1 = (a0 >> 32) + (uint32_t)a1 + (uint32_t)b0;  // bits 32.. (< 3 2^32)
    const uint64_t T2 = b1 + c0 + (c1 << 32) + (a1 >> 32) + (b0 >> 32) + (col1 >> 32);
    const int64_t e1 = (int64_t)(0ull - T2);
    // r2 = r1 + r1 e1 = R1 2^32 + R1 e1 2^-62 (units of 2^-94)
    const uint64_t u = e1 < 0 ? (uint64_t)0 - (uint64_t)e1 : (uint64_t)e1;
    const uint64_t corr = (umul64hi(R1, u) << 2) | ((R1 * u) >> 62);
    add_signed96(q.m, rh, (uint64_t)rl << 32, e1 < 0 ? -(int64_t)corr : (int64_t)corr);
    const int sh = normalize_mant<3>(q.m);  // r2 2^94 -> 0.Q: 1 / a = 0.Q 2^(2 - sh - e)
    q.e = 2 - sh - a.e;
    return q;
}

// sqrt(a) for a > 0 to about 2^-91, on the integer pipe. With a = f 2^(2h),
// f in [1/4, 1) (M shifted right by one bit when the exponent is odd): an
// FP32 seed y0 ~ 1/sqrt(f), one Newton step y1 = y0 + y0 (1 - f y0^2) / 2
// (about 2^-46) in fixed point, d = f y1 truncated to 64 bits, the residual
// f - d^2 exactly in 128 bits, and sqrt(f) = d + (f - d^2) y1 / 2, whose
// error is about twice the square of y1's.
template <int K>
SPHX_HD W<K> sqrt_int(const W<K> &a) {
    static_assert(K == 3, "sqrt_int works on 96-bit mantissas");
    const int odd = a.e & 1;
    const int h = (a.e + odd) / 2;
    // F = f 2^96
    const uint32_t f0 = odd ? funnel_r(a.m[0], a.m[1], 1) : a.m[0];
    const uint32_t f1 = odd ? funnel_r(a.m[1], a.m[2], 1) : a.m[1];
    const uint32_t f2 = odd ? (a.m[2] >> 1) : a.m[2];
    // seed: the top limb rounded to a float and scaled by 2^-32 (exact)
    const uint32_t Y0 = fixed31_of(rsqrt32(f32_of_u32(f2) * 2.3283064365386963e-10f));  // y0 2^31
    // step 1: F Y0^2 = f y0^2 2^158; its bits 96.. are f y0^2 2^62 (lower
    // partial products dropped: a few units)
    const uint64_t Q = (uint64_t)Y0 * Y0;  // y0^2 2^62 < 2^64
    const uint32_t ql = (uint32_t)Q, qh = (uint32_t)(Q >> 32);
    const uint64_t TT = (uint64_t)f2 * qh + (((uint64_t)f1 * qh) >> 32) + (((uint64_t)f2 * ql) >> 32);
    const int64_t g = (int64_t)(0x4000000000000000ull - TT);  // (1 - f y0^2) 2^62
    const uint64_t Y1 = ((uint64_t)Y0 << 31) + (uint64_t)mul_fixed31(Y0, g);  // y1 2^62
    // d 2^64 = F Y1 2^-94 (bits 94.. of the product; clamped below 1)
    const uint32_t yl = (uint32_t)Y1, yh = (uint32_t)(Y1 >> 32);
    const uint64_t top = (uint64_t)f2 * yh;
    const uint64_t D0 = top << 2;
    uint64_t D = D0 + (((uint64_t)f2 * yl) >> 30) + (((uint64_t)f1 * yh) >> 30);
    if ((top >> 62) != 0u || D < D0) D = ~0ull;
    // (f - d^2) 2^128 = F 2^32 - D^2, exact modulo 2^128; |f - d^2| < 2^-45,
    // so bits 30..93 hold it as a signed 64-bit number (units of 2^-98)
    const uint64_t dl = D * D, dh = umul64hi(D, D);
    const uint64_t al = (uint64_t)f0 << 32, ah = ((uint64_t)f2 << 32) | f1;
    const uint64_t rl = al - dl;
    const uint64_t rh = ah - dh - (al < dl ? 1u : 0u);
    const int64_t rho = (int64_t)((rh << 34) | (rl >> 30));
    // sqrt(f) 2^96 = D 2^32 + rho Y1 2^-65
    const uint64_t u = rho < 0 ? (uint64_t)0 - (uint64_t)rho : (uint64_t)rho;
    const uint64_t corr = umul64hi(u, Y1) >> 1;
    W<3> r;
    add_signed96(r.m, (uint32_t)(D >> 32), (uint64_t)(uint32_t)D << 32,
                 rho < 0 ? -(int64_t)corr : (int64_t)corr);
    const int sh = normalize_mant<3>(r.m);
    r.e = h - sh;
    r.neg = 0u;
    return r;
}

// s = a + b and d = a - b, sharing the alignment
template <int K>
SPHX_HD void add_sub(W<K> a, W<K> b, W<K> &s, W<K> &d) {
    const bool sw = a.e < b.e;
    if (sw) {
        const W<K> t = a;
        a = b;
        b = t;
    }
    shr<K>(b.m, a.e - b.e);
    W<K> ad, sb;  // magnitude sum and difference, signed like a
    ad.e = sb.e = a.e;
    ad.neg = sb.neg = a.neg;
    if (add_limbs<K>(ad.m, a.m, b.m)) {
#pragma unroll
        for (int i = 0; i < K - 1; ++i) ad.m[i] = funnel_r(ad.m[i], ad.m[i + 1], 1);
        ad.m[K - 1] = (ad.m[K - 1] >> 1) | 0x80000000u;
        ad.e += 1;
    }
    if (is_zero(ad)) ad.e = kZeroExp;
    if (sub_limbs<K>(sb.m, a.m, b.m)) {
        uint32_t z[K];
#pragma unroll
        for (int i = 0; i < K; ++i) z[i] = 0u;
        sub_limbs<K>(sb.m, z, sb.m);
        sb.neg ^= 1u;
    }
    normalize<K>(sb);
    // a + b is the magnitude sum when the signs agree, else the difference;
    // a - b the other one (negated back when the operands were swapped)
    const bool same = a.neg == b.neg;
    s = same ? ad : sb;
    d = same ? sb : ad;
    if (sw) d.neg ^= 1u;
    if (is_zero(d)) d.neg = 0u;
}

}  // namespace wide
}  // namespace sphx
