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
    const int c = clz32(m[K - 1]);
#pragma unroll
    for (int i = K - 1; i > 0; --i) m[i] = funnel_l(m[i - 1], m[i], c);
    m[0] = c ? (m[0] << c) : m[0];
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
    const int ex = (int)((b >> 52) & 0x7ff);
    uint64_t frac = b & ((1ull << 52) - 1);
    W<K> r = zero<K>();
    if (ex == 0 && frac == 0) return r;
    r.neg = (uint32_t)(b >> 63);
    uint64_t t;
    if (ex == 0) {  // subnormal: value = frac 2^-1074
        int lz = clz32((uint32_t)(frac >> 32));
        if (lz == 32) lz += clz32((uint32_t)frac);
        t = frac << lz;  // top bit set
        r.e = (64 - lz) - 1074;
    } else {
        t = (frac | (1ull << 52)) << 11;
        r.e = ex - 1022;
    }
    r.m[K - 1] = (uint32_t)(t >> 32);
    r.m[K - 2] = (uint32_t)t;
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

// top K limbs of a * b (see the header comment for the truncation)
template <int K>
SPHX_HD W<K> mul(const W<K> &a, const W<K> &b) {
    uint32_t acc[2 * K];
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) acc[i] = 0u;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        uint32_t carry = 0u;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (i + j >= K - 1) {
                const uint64_t t = (uint64_t)a.m[i] * b.m[j] + acc[i + j] + carry;
                acc[i + j] = (uint32_t)t;
                carry = (uint32_t)(t >> 32);
            }
        }
        acc[i + K] = carry;
    }
    W<K> r;
    r.neg = a.neg ^ b.neg;
    r.e = a.e + b.e;
    if (is_zero(a) || is_zero(b)) return zero<K>();
    if (acc[2 * K - 1] >> 31) {
#pragma unroll
        for (int i = 0; i < K; ++i) r.m[i] = acc[K + i];
    } else {  // product in [1/4, 1/2): one bit up, taking the guard limb's top bit
#pragma unroll
        for (int i = 0; i < K; ++i) r.m[i] = funnel_l(acc[K - 1 + i], acc[K + i], 1);
        r.e -= 1;
    }
    return r;
}

// exact product of two 2-limb values as a 4-limb value
SPHX_HD W<4> mul_exact(const W<2> &a, const W<2> &b) {
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        uint32_t carry = 0u;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint64_t t = (uint64_t)a.m[i] * b.m[j] + acc[i + j] + carry;
            acc[i + j] = (uint32_t)t;
            carry = (uint32_t)(t >> 32);
        }
        acc[i + 2] = carry;
    }
    W<4> r;
    if (is_zero(a) || is_zero(b)) return zero<4>();
    r.neg = a.neg ^ b.neg;
    r.e = a.e + b.e;
    if (acc[3] >> 31) {
#pragma unroll
        for (int i = 0; i < 4; ++i) r.m[i] = acc[i];
    } else {
#pragma unroll
        for (int i = 3; i > 0; --i) r.m[i] = funnel_l(acc[i - 1], acc[i], 1);
        r.m[0] = acc[0] << 1;
        r.e -= 1;
    }
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
    const uint32_t sub = a.neg ^ b.neg;
    const uint32_t mask = 0u - sub;
    uint32_t carry = sub;
    W<K> r;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const uint64_t t = (uint64_t)a.m[i] + (b.m[i] ^ mask) + carry;
        r.m[i] = (uint32_t)t;
        carry = (uint32_t)(t >> 32);
    }
    r.e = a.e;
    r.neg = a.neg;
    if (!sub) {
        if (carry) {  // overflow into a new top bit
#pragma unroll
            for (int i = 0; i < K - 1; ++i) r.m[i] = funnel_r(r.m[i], r.m[i + 1], 1);
            r.m[K - 1] = (r.m[K - 1] >> 1) | 0x80000000u;
            r.e += 1;
        }
        if (is_zero(a)) return b;  // both operands were zero or a was
        return r;
    }
    if (!carry) {  // |b| > |a|: the difference is negative, take its magnitude
        uint32_t c = 1u;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const uint64_t t = (uint64_t)(~r.m[i]) + c;
            r.m[i] = (uint32_t)t;
            c = (uint32_t)(t >> 32);
        }
        r.neg ^= 1u;
    }
    normalize<K>(r);
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

// 0.M of a non-zero value as a float (top 24 bits, truncated), in [1/2, 1)
template <int K>
SPHX_HD float mant_float(const W<K> &a) {
    return float_of((126u << 23) | ((a.m[K - 1] >> 8) & 0x7fffffu));
}

// a small non-negative float as a W<K> (exact)
template <int K>
SPHX_HD W<K> from_float(float f) {
    const uint32_t b = fbits_of(f);
    W<K> r = zero<K>();
    if ((b & 0x7fffffffu) == 0u) return r;
    r.neg = b >> 31;
    r.e = (int)((b >> 23) & 0xff) - 126;
    r.m[K - 1] = ((b & 0x7fffffu) | 0x800000u) << 8;
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

SPHX_HD float rsqrt_seed(float x) {
#if defined(__CUDA_ARCH__)
    return __frsqrt_rn(x);
#else
    return (float)(1.0 / __builtin_sqrt((double)x));
#endif
}

SPHX_HD float rcp_seed(float x) {
#if defined(__CUDA_ARCH__)
    return __frcp_rn(x);
#else
    return (float)(1.0 / (double)x);
#endif
}

// sqrt(a) for a > 0: Newton's iteration y <- y (3 - f y^2) / 2 for 1/sqrt(f)
// from a correctly rounded FP32 seed (about 2^-23), twice (about 2^-88),
// then sqrt(a) = f y 2^h
template <int K>
SPHX_HD W<K> sqrt_pos(const W<K> &a) {
    // a = f 2^(2h): f = 0.M in [1/2, 1) for an even exponent, 0.M / 2 in
    // [1/4, 1/2) for an odd one
    W<K> f = a;
    const int odd = a.e & 1;
    f.e = -odd;
    f.neg = 0u;
    const int h = (a.e + odd) / 2;
    float ff = mant_float<K>(a);
    if (odd) ff *= 0.5f;
    W<K> y = from_float<K>(rsqrt_seed(ff));
    W<K> three = zero<K>();
    three.m[K - 1] = 0xC0000000u;  // 0.75 * 2^2
    three.e = 2;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        W<K> t = mul<K>(f, mul<K>(y, y));
        y = mul<K>(y, sub<K>(three, t));
        y.e -= 1;
    }
    W<K> s = mul<K>(f, y);
    s.e += h;
    return s;
}

// 1 / a for a != 0: Newton's iteration r <- r (2 - f r) from an FP32 seed, twice
template <int K>
SPHX_HD W<K> recip(const W<K> &a) {
    W<K> f = a;
    f.e = 0;
    f.neg = 0u;
    W<K> r = from_float<K>(rcp_seed(mant_float<K>(a)));
    W<K> two = zero<K>();
    two.m[K - 1] = 0x80000000u;  // 0.5 * 2^2
    two.e = 2;
#pragma unroll
    for (int it = 0; it < 2; ++it) r = mul<K>(r, sub<K>(two, mul<K>(f, r)));
    r.e -= a.e;
    r.neg = a.neg;
    return r;
}

}  // namespace wide
}  // namespace sphx
