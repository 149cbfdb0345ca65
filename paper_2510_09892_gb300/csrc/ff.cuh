// Float-float arithmetic: unevaluated pairs hi + lo of FP32 values (about 48
// bits), built from the error-free transformations of Sec. 5 of Chen,
// Ullrich, Panetta (TwoSum, FastTwoSum, FMA-based TwoProd) applied to FP32.
// GB300 runs FP32 FMAs at about 120 per SM per clock against 2 for FP64.
//
// Every step is one correctly rounded FP32 operation written with an explicit
// rounding intrinsic on the device (and as a plain operation on the host,
// where the code must be compiled without floating-point contraction), so the
// two builds compute identical bits.
#pragma once
#include "wide.cuh"

namespace sphx {
namespace ffa {

SPHX_HD float add(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
SPHX_HD float sub(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
SPHX_HD float mul(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
SPHX_HD float fma(float a, float b, float c) { return wide::fma32(a, b, c); }
SPHX_HD float sqrt(float a) {
#if defined(__CUDA_ARCH__)
    return __fsqrt_rn(a);
#else
    return __builtin_sqrtf(a);
#endif
}
SPHX_HD float rcp(float a) { return wide::rcp32(a); }

struct F2 {
    float hi, lo;
};

// TwoSum (Knuth): a + b = s + e exactly
SPHX_HD F2 two_sum(float a, float b) {
    const float s = add(a, b);
    const float bv = sub(s, a);
    const float av = sub(s, bv);
    return {s, add(sub(a, av), sub(b, bv))};
}
// FastTwoSum (Dekker): exact when exponent(a) >= exponent(b)
SPHX_HD F2 fast_two_sum(float a, float b) {
    const float s = add(a, b);
    return {s, sub(b, sub(s, a))};
}
SPHX_HD F2 neg(F2 a) { return {-a.hi, -a.lo}; }

// (a.hi + a.lo) + (b.hi + b.lo)
SPHX_HD F2 add2(F2 a, F2 b) {
    const F2 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, add(s.lo, add(a.lo, b.lo)));
}
// (a.hi + a.lo) (b.hi + b.lo): TwoProd of the high parts plus the cross terms
SPHX_HD F2 mul2(F2 a, F2 b) {
    const float p = mul(a.hi, b.hi);
    float e = fma(a.hi, b.hi, -p);
    e = fma(a.hi, b.lo, e);
    e = fma(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
SPHX_HD F2 sqr2(F2 a) {
    const float p = mul(a.hi, a.hi);
    float e = fma(a.hi, a.hi, -p);
    e = fma(add(a.hi, a.hi), a.lo, e);
    return fast_two_sum(p, e);
}
// sqrt of a >= 0: r = RN(sqrt a.hi), the remainder a.hi - r^2 is exact by one
// FMA, and the first Taylor term gives the low part (rem + a.lo) / (2 r)
SPHX_HD F2 sqrt2(F2 a) {
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    const float r = sqrt(a.hi);
    const float rem = add(fma(-r, r, a.hi), a.lo);
    return fast_two_sum(r, mul(rem, mul(0.5f, rcp(r))));
}
// 1 / b: r0 = RN(1 / b.hi), then one Newton step r0 (1 + e), e = 1 - b r0
SPHX_HD F2 rcp2(F2 b) {
    const float r0 = rcp(b.hi);
    const float e = sub(fma(-b.hi, r0, 1.0f), mul(b.lo, r0));
    return fast_two_sum(r0, mul(r0, e));
}

// value(a) 2^-sc as hi + lo, for an integer-limb value a (K >= 2): hi holds
// the top 24 mantissa bits, lo the next 24 rounded to nearest, so the pair is
// within 2^-49 relative of the value. 0 when the value is below 2^-125 (the
// callers' values are at most 2 in magnitude).
template <int K>
SPHX_HD F2 ff_of(const wide::W<K> &a, int sc) {
    if (wide::is_zero(a)) return {0.0f, 0.0f};
    const uint32_t top = a.m[K - 1], nxt = a.m[K - 2];
    const int eh = a.e - sc;  // value = 0.M 2^eh, in [2^(eh-1), 2^eh)
    if (eh - 1 + 127 <= 1 || eh - 1 + 127 >= 255) return {0.0f, 0.0f};
    const uint32_t sign = a.neg << 31;
    const float hi = wide::float_of(sign | ((uint32_t)(eh - 1 + 127) << 23) | ((top >> 8) & 0x7fffffu));
    // the next 24 bits, rounded on the bit below them: L 2^(eh - 48), L <= 2^24
    const uint32_t L = (((top & 0xffu) << 16) | (nxt >> 16)) + ((nxt >> 15) & 1u);
    const int le = eh - 48 + 127;  // exponent field of 2^(eh - 48)
    if (L == 0u || le <= 0) return {hi, 0.0f};
    const float lo = mul(wide::f32_of_u32(L), wide::float_of((uint32_t)le << 23));
    return fast_two_sum(hi, a.neg ? -lo : lo);
}

// a normal or zero float as a double (exact), by its bits
SPHX_HD double to_f64(float f) {
    const uint32_t b = wide::fbits_of(f);
    const uint32_t fe = (b >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    if (fe == 0) return wide::double_of(sign);
    return wide::double_of(sign | ((uint64_t)(fe - 127u + 1023u) << 52) |
                           ((uint64_t)(b & 0x7fffffu) << 29));
}

}  // namespace ffa
}  // namespace sphx
