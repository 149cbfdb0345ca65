// Host build of the integer-limb arithmetic (paper_2510_09892_gb300/csrc/wide.cuh
// compiles for the host as well), exported for tests/test_host_builds.py.
// A value is passed as three 32-bit limbs (0.M with the top bit set), an
// exponent and a sign.
#include "../paper_2510_09892_gb300/csrc/wide.cuh"

using namespace sphx::wide;

static W<3> mk(const uint32_t *m, int e, int neg) {
    W<3> a;
    a.m[0] = m[0];
    a.m[1] = m[1];
    a.m[2] = m[2];
    a.e = e;
    a.neg = (uint32_t)neg;
    return a;
}

static void put(const W<3> &r, uint32_t *m, int *e, int *neg) {
    m[0] = r.m[0];
    m[1] = r.m[1];
    m[2] = r.m[2];
    *e = r.e;
    *neg = (int)r.neg;
}

extern "C" {
void h_recip(const uint32_t *a, int ea, int na, uint32_t *r, int *er, int *nr) {
    put(recip_int<3>(mk(a, ea, na)), r, er, nr);
}
void h_sqrt(const uint32_t *a, int ea, uint32_t *r, int *er, int *nr) {
    put(sqrt_int<3>(mk(a, ea, 0)), r, er, nr);
}
void h_mul(const uint32_t *a, int ea, int na, const uint32_t *b, int eb, int nb, uint32_t *r,
           int *er, int *nr) {
    put(mul<3>(mk(a, ea, na), mk(b, eb, nb)), r, er, nr);
}
void h_add(const uint32_t *a, int ea, int na, const uint32_t *b, int eb, int nb, uint32_t *r,
           int *er, int *nr) {
    put(add<3>(mk(a, ea, na), mk(b, eb, nb)), r, er, nr);
}
double h_to_double(const uint32_t *a, int ea, int na) { return to_double<3>(mk(a, ea, na)); }
}

// Exhaustive check of the FP32 seeds' host forms: rcp32 over every float in
// [1, 2) and rsqrt32 over every float in [1, 4) (scaling by powers of two is
// exact, so these binades stand for every normal input), each against the
// correctly rounded value decided in exact integer arithmetic. The device
// forms are __frcp_rn and __frsqrt_rn, which are correctly rounded by
// definition, so agreement here makes the host and device seeds identical.
// Returns the number of inputs whose result is not correctly rounded and
// stores the first such input's bit pattern in *first_bad.
static bool rcp_ok(uint32_t X) {  // x = X 2^-23, X in [2^23, 2^24)
    const float x = (float)X * 0x1p-23f;
    const float y = rcp32(x);
    if (X == (1u << 23)) return y == 1.0f;
    const uint64_t Y = (uint64_t)(y * 0x1p24f);  // y = Y 2^-24, Y in [2^23, 2^24)
    if ((float)Y * 0x1p-24f != y || Y < (1u << 23) || Y >= (1u << 24)) return false;
    const __int128 d = (__int128)2 * Y * X - ((__int128)1 << 48);  // 2^48 (y - 1/x) x
    const __int128 ad = d < 0 ? -d : d;
    return ad < (__int128)X || (ad == (__int128)X && (Y & 1) == 0);
}

static bool rsqrt_ok(uint32_t X, int s) {  // x = X 2^-s, s = 23 ([1, 2)) or 22 ([2, 4))
    const float x = (float)X * (s == 23 ? 0x1p-23f : 0x1p-22f);
    const float y = rsqrt32(x);
    if (X == (1u << 23) && s == 23) return y == 1.0f;
    const uint64_t Y = (uint64_t)(y * 0x1p24f);
    if ((float)Y * 0x1p-24f != y || Y < (1u << 23) || Y >= (1u << 24)) return false;
    // y is correctly rounded iff (2Y - 1)^2 x <= 2^50 <= (2Y + 1)^2 x
    const __int128 lo = (__int128)(2 * Y - 1) * (2 * Y - 1) * X;
    const __int128 hi = (__int128)(2 * Y + 1) * (2 * Y + 1) * X;
    const __int128 t = (__int128)1 << (50 + s);
    return lo <= t && t <= hi;
}

extern "C" uint64_t h_check_seeds(int which, uint32_t *first_bad) {
    uint64_t bad = 0;
    *first_bad = 0;
    for (uint32_t X = 1u << 23; X < (1u << 24); ++X) {
        bool ok = which == 0 ? rcp_ok(X) : (rsqrt_ok(X, 23) && rsqrt_ok(X, 22));
        if (!ok && bad++ == 0) *first_bad = X;
    }
    return bad;
}
