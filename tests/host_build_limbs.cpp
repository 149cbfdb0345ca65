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
