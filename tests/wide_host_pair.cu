// Host build of the integer-limb pair evaluation (pair_wide in
// paper_2510_09892_gb300/csrc/intersect.cuh is __host__ __device__), exported
// for tests/test_wide_host.py: the same source as the GPU kernels, run on the
// CPU against the exact oracle.
#include "../paper_2510_09892_gb300/csrc/intersect.cuh"

extern "C" void h_pair_wide(const double *A, const double *B, const double *Z, long long n,
                            double *pts, int *cnt) {
    const double nan = __builtin_nan("");
    for (long long i = 0; i < n; ++i) {
        const double x1[3] = {A[3 * i], A[3 * i + 1], A[3 * i + 2]};
        const double x2[3] = {B[3 * i], B[3 * i + 1], B[3 * i + 2]};
        sphx::PairOut o;
        sphx::pair_wide(x1, x2, Z[i], o);
        for (int r = 0; r < 2; ++r) {
            pts[6 * i + 3 * r + 0] = o.hit[r] ? o.px[r] : nan;
            pts[6 * i + 3 * r + 1] = o.hit[r] ? o.py[r] : nan;
            pts[6 * i + 3 * r + 2] = o.hit[r] ? Z[i] : nan;
        }
        cnt[i] = o.count;
    }
}
