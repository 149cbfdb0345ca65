// The adaptive mode of the dense call: dense_kernel<kAdaptive> (dense.cuh)
// with the filter of adaptive.cuh and the integer-limb form as its fallback.
#include "dense.cuh"

namespace sphx {

void launch_adaptive(const double *A, const double *B, const double *Z, int64_t n, double *P,
                     int32_t *C, double gate_ulps, unsigned long long *fallback, cudaStream_t s) {
    launch_dense<kAdaptive>(A, B, Z, n, P, C, s, fallback, gate_ulps);
}

}  // namespace sphx

using namespace sphx;

extern "C" sphx_status sphx_intersect_gca_constlat_adaptive(const double *A, const double *B,
                                                            const double *z0, int64_t n,
                                                            double *out_pts, int32_t *out_count,
                                                            double gate_ulps,
                                                            unsigned long long *fallback_count,
                                                            sphx_stream stream) {
    if (n < 0 || !(gate_ulps >= 1.0 && gate_ulps <= 67108864.0)) return SPHX_ERR_INVALID_ARG;
    if (n == 0) return SPHX_OK;
    if (!A || !B || !z0 || !out_pts || !out_count) return SPHX_ERR_INVALID_ARG;
    auto misaligned = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
    if (misaligned(A) || misaligned(B) || misaligned(z0) || misaligned(out_pts) ||
        misaligned(out_count) || (reinterpret_cast<uintptr_t>(fallback_count) & 7u))
        return SPHX_ERR_INVALID_ARG;
    launch_adaptive(A, B, z0, n, out_pts, out_count, gate_ulps, fallback_count,
                    reinterpret_cast<cudaStream_t>(stream));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return SPHX_ERR_CUDA;
    }
    return SPHX_OK;
}
