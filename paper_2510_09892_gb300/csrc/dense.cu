// Dense call entry points: the non-adaptive modes of dense_kernel (dense.cuh)
// and the App. A intermediates.
#include "dense.cuh"

using namespace sphx;

extern "C" sphx_status sphx_intersect_gca_constlat(const double *A, const double *B,
                                                   const double *z0, int64_t n, double *out_pts,
                                                   int32_t *out_count, sphx_mode mode,
                                                   sphx_stream stream) {
    if (n < 0) return SPHX_ERR_INVALID_ARG;
    if (n == 0) return SPHX_OK;
    if (!A || !B || !z0 || !out_pts || !out_count) return SPHX_ERR_INVALID_ARG;
    auto misaligned = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
    if (misaligned(A) || misaligned(B) || misaligned(z0) || misaligned(out_pts) ||
        misaligned(out_count))
        return SPHX_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (mode) {
        case SPHX_MODE_DIRECT_FP64: launch_dense<kDirect>(A, B, z0, n, out_pts, out_count, s); break;
        case SPHX_MODE_EFT_FP64: launch_dense<kEftFp64>(A, B, z0, n, out_pts, out_count, s); break;
        case SPHX_MODE_EFT_FF32: launch_dense<kEftFf32>(A, B, z0, n, out_pts, out_count, s); break;
        case SPHX_MODE_EFT_FP64_PRINTED:
            launch_dense<kEftFp64Printed>(A, B, z0, n, out_pts, out_count, s);
            break;
        case SPHX_MODE_WIDE_INT: launch_dense<kWideInt>(A, B, z0, n, out_pts, out_count, s); break;
        case SPHX_MODE_ADAPTIVE: launch_adaptive(A, B, z0, n, out_pts, out_count, 4.0, nullptr, s); break;
        default: return SPHX_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return SPHX_ERR_CUDA;
    }
    return SPHX_OK;
}

namespace sphx {
sphx_status dense_host_inplace(const double *A, const double *B, const double *z0, int64_t n,
                               double *out_pts, int32_t *out_count, sphx_mode mode,
                               cudaStream_t s) {
    switch (mode) {
        case SPHX_MODE_DIRECT_FP64: launch_dense_plain<kDirect>(A, B, z0, n, out_pts, out_count, s); break;
        case SPHX_MODE_EFT_FP64: launch_dense_plain<kEftFp64>(A, B, z0, n, out_pts, out_count, s); break;
        case SPHX_MODE_EFT_FF32: launch_dense_plain<kEftFf32>(A, B, z0, n, out_pts, out_count, s); break;
        case SPHX_MODE_EFT_FP64_PRINTED:
            launch_dense_plain<kEftFp64Printed>(A, B, z0, n, out_pts, out_count, s);
            break;
        case SPHX_MODE_WIDE_INT: launch_dense_plain<kWideInt>(A, B, z0, n, out_pts, out_count, s); break;
        case SPHX_MODE_ADAPTIVE: launch_adaptive(A, B, z0, n, out_pts, out_count, 4.0, nullptr, s); break;
        default: return SPHX_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return SPHX_ERR_CUDA;
    }
    return SPHX_OK;
}

__global__ void accux_mid_kernel(const double *__restrict__ A, const double *__restrict__ B,
                                 const double *__restrict__ Z, int64_t n, double *__restrict__ mid) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x1[3] = {A[3 * i], A[3 * i + 1], A[3 * i + 2]};
        const double x2[3] = {B[3 * i], B[3 * i + 1], B[3 * i + 2]};
        PairOut o;
        pair_accux<true>(x1, x2, Z[i], o, mid + 16 * i);
    }
}
}  // namespace sphx

extern "C" sphx_status sphx_accux_intermediates(const double *A, const double *B,
                                                const double *z0, int64_t n, double *out_mid,
                                                sphx_stream stream) {
    if (n < 0) return SPHX_ERR_INVALID_ARG;
    if (n == 0) return SPHX_OK;
    if (!A || !B || !z0 || !out_mid) return SPHX_ERR_INVALID_ARG;
    const int64_t blocks = std::min<int64_t>((n + 127) / 128, 152 * 16);
    accux_mid_kernel<<<(unsigned)blocks, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        A, B, z0, n, out_mid);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return SPHX_ERR_CUDA;
    }
    return SPHX_OK;
}

extern "C" sphx_status sphx_autotune_dense(const double *A, const double *B, const double *z0,
                                          int64_t n, double *out_pts, int32_t *out_count,
                                          sphx_mode mode, sphx_stream stream, double *ms_out) {
    if (n <= 0 || (int)mode < 0 || (int)mode > 5) return SPHX_ERR_INVALID_ARG;
    char keybuf[256];
    std::snprintf(keybuf, sizeof keybuf, "%s|dense|mode=%d|n=2^%d", tune_device_name().c_str(),
                  (int)mode, 63 - __builtin_clzll((unsigned long long)n));
    const std::string key(keybuf);
    TuneEntry hit;
    if (tune_lookup(key, hit)) {
        set_dense_waves((int)mode, hit.waves);
        if (ms_out) *ms_out = hit.ms;
        return SPHX_OK;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    SPHX_CUDA(cudaEventCreate(&e0));
    SPHX_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_w = 1;
    for (int w : {1, 2, 4, 8}) {
        set_dense_waves((int)mode, w);
        sphx_status st = sphx_intersect_gca_constlat(A, B, z0, n, out_pts, out_count, mode, stream);
        if (st != SPHX_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            set_dense_waves((int)mode, 1);
            return st;
        }
        float tot = 0.0f;
        for (int rep = 0; rep < 3; ++rep) {
            SPHX_CUDA(cudaEventRecord(e0, s));
            sphx_intersect_gca_constlat(A, B, z0, n, out_pts, out_count, mode, stream);
            SPHX_CUDA(cudaEventRecord(e1, s));
            SPHX_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            tot += ms;
        }
        if (tot / 3 < best) {
            best = tot / 3;
            best_w = w;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_dense_waves((int)mode, best_w);
    if (ms_out) *ms_out = best;
    TuneEntry te;
    te.waves = best_w;
    te.ms = best;
    tune_store(key, te);
    return SPHX_OK;
}
