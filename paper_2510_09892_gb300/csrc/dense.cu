// Dense call: one latitude per arc (sphx_intersect_gca_constlat).
//
// One thread evaluates one arc (both roots). A block owns a tile of kTile
// consecutive arcs: the tile's endpoints (kTile x 3 doubles each, contiguous
// in the caller's row-major (n, 3) arrays) and latitudes are staged into
// shared memory with coalesced 16-byte loads, the per-thread work runs from
// registers, and the tile's results (kTile x 6 doubles, kTile counts) are
// staged back through shared memory and written with coalesced 16-byte
// stores. The grid is one wave of resident blocks (a multiple of the SM count)
// and strides over the tiles.
#include "common.cuh"
#include "intersect.cuh"

namespace sphx {

constexpr int kTile = 128;  // arcs per tile = threads per block

template <int Mode>
__global__ void __launch_bounds__(kTile) dense_kernel(const double *__restrict__ A,
                                                      const double *__restrict__ B,
                                                      const double *__restrict__ Z, int64_t n,
                                                      double *__restrict__ out_pts,
                                                      int32_t *__restrict__ out_count) {
    __shared__ __align__(16) double sA[3 * kTile];
    __shared__ __align__(16) double sB[3 * kTile];
    __shared__ __align__(16) double sZ[kTile];
    __shared__ __align__(16) double sP[6 * kTile];
    __shared__ __align__(16) int32_t sC[kTile];
    const int t = threadIdx.x;
    const int64_t ntiles = (n + kTile - 1) / kTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * kTile;
        const int cnt = (int)(n - base < kTile ? n - base : kTile);
        if (cnt == kTile) {
            // full tile: 16-byte loads (base is a multiple of kTile, so
            // 3 * base doubles is a multiple of 16 bytes)
            const double2 *A2 = reinterpret_cast<const double2 *>(A + 3 * base);
            const double2 *B2 = reinterpret_cast<const double2 *>(B + 3 * base);
            const double2 *Z2 = reinterpret_cast<const double2 *>(Z + base);
            double2 *sA2 = reinterpret_cast<double2 *>(sA);
            double2 *sB2 = reinterpret_cast<double2 *>(sB);
            double2 *sZ2 = reinterpret_cast<double2 *>(sZ);
            for (int i = t; i < 3 * kTile / 2; i += kTile) {
                sA2[i] = __ldg(A2 + i);
                sB2[i] = __ldg(B2 + i);
            }
            if (t < kTile / 2) sZ2[t] = __ldg(Z2 + t);
        } else {
            for (int i = t; i < 3 * cnt; i += kTile) {
                sA[i] = A[3 * base + i];
                sB[i] = B[3 * base + i];
            }
            if (t < cnt) sZ[t] = Z[base + t];
        }
        __syncthreads();
        if (t < cnt) {
            const double x1[3] = {sA[3 * t], sA[3 * t + 1], sA[3 * t + 2]};
            const double x2[3] = {sB[3 * t], sB[3 * t + 1], sB[3 * t + 2]};
            const double z0 = sZ[t];
            PairOut o;
            intersect_pair<Mode>(x1, x2, z0, o);
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                sP[6 * t + 3 * r + 0] = o.hit[r] ? o.px[r] : nan;
                sP[6 * t + 3 * r + 1] = o.hit[r] ? o.py[r] : nan;
                sP[6 * t + 3 * r + 2] = o.hit[r] ? z0 : nan;
            }
            sC[t] = o.count;
        }
        __syncthreads();
        if (cnt == kTile) {
            double2 *P2 = reinterpret_cast<double2 *>(out_pts + 6 * base);
            const double2 *sP2 = reinterpret_cast<const double2 *>(sP);
            for (int i = t; i < 3 * kTile; i += kTile) P2[i] = sP2[i];
            int4 *C4 = reinterpret_cast<int4 *>(out_count + base);
            if (t < kTile / 4) C4[t] = reinterpret_cast<const int4 *>(sC)[t];
        } else {
            for (int i = t; i < 6 * cnt; i += kTile) out_pts[6 * base + i] = sP[i];
            if (t < cnt) out_count[base + t] = sC[t];
        }
        __syncthreads();
    }
}

static int sm_count_of_current() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// resident blocks per SM of dense_kernel<Mode> (its registers decide)
template <int Mode>
static int resident_blocks() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, dense_kernel<Mode>, kTile, 0) !=
            cudaSuccess ||
        b < 1) {
        cudaGetLastError();
        b = 4;
    }
    return b;
}

template <int Mode>
static void launch_dense(const double *A, const double *B, const double *Z, int64_t n,
                         double *P, int32_t *C, cudaStream_t s) {
    static const int sms = sm_count_of_current();
    static const int per_sm = resident_blocks<Mode>();
    const int64_t ntiles = (n + kTile - 1) / kTile;
    // exactly one wave of resident blocks: a second, partial wave would leave
    // most SMs idle while it finishes
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
    dense_kernel<Mode><<<(unsigned)grid, kTile, 0, s>>>(A, B, Z, n, P, C);
}

}  // namespace sphx

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
