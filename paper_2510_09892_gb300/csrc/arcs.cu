// Arc x arc call (sphx_intersect_gca_gca): pair i = arcs (A1[i], A2[i]) and
// (B1[i], B2[i]). Same structure as the dense latitude call: a block owns a
// tile of kArcTile consecutive pairs, the tile's four endpoint arrays are
// staged into shared memory with coalesced 16-byte loads, one thread
// evaluates one pair from registers, and the tile's points and counts go back
// through shared memory as coalesced 16-byte stores; the grid is one wave of
// resident blocks and strides over the tiles.
#include "arcs.cuh"
#include "common.cuh"

namespace sphx {

constexpr int kArcTile = 128;

// The integer-limb form asks for 5 resident blocks per SM (at most 96
// registers, a few bytes of spills) against the unbounded 119 registers and
// 4 blocks: measured on GB300, 0.1775 -> 0.161 ms per 10^6 pairs (6 blocks
// 0.162 with more spills, 7 blocks 0.171)
template <int Mode>
__global__ void __launch_bounds__(kArcTile, Mode == kWideInt ? 5 : 1)
    arcs_kernel(const double *__restrict__ A1, const double *__restrict__ A2,
                const double *__restrict__ B1, const double *__restrict__ B2, int64_t n,
                double *__restrict__ out_pts, int32_t *__restrict__ out_count) {
    __shared__ __align__(16) double s[4][3 * kArcTile];
    __shared__ __align__(16) double sP[6 * kArcTile];
    __shared__ __align__(16) int32_t sC[kArcTile];
    const int t = threadIdx.x;
    const double *in[4] = {A1, A2, B1, B2};
    const int64_t ntiles = (n + kArcTile - 1) / kArcTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * kArcTile;
        const int cnt = (int)(n - base < kArcTile ? n - base : kArcTile);
        if (cnt == kArcTile) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const double2 *src = reinterpret_cast<const double2 *>(in[a] + 3 * base);
                double2 *dst = reinterpret_cast<double2 *>(s[a]);
                for (int i = t; i < 3 * kArcTile / 2; i += kArcTile) dst[i] = __ldg(src + i);
            }
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a)
                for (int i = t; i < 3 * cnt; i += kArcTile) s[a][i] = in[a][3 * base + i];
        }
        __syncthreads();
        if (t < cnt) {
            const double a1[3] = {s[0][3 * t], s[0][3 * t + 1], s[0][3 * t + 2]};
            const double a2[3] = {s[1][3 * t], s[1][3 * t + 1], s[1][3 * t + 2]};
            const double b1[3] = {s[2][3 * t], s[2][3 * t + 1], s[2][3 * t + 2]};
            const double b2[3] = {s[3][3 * t], s[3][3 * t + 1], s[3][3 * t + 2]};
            ArcOut r;
            r.pz = 0.0;
            intersect_arcs<Mode>(a1, a2, b1, b2, r);
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const bool h = r.o.hit[k] && r.o.count > 0;
                sP[6 * t + 3 * k + 0] = h ? r.o.px[k] : nan;
                sP[6 * t + 3 * k + 1] = h ? r.o.py[k] : nan;
                sP[6 * t + 3 * k + 2] = h ? (k == 0 ? r.pz : -r.pz) : nan;
            }
            sC[t] = r.o.count;
        }
        __syncthreads();
        if (cnt == kArcTile) {
            double2 *P2 = reinterpret_cast<double2 *>(out_pts + 6 * base);
            const double2 *sP2 = reinterpret_cast<const double2 *>(sP);
            for (int i = t; i < 3 * kArcTile; i += kArcTile) P2[i] = sP2[i];
            int4 *C4 = reinterpret_cast<int4 *>(out_count + base);
            if (t < kArcTile / 4) C4[t] = reinterpret_cast<const int4 *>(sC)[t];
        } else {
            for (int i = t; i < 6 * cnt; i += kArcTile) out_pts[6 * base + i] = sP[i];
            if (t < cnt) out_count[base + t] = sC[t];
        }
        __syncthreads();
    }
}

template <int Mode>
static void launch_arcs(const double *A1, const double *A2, const double *B1, const double *B2,
                        int64_t n, double *P, int32_t *C, cudaStream_t s) {
    static int sms = 0, per_sm = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, arcs_kernel<Mode>, kArcTile,
                                                          0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 2;
        }
        if (sms < 1) sms = 1;
    }
    const int64_t ntiles = (n + kArcTile - 1) / kArcTile;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
    arcs_kernel<Mode><<<(unsigned)grid, kArcTile, 0, s>>>(A1, A2, B1, B2, n, P, C);
}

}  // namespace sphx

using namespace sphx;

extern "C" sphx_status sphx_intersect_gca_gca(const double *A1, const double *A2,
                                              const double *B1, const double *B2, int64_t n,
                                              double *out_pts, int32_t *out_count,
                                              sphx_mode mode, sphx_stream stream) {
    if (n < 0) return SPHX_ERR_INVALID_ARG;
    if (n == 0) return SPHX_OK;
    if (!A1 || !A2 || !B1 || !B2 || !out_pts || !out_count) return SPHX_ERR_INVALID_ARG;
    auto misaligned = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
    if (misaligned(A1) || misaligned(A2) || misaligned(B1) || misaligned(B2) ||
        misaligned(out_pts) || misaligned(out_count))
        return SPHX_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (mode) {
        case SPHX_MODE_DIRECT_FP64: launch_arcs<kDirect>(A1, A2, B1, B2, n, out_pts, out_count, s); break;
        case SPHX_MODE_EFT_FP64: launch_arcs<kEftFp64>(A1, A2, B1, B2, n, out_pts, out_count, s); break;
        case SPHX_MODE_WIDE_INT: launch_arcs<kWideInt>(A1, A2, B1, B2, n, out_pts, out_count, s); break;
        case SPHX_MODE_EFT_FF32:
        case SPHX_MODE_EFT_FP64_PRINTED:
        case SPHX_MODE_ADAPTIVE: return SPHX_ERR_UNSUPPORTED;
        default: return SPHX_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return SPHX_ERR_CUDA;
    }
    return SPHX_OK;
}
