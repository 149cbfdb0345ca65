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
//
// The adaptive mode runs in two phases per tile: every thread first tries the
// filtered FP64 evaluation; the lanes it cannot vouch for append their tile
// index to a shared-memory queue (one atomic per warp), and after a barrier
// the block's first threads evaluate the queued arcs with the integer-limb
// form, densely, so that the accurate form's divergence is confined to the
// queue's last warp instead of every warp that holds one failing lane.
#pragma once
#include <algorithm>

#include "adaptive.cuh"
#include "common.cuh"
#include "intersect.cuh"

namespace sphx {

constexpr int kTile = 128;  // arcs per tile = threads per block
constexpr int kAdaptive = 5;

// The integer-limb mode asks for 7 resident blocks per SM (72 registers, a
// few bytes of spills): with its square root and reciprocal on the integer
// pipe it is bound by instruction issue, and the extra warps hide more of the
// carry chains' latency (1-1.5 % on GB300 against 6 blocks at 80 registers).
// The float-float mode shares its integer-limb core and asks for 6 (80
// registers, no spills, against 107 and 4 blocks unbounded).
template <int Mode>
__global__ void __launch_bounds__(kTile, Mode == kWideInt ? 7 : (Mode == kEftFf32 ? 6 : 1))
    dense_kernel(const double *__restrict__ A, const double *__restrict__ B,
                 const double *__restrict__ Z, int64_t n, double *__restrict__ out_pts,
                 int32_t *__restrict__ out_count, unsigned long long *fallback, double gate) {
    __shared__ __align__(16) double sA[3 * kTile];
    __shared__ __align__(16) double sB[3 * kTile];
    __shared__ __align__(16) double sZ[kTile];
    __shared__ __align__(16) double sP[6 * kTile];
    __shared__ __align__(16) int32_t sC[kTile];
    __shared__ int sQ[Mode == kAdaptive ? kTile : 1];
    __shared__ int sQn;
    const int t = threadIdx.x;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    auto stage_result = [&](int j, const PairOut &o, double z0) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            sP[6 * j + 3 * r + 0] = o.hit[r] ? o.px[r] : nan;
            sP[6 * j + 3 * r + 1] = o.hit[r] ? o.py[r] : nan;
            sP[6 * j + 3 * r + 2] = o.hit[r] ? z0 : nan;
        }
        sC[j] = o.count;
    };
    const int64_t ntiles = (n + kTile - 1) / kTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * kTile;
        const int cnt = (int)(n - base < kTile ? n - base : kTile);
        if (Mode == kAdaptive && t == 0) sQn = 0;
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
        if constexpr (Mode == kAdaptive) {
            bool pending = false;
            if (t < cnt) {
                const double x1[3] = {sA[3 * t], sA[3 * t + 1], sA[3 * t + 2]};
                const double x2[3] = {sB[3 * t], sB[3 * t + 1], sB[3 * t + 2]};
                PairOut o;
                if (filt::pair_filtered(x1, x2, sZ[t], gate, o))
                    stage_result(t, o, sZ[t]);
                else
                    pending = true;
            }
            const unsigned m = __ballot_sync(0xffffffffu, pending);
            if (m) {
                const int lane = t & 31, leader = __ffs(m) - 1;
                int at = 0;
                if (lane == leader) at = atomicAdd(&sQn, __popc(m));
                at = __shfl_sync(0xffffffffu, at, leader);
                if (pending) sQ[at + __popc(m & ((1u << lane) - 1u))] = t;
            }
            __syncthreads();
            const int qn = sQn;
            if (t < qn) {
                const int j = sQ[t];
                const double x1[3] = {sA[3 * j], sA[3 * j + 1], sA[3 * j + 2]};
                const double x2[3] = {sB[3 * j], sB[3 * j + 1], sB[3 * j + 2]};
                PairOut o;
                pair_wide(x1, x2, sZ[j], o);
                stage_result(j, o, sZ[j]);
            }
            if (fallback && t == 0 && qn) atomicAdd(fallback, (unsigned long long)qn);
        } else {
            if (t < cnt) {
                const double x1[3] = {sA[3 * t], sA[3 * t + 1], sA[3 * t + 2]};
                const double x2[3] = {sB[3 * t], sB[3 * t + 1], sB[3 * t + 2]};
                PairOut o;
                intersect_pair<Mode>(x1, x2, sZ[t], o);
                stage_result(t, o, sZ[t]);
            }
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

// ---- the dense kernel of every mode but the adaptive one ---------------------------
// As dense_kernel, with the next tile's endpoints and latitudes (7 KB) fetched
// into a second shared-memory buffer by 16-byte asynchronous copies while the
// current tile is evaluated, so the loads' latency is hidden behind the
// arithmetic. Measured on GB300 against dense_kernel, outputs identical
// (2x10^7 mixed arcs): integer limbs 1.816 -> 1.775 ms, float-float 1.517 ->
// 1.434, direct FP64 4.71 -> 4.59, FP64-EFT 17.32 -> 17.18. A warp-tiled form
// (tiles of 32 arcs per warp, no block barriers) was slower for the integer
// limbs (1.885 ms).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The float-float mode asks for 7 resident blocks per SM here too (72
// registers): 1.434 -> 1.413 ms per 2x10^7 mixed arcs against 6; the integer
// limbs measured 1.776 ms at 7, 1.781 at 8 and 1.792 at 6.
template <int Mode>
__global__ void __launch_bounds__(kTile, Mode == kWideInt || Mode == kEftFf32 ? 7 : 1)
    dense_pf_kernel(const double *__restrict__ A, const double *__restrict__ B,
                    const double *__restrict__ Z, int64_t n, double *__restrict__ out_pts,
                    int32_t *__restrict__ out_count) {
    __shared__ __align__(16) double sIn[2][7 * kTile];  // A (3 kTile), B (3 kTile), z0 (kTile)
    __shared__ __align__(16) double sP[6 * kTile];
    __shared__ __align__(16) int32_t sC[kTile];
    const int t = threadIdx.x;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const int64_t ntiles = (n + kTile - 1) / kTile;
    auto prefetch = [&](int64_t tile, int b) {
        if (tile < ntiles && n - tile * kTile >= kTile) {
            const char *ga = reinterpret_cast<const char *>(A + 3 * tile * kTile);
            const char *gb = reinterpret_cast<const char *>(B + 3 * tile * kTile);
            const char *gz = reinterpret_cast<const char *>(Z + tile * kTile);
            char *s = reinterpret_cast<char *>(sIn[b]);
            constexpr int CA = 3 * kTile * 8 / 16, CZ = kTile * 8 / 16;
            for (int i = t; i < 2 * CA + CZ; i += kTile) {
                if (i < CA)
                    cp_async16(s + 16 * i, ga + 16 * i);
                else if (i < 2 * CA)
                    cp_async16(s + 16 * i, gb + 16 * (i - CA));
                else
                    cp_async16(s + 16 * i, gz + 16 * (i - 2 * CA));
            }
        }
        cp_async_commit();
    };
    int b = 0;
    prefetch(blockIdx.x, 0);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, b ^= 1) {
        prefetch(tile + gridDim.x, b ^ 1);
        cp_async_wait<1>();
        const int64_t base = tile * kTile;
        const int cnt = (int)(n - base < kTile ? n - base : kTile);
        double *in = sIn[b];
        if (cnt < kTile) {
            for (int i = t; i < 3 * cnt; i += kTile) {
                in[i] = A[3 * base + i];
                in[3 * kTile + i] = B[3 * base + i];
            }
            if (t < cnt) in[6 * kTile + t] = Z[base + t];
        }
        __syncthreads();
        if (t < cnt) {
            const double x1[3] = {in[3 * t], in[3 * t + 1], in[3 * t + 2]};
            const double x2[3] = {in[3 * kTile + 3 * t], in[3 * kTile + 3 * t + 1],
                                  in[3 * kTile + 3 * t + 2]};
            const double z0 = in[6 * kTile + t];
            PairOut o;
            intersect_pair<Mode>(x1, x2, z0, o);
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
            if (t < kTile / 4)
                reinterpret_cast<int4 *>(out_count + base)[t] = reinterpret_cast<const int4 *>(sC)[t];
        } else {
            for (int i = t; i < 6 * cnt; i += kTile) out_pts[6 * base + i] = sP[i];
            if (t < cnt) out_count[base + t] = sC[t];
        }
    }
    cp_async_wait<0>();
}

static inline int sm_count_of_current() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// resident blocks per SM of the mode's dense kernel (its registers decide)
template <int Mode>
static int resident_blocks() {
    int b = 0;
    cudaError_t e;
    if constexpr (Mode == kAdaptive)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, dense_kernel<Mode>, kTile, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, dense_pf_kernel<Mode>, kTile, 0);
    if (e !=
            cudaSuccess ||
        b < 1) {
        cudaGetLastError();
        b = 4;
    }
    return b;
}

template <int Mode>
static void launch_dense(const double *A, const double *B, const double *Z, int64_t n,
                         double *P, int32_t *C, cudaStream_t s,
                         unsigned long long *fallback = nullptr, double gate_ulps = 4.0) {
    static const int sms = sm_count_of_current();
    static const int per_sm = resident_blocks<Mode>();
    const int64_t ntiles = (n + kTile - 1) / kTile;
    // one wave of resident blocks striding over the tiles (a second, partial
    // wave would leave most SMs idle while it finishes), or the multiple of
    // it that sphx_autotune_dense found fastest
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sms * per_sm * dense_waves(Mode));
    if constexpr (Mode == kAdaptive)
        dense_kernel<Mode><<<(unsigned)grid, kTile, 0, s>>>(A, B, Z, n, P, C, fallback,
                                                            0.975 * gate_ulps);
    else
        dense_pf_kernel<Mode><<<(unsigned)grid, kTile, 0, s>>>(A, B, Z, n, P, C);
}

// dense_kernel without the asynchronous prefetch, for arrays in page-locked
// host memory that the kernel reads in place (the host-buffer call): plain
// loads, as asynchronous copies are specified for device global memory
template <int Mode>
static void launch_dense_plain(const double *A, const double *B, const double *Z, int64_t n,
                               double *P, int32_t *C, cudaStream_t s) {
    static const int sms = sm_count_of_current();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_kernel<Mode>, kTile, 0) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 4;
    }
    const int64_t ntiles = (n + kTile - 1) / kTile;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
    dense_kernel<Mode><<<(unsigned)grid, kTile, 0, s>>>(A, B, Z, n, P, C, nullptr, 4.0);
}

// the adaptive mode's launcher (adaptive.cu)
void launch_adaptive(const double *A, const double *B, const double *Z, int64_t n, double *P,
                     int32_t *C, double gate_ulps, unsigned long long *fallback, cudaStream_t s);

}  // namespace sphx
