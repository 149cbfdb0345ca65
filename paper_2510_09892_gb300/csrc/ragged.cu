// Ragged call: every edge of a mesh batch against every latitude of its mesh
// in the edge's z-range (steps a11 and a12 of the hot path, around the
// per-pair evaluation of intersect.cuh).
//
//  1. candidate_kernel  per edge: z-range of the arc (endpoint z's, and the
//                       apex +-|n_xy|/|n| when the arc passes it), widened
//                       (FP32 for unit endpoints, FP64 otherwise), then two
//                       binary searches into the mesh's sorted latitudes
//                       give [lo, hi).
//  2. scan_*            exclusive prefix sum of hi - lo over all edges
//                       (int64): pair p belongs to the edge e with
//                       offsets[e] <= p < offsets[e + 1].
//  3. ragged_kernel     persistent grid (a multiple of the SM count); each
//                       warp claims chunks of 32 * K consecutive pairs from a
//                       global ticket counter, evaluates them (lane l takes
//                       pairs l*K .. l*K + K - 1 of the chunk, so record order
//                       inside a chunk is pair order), counts its hits with a
//                       warp scan and obtains the chunk's output offset either
//                       with one atomicAdd (ATOMIC) or by a decoupled
//                       look-back over the preceding chunks (ORDERED: output in
//                       pair order, i.e. (edge, lat, root) order).
#include "common.cuh"
#include "intersect.cuh"
#include "ranges.cuh"

namespace sphx {

// ---- candidate ranges ---------------------------------------------------------
__global__ void candidate_kernel(const double *__restrict__ A, const double *__restrict__ B,
                                 const int64_t *__restrict__ edge_offsets, int M, int64_t E,
                                 const double *__restrict__ lat_z, int64_t L,
                                 const int64_t *__restrict__ lat_offsets,
                                 int32_t *__restrict__ lo_out, int32_t *__restrict__ hi_out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        // the warp's edges are consecutive and nearly always in one mesh: the
        // warp's first lane searches, the others step forward past at most the
        // few mesh boundaries inside the warp's 32 edges. The offsets live on
        // the device and are not validated by the host: clamp every index
        // derived from them into its buffer.
        const unsigned act = __activemask();
        const int first = __ffs(act) - 1;
        int m = 0;
        if ((threadIdx.x & 31) == first) m = (int)upper_bound_dev<int64_t>(edge_offsets, M + 1, e) - 1;
        m = __shfl_sync(act, m, first);
        m = m < 0 ? 0 : (m >= M ? M - 1 : m);
        for (int k = 0; k < 32 && m < M - 1 && edge_offsets[m + 1] <= e; ++k) ++m;
        int64_t ls = lat_offsets[m], le = lat_offsets[m + 1];
        ls = ls < 0 ? 0 : (ls > L ? L : ls);
        le = le < ls ? ls : (le > L ? L : le);
        const double x1[3] = {A[3 * e], A[3 * e + 1], A[3 * e + 2]};
        const double x2[3] = {B[3 * e], B[3 * e + 1], B[3 * e + 2]};
        int32_t lo = (int32_t)ls, hi = (int32_t)ls;
        double zmin, zmax;
        // the FP32 range fails for every non-finite endpoint (its unit-norm
        // test does), so only the FP64 one needs the finiteness check
        if (z_range_fp32(x1, x2, zmin, zmax) ||
            (finite_bits(x1[0]) && finite_bits(x1[1]) && finite_bits(x1[2]) &&
             finite_bits(x2[0]) && finite_bits(x2[1]) && finite_bits(x2[2]) &&
             z_range_fp64(x1, x2, zmin, zmax))) {
            const double *lz = lat_z + ls;
            const int64_t l = lower_bound_ord(lz, le - ls, ord64(zmin));
            lo = (int32_t)(ls + l);
            hi = (int32_t)(ls + upper_bound_ord_from(lz, le - ls, l, ord64(zmax)));
            if (hi < lo) hi = lo;
        }
        lo_out[e] = lo;
        hi_out[e] = hi;
    }
}

// ---- exclusive scan of (hi - lo) into int64 offsets[E + 1] ----------------------
// (kScanThreads, kScanItems and kScanTile are in common.cuh: the allocation-free
// call sizes its fixed block-sum area from them)

__device__ __forceinline__ long long count_of(const int32_t *lo, const int32_t *hi, int64_t e) {
    const int d = hi[e] - lo[e];
    return d > 0 ? d : 0;
}

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *warp_sums, T &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    total = warp_sums[nw - 1];
    T before = warp > 0 ? warp_sums[warp - 1] : T(0);
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_reduce(const int32_t *__restrict__ lo, const int32_t *__restrict__ hi, int64_t E,
                long long *__restrict__ block_sums) {
    __shared__ long long ws[32];
    const int64_t base = blockIdx.x * (int64_t)kScanTile;
    long long s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        const int64_t e = base + i;
        if (e < E) s += count_of(lo, hi, e);
    }
    long long total;
    block_exclusive_scan<long long>(s, ws, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// one block: exclusive scan of block_sums[0..nb) in place; total -> block_sums[nb], *tail
__global__ void __launch_bounds__(1024)
    scan_blocks(long long *__restrict__ block_sums, int64_t nb, long long *__restrict__ tail) {
    __shared__ long long ws[32];
    long long carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int64_t b = b0 + threadIdx.x;
        long long v = b < nb ? block_sums[b] : 0;
        long long total;
        long long ex = block_exclusive_scan<long long>(v, ws, total);
        if (b < nb) block_sums[b] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        block_sums[nb] = carry;
        *tail = carry;
    }
}

__global__ void __launch_bounds__(kScanThreads)
    scan_apply(const int32_t *__restrict__ lo, const int32_t *__restrict__ hi, int64_t E,
               const long long *__restrict__ block_sums, long long *__restrict__ offsets) {
    __shared__ long long ws[32];
    // the block's counts, then their exclusive scan; one pad slot per 16 so
    // that the per-thread runs of 16 fall in different banks
    __shared__ long long tile[kScanTile + kScanTile / 16];
    const int64_t base = blockIdx.x * (int64_t)kScanTile;
    // coalesced loads into shared memory ...
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int idx = i * kScanThreads + threadIdx.x;
        const int64_t e = base + idx;
        tile[idx + (idx >> 4)] = e < E ? count_of(lo, hi, e) : 0;
    }
    __syncthreads();
    // ... each thread scans its kScanItems consecutive counts ...
    long long c[kScanItems];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        c[i] = tile[threadIdx.x * (kScanItems + 1) + i];
        s += c[i];
    }
    long long total;
    long long ex = block_exclusive_scan<long long>(s, ws, total) + block_sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        tile[threadIdx.x * (kScanItems + 1) + i] = ex;
        ex += c[i];
    }
    __syncthreads();
    // ... and coalesced stores
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int idx = i * kScanThreads + threadIdx.x;
        const int64_t e = base + idx;
        if (e < E) offsets[e] = tile[idx + (idx >> 4)];
    }
}

// ---- persistent intersection + compaction ----------------------------------------
// look-back word: flag (2 bits) | tag (22 bits) | value (40 bits)
constexpr unsigned long long kFlagAgg = 1ull, kFlagInc = 2ull;
__device__ __forceinline__ unsigned long long lb_pack(unsigned long long flag,
                                                      unsigned long long tag,
                                                      unsigned long long v) {
    return (flag << 62) | ((tag & 0x3fffffull) << 40) | (v & 0xffffffffffull);
}



// first index i in [0, n) with a[i] > key (n if none), found by the whole
// warp: each round probes 32 evenly spaced positions at once and narrows the
// interval to one of the 32 gaps (a monotone array makes the probes <= key a
// prefix of the lanes), so a search over n entries takes log32(n) rounds of
// parallel loads instead of log2(n) dependent ones
__device__ __forceinline__ int64_t warp_upper_bound(const long long *a, int64_t n, long long key,
                                                    int lane) {
    int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t pos = lo + (int64_t)lane * step;
        const bool le = pos < hi && a[pos] <= key;
        const int c = __popc(__ballot_sync(0xffffffffu, le));
        if (c == 0) return lo;
        const int64_t nlo = lo + (int64_t)(c - 1) * step + 1;
        const int64_t nhi = lo + (int64_t)c * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    const int64_t pos = lo + lane;
    const bool le = pos < hi && a[pos] <= key;
    return lo + __popc(__ballot_sync(0xffffffffu, le));
}

template <int Mode, int K, bool Ordered>
__global__ void ragged_kernel(RaggedArgs a) {
    const int lane = threadIdx.x & 31;
    const long long T = a.offsets[a.E];
    constexpr int CH = 32 * K;
    const long long nchunks = (T + CH - 1) / CH;
    const int ring_bits = __ffsll(a.ring_slots) - 1;
    while (true) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(a.counters, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if ((long long)c >= nchunks) break;
        const long long p0 = (long long)c * CH;
        const long long p1 = min(p0 + CH, T);
        // edges of the first and last pair of the chunk (warp-cooperative searches)
        const long long e_first = warp_upper_bound(a.offsets, a.E + 1, p0, lane) - 1;
        const long long e_last =
            e_first + warp_upper_bound(a.offsets + e_first, a.E + 1 - e_first, p1 - 1, lane) - 1;
        PairOut res[K];
        long long edge[K];
        int32_t lat[K];
        int h = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const long long p = p0 + (long long)lane * K + j;
            res[j].count = 0;
            res[j].hit[0] = res[j].hit[1] = false;
            edge[j] = 0;
            lat[j] = 0;
            if (p < p1) {
                const long long e =
                    e_first + upper_bound_dev<long long>(a.offsets + e_first, e_last - e_first + 1, p) - 1;
                const long long k = a.lo[e] + (p - a.offsets[e]);
                edge[j] = e;
                lat[j] = (int32_t)k;
                if (k < 0 || k >= a.L) {
                    atomicOr(a.status, kStatusScratch);
                    continue;
                }
                const double x1[3] = {a.A[3 * e], a.A[3 * e + 1], a.A[3 * e + 2]};
                const double x2[3] = {a.B[3 * e], a.B[3 * e + 1], a.B[3 * e + 2]};
                intersect_pair<Mode>(x1, x2, a.lat_z[k], res[j]);
                h += (int)res[j].hit[0] + (int)res[j].hit[1];
            }
        }
        // warp scan of the hit counts
        int incl = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned long long total = (unsigned)__shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 0) {
            if (!Ordered) {
                base = total ? atomicAdd(a.out_total, total) : 0ull;
            } else {
                const unsigned long long mask = (unsigned long long)a.ring_slots - 1;
                const unsigned long long tag = c >> ring_bits;
                if (c == 0) {
                    if (!a.hold_first) atomicExch(a.ring, lb_pack(kFlagInc, 0, total));
                } else {
                    atomicExch(a.ring + (c & mask), lb_pack(kFlagAgg, tag, total));
                    unsigned long long run = 0;
                    long long j = (long long)c - 1;
                    long long spins = 0;
                    while (j >= 0) {
                        const unsigned long long w =
                            *reinterpret_cast<volatile unsigned long long *>(a.ring + (j & mask));
                        const unsigned long long f = w >> 62;
                        const unsigned long long wt = (w >> 40) & 0x3fffffull;
                        if (f != 0 && wt == (((unsigned long long)j >> ring_bits) & 0x3fffffull)) {
                            run += w & 0xffffffffffull;
                            if (f == kFlagInc) break;
                            --j;
                            continue;
                        }
                        if (++spins > kSpinLimit) {
                            atomicOr(a.status, kStatusTimeout);
                            break;
                        }
                        __nanosleep(64);
                    }
                    base = run;
                    atomicExch(a.ring + (c & mask), lb_pack(kFlagInc, tag, run + total));
                }
                if ((long long)c == nchunks - 1) *a.out_total = base + total;
            }
            if (base + total > (unsigned long long)a.cap) atomicOr(a.status, kStatusCapacity);
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        unsigned long long idx = base + (unsigned long long)(incl - h);
#pragma unroll
        for (int j = 0; j < K; ++j) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (res[j].hit[r]) {
                    if (idx < (unsigned long long)a.cap) {
                        sphx_hit rec;
                        rec.edge = edge[j];
                        rec.lat = lat[j];
                        rec.root = r;
                        rec.x = res[j].px[r];
                        rec.y = res[j].py[r];
                        a.out[idx] = rec;
                    }
                    ++idx;
                }
            }
        }
    }
}

// ---- host side -----------------------------------------------------------------
typedef void (*RaggedKernelFn)(RaggedArgs);

template <int Mode>
static RaggedKernelFn pick_k(int K, bool ordered) {
    if (ordered) {
        if (K == 1) return ragged_kernel<Mode, 1, true>;
        if (K == 2) return ragged_kernel<Mode, 2, true>;
        return ragged_kernel<Mode, 4, true>;
    }
    if (K == 1) return ragged_kernel<Mode, 1, false>;
    if (K == 2) return ragged_kernel<Mode, 2, false>;
    return ragged_kernel<Mode, 4, false>;
}

static RaggedKernelFn pick_kernel(int mode, int K, bool ordered) {
    switch (mode) {
        case kDirect: return pick_k<kDirect>(K, ordered);
        case kEftFp64: return pick_k<kEftFp64>(K, ordered);
        case kEftFf32: return pick_k<kEftFf32>(K, ordered);
        case kWideInt: return pick_k<kWideInt>(K, ordered);
        default: return pick_k<kEftFp64Printed>(K, ordered);
    }
}

int64_t scan_blocks_for(int64_t E) { return scan_blocks_const(E); }

cudaError_t launch_candidates(const double *A, const double *B, const int64_t *edge_offsets,
                              int M, int64_t E, const double *lat_z, int64_t L,
                              const int64_t *lat_offsets, int32_t *lo, int32_t *hi,
                              int sm_count, cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((E + 255) / 256, (int64_t)sm_count * 16);
    candidate_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, B, edge_offsets, M, E, lat_z, L,
                                                      lat_offsets, lo, hi);
    return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t *lo, const int32_t *hi, int64_t E, long long *block_sums,
                        long long *offsets, cudaStream_t s) {
    const int64_t nb = scan_blocks_for(E);
    scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(lo, hi, E, block_sums);
    scan_blocks<<<1, 1024, 0, s>>>(block_sums, nb, offsets + E);
    scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(lo, hi, E, block_sums, offsets);
    return cudaGetLastError();
}

cudaError_t launch_ragged(int mode, const RaggedShape &sh, const RaggedArgs &a, int sm_count,
                          cudaStream_t s) {
    RaggedKernelFn fn = pick_kernel(mode, sh.pairs_per_lane, sh.compaction == SPHX_COMPACT_ORDERED);
    const unsigned grid = (unsigned)(sm_count * sh.blocks_per_sm);
    fn<<<grid, sh.threads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sphx

using namespace sphx;

extern "C" sphx_status sphx_candidate_ranges(const double *A, const double *B,
                                             const int64_t *edge_offsets, int32_t M, int64_t E,
                                             const double *lat_z, const int64_t *lat_offsets,
                                             int64_t L, int32_t *lo, int32_t *hi,
                                             sphx_stream stream) {
    if (M < 1 || E < 0 || L < 0 || L > INT32_MAX) return SPHX_ERR_INVALID_ARG;
    if (E == 0) return SPHX_OK;
    if (!A || !B || !edge_offsets || !lat_z || !lat_offsets || !lo || !hi)
        return SPHX_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = launch_candidates(A, B, edge_offsets, M, E, lat_z, L, lat_offsets, lo, hi,
                                      sms > 0 ? sms : 1, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return SPHX_ERR_CUDA;
    }
    return SPHX_OK;
}
