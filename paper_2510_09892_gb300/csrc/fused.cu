// Ragged call in one persistent kernel (SPHX_COMPACT_FUSED): candidate
// latitudes, pair enumeration and the per-pair evaluation of Eq. 2.2 (steps
// a1, a11, a12 and a2-a10 of the hot path) without the intermediate ranges,
// prefix sum and their passes over HBM.
//
// Each block claims chunks of NT x EPT consecutive edges (EPT = 1, 2 or 4
// edges per thread) from a global ticket counter (dynamic load balance; edges with
// many candidates and edges with none cost what they cost). For a chunk:
//
//  1. the chunk's mesh: when all its edges lie in one mesh whose latitude grid
//     fits (kStageLats doubles, 23 KB), that grid is staged in shared memory as
//     order-preserving integer images, once per mesh change, and every
//     latitude search and latitude read below goes to shared memory; other
//     chunks read the grids in global memory;
//  2. per edge (EPT per thread): the edge's height range (FP32 for unit endpoints,
//     FP64 otherwise, widened) and two searches into its mesh's sorted
//     latitudes give the candidate indices [lo, hi) (or the caller's ranges);
//     on a staged grid the searches of a thread's edges run in lock step,
//     branch-free, so that their shared-memory reads overlap;
//  3. a block scan of the counts hi - lo numbers the chunk's (edge, latitude)
//     pairs; they are appended to a block-wide queue in shared memory
//     ({edge, latitude index, z0}), each thread locating its pair's edge by a
//     binary search of the scan;
//  4. whenever the queue holds NT pairs, every thread evaluates one of them
//     (intersect_pair, any mode) and the hits are compacted with one atomicAdd
//     per warp (record order unspecified). Pairs left in the queue carry over
//     to the next chunk; the last partial queue is evaluated at the end.
//
// So the evaluation, which is nearly all of the arithmetic, always runs on
// full warps, however sparse the candidates are among the edges (about one
// pair per five edges on a 0.09-degree cubed sphere against 0.25-degree
// latitudes, hundreds per edge for coarse meshes on fine grids).
#include "common.cuh"
#include "intersect.cuh"
#include "ranges.cuh"

namespace sphx {

constexpr int kStageLats = 2944;  // latitudes of one mesh staged in shared memory (23 KB)

// Searches in a staged grid, which holds the order-preserving integer images
// (ord64) of the latitudes: the same results as lower_bound_ord and
// upper_bound_ord_from on the doubles, without the per-probe conversion and
// with 32-bit indices.
__device__ __forceinline__ int lower_bound_s(const long long *a, int n, long long key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] >= key)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ int upper_bound_from_s(const long long *a, int n, int from,
                                                  long long key) {
    int lo = from, hi = from, step = 1;
    while (hi < n && a[hi] <= key) {
        lo = hi + 1;
        hi += step;
        step <<= 1;
    }
    if (hi > n) hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] > key)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// the double whose ord64 image is o (ord64 is its own inverse on the bits)
__device__ __forceinline__ double from_ord(long long o) {
    return __longlong_as_double(o < 0 ? (o ^ 0x7fffffffffffffffLL) : o);
}

template <int NT>
__device__ __forceinline__ long long block_inclusive_scan(long long v, long long *ws,
                                                          long long &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < NW ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) ws[lane] = w;
    }
    __syncthreads();
    total = ws[NW - 1];
    const long long before = warp > 0 ? ws[warp - 1] : 0;
    __syncthreads();  // ws is reused by the next scan
    return before + x;
}

// evaluate queue entries [0, n) (thread t takes entry t) and append the hits
template <int Mode>
__device__ __forceinline__ void eval_queue(const FusedArgs &a, int n, const long long *qe,
                                           const int *qk, const double *qz) {
    const int t = threadIdx.x, lane = t & 31;
    if ((t & ~31) >= n) return;  // the whole warp is past the queue's end
    PairOut res;
    res.hit[0] = res.hit[1] = false;
    long long e = 0;
    int k = 0;
    int h = 0;
    if (t < n) {
        e = qe[t];
        k = qk[t];
        const double z0 = qz[t];
        const double x1[3] = {a.A[3 * e], a.A[3 * e + 1], a.A[3 * e + 2]};
        const double x2[3] = {a.B[3 * e], a.B[3 * e + 1], a.B[3 * e + 2]};
        intersect_pair<Mode>(x1, x2, z0, res);
        h = (int)res.hit[0] + (int)res.hit[1];
    }
    int incl = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned long long total = (unsigned)__shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 0 && total) {
        base = atomicAdd(a.out_total, total);
        if (base + total > (unsigned long long)a.cap) atomicOr(a.status, kStatusCapacity);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    unsigned long long idx = base + (unsigned long long)(incl - h);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (res.hit[r]) {
            if (idx < (unsigned long long)a.cap) {
                sphx_hit rec;
                rec.edge = e;
                rec.lat = k;
                rec.root = r;
                rec.x = res.px[r];
                rec.y = res.py[r];
                a.out[idx] = rec;
            }
            ++idx;
        }
    }
}

// 7 resident blocks of 128 threads per SM (3 of 256): at most 72 (85)
// registers (a few bytes of spills in the integer-limb evaluation); measured
// on GB300 against the unbounded 96: 52.1 -> 49.2 ms on the 512-mesh batch,
// 0.71 -> 0.65 ms on the cubed sphere. Two edges per thread and chunk halve
// the barriers per edge: 45.7 -> 44.5 ms and 0.626 -> 0.562 ms (256 threads);
// four: 44.7 ms and 0.539 ms; with the searches of a thread's edges in lock
// step and the finiteness test after the FP32 range: 43.1 ms and 0.493 ms.
template <int Mode, int NT, int EPT>
__global__ void __launch_bounds__(NT, NT == 128 ? 7 : 3) fused_kernel(FusedArgs a) {
    constexpr int CH = NT * EPT;              // edges per chunk
    __shared__ long long s_ord[kStageLats];  // ord64 images of the staged latitudes
    __shared__ long long s_qe[NT];
    __shared__ int s_qk[NT];
    __shared__ double s_qz[NT];
    __shared__ long long s_incl[CH];  // inclusive prefix of pair counts, by slot t EPT + j
    __shared__ int s_lo[CH];
    __shared__ long long s_ws[32];
    __shared__ long long s_chunk;
    __shared__ int s_m0, s_single;
    __shared__ int s_staged;  // mesh whose grid s_ord holds (-1: none)

    const int t = threadIdx.x;
    const long long nchunks = (a.E + CH - 1) / CH;
    if (t == 0) s_staged = -1;
    int qn = 0;  // queue length (the same in every thread)
    while (true) {
        if (t == 0) {
            const long long c = (long long)atomicAdd(a.counters, 1ull);
            s_chunk = c;
            if (c < nchunks) {
                // the chunk's first mesh; it is the only one if the mesh
                // extends past the chunk's last edge (offsets are not
                // validated by the host: clamp what is derived from them)
                const long long e0 = c * CH;
                int m = (int)upper_bound_dev<int64_t>(a.edge_offsets, a.M + 1, e0) - 1;
                m = m < 0 ? 0 : (m >= a.M ? a.M - 1 : m);
                const long long e_last = min(e0 + CH, (long long)a.E) - 1;
                s_m0 = m;
                s_single = a.edge_offsets[m + 1] > e_last ? 1 : 0;
            }
        }
        __syncthreads();
        const long long c = s_chunk;
        if (c >= nchunks) break;
        const bool single = s_single != 0;
        // the chunk's grid, when all its edges are in one mesh
        const int m0 = s_m0;
        long long ls0 = a.lat_offsets[m0], le0 = a.lat_offsets[m0 + 1];
        ls0 = ls0 < 0 ? 0 : (ls0 > a.L ? a.L : ls0);
        le0 = le0 < ls0 ? ls0 : (le0 > a.L ? a.L : le0);
        const bool staged = single && le0 - ls0 <= kStageLats && !a.lo_in;
        if (staged && s_staged != m0) {
            __syncthreads();  // every thread has read s_staged
            for (long long i = t; i < le0 - ls0; i += NT) s_ord[i] = ord64(a.lat_z[ls0 + i]);
            if (t == 0) s_staged = m0;
            __syncthreads();
        }
        // candidate ranges of this thread's edges c CH + j NT + t (coalesced
        // across the block for each j), as absolute latitude indices
        int32_t lo[EPT], hi[EPT];
        long long own = 0;
        long long kl[EPT], kh[EPT];
        bool ok[EPT];
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const long long e = c * CH + j * NT + t;
            int m = m0;
            if (!single)
                while (m < a.M - 1 && a.edge_offsets[m + 1] <= e) ++m;
            long long ls = ls0, le = le0;
            if (!single) {
                ls = a.lat_offsets[m];
                le = a.lat_offsets[m + 1];
                ls = ls < 0 ? 0 : (ls > a.L ? a.L : ls);
                le = le < ls ? ls : (le > a.L ? a.L : le);
            }
            lo[j] = hi[j] = (int32_t)ls;
            ok[j] = false;
            kl[j] = kh[j] = 0;
            if (e < a.E) {
                if (a.lo_in) {
                    lo[j] = a.lo_in[e];
                    hi[j] = a.hi_in[e];
                } else {
                    const double x1[3] = {a.A[3 * e], a.A[3 * e + 1], a.A[3 * e + 2]};
                    const double x2[3] = {a.B[3 * e], a.B[3 * e + 1], a.B[3 * e + 2]};
                    double zmin, zmax;
                    // the FP32 range fails for every non-finite endpoint
                    // (its unit-norm test does), so only the FP64 one needs
                    // the finiteness check
                    ok[j] = z_range_fp32(x1, x2, zmin, zmax) ||
                            (finite_bits(x1[0]) && finite_bits(x1[1]) && finite_bits(x1[2]) &&
                             finite_bits(x2[0]) && finite_bits(x2[1]) && finite_bits(x2[2]) &&
                             z_range_fp64(x1, x2, zmin, zmax));
                    if (ok[j]) {
                        kl[j] = ord64(zmin);
                        kh[j] = ord64(zmax);
                        if (!staged) {
                            const double *lz = a.lat_z + ls;
                            const int64_t l = lower_bound_ord(lz, le - ls, kl[j]);
                            lo[j] = (int32_t)(ls + l);
                            hi[j] = (int32_t)(ls + upper_bound_ord_from(lz, le - ls, l, kh[j]));
                        }
                    }
                }
            }
        }
        if (staged && !a.lo_in) {
            // both searches of every edge of this thread in lock step over
            // the staged grid (one length for all: the chunk has one mesh),
            // so that their shared-memory reads overlap: a lower bound of
            // zmin and an upper bound of zmax, branch-free halving
            const int n = (int)(le0 - ls0);
            if (n > 0) {
                int bl[EPT], bh[EPT];
#pragma unroll
                for (int j = 0; j < EPT; ++j) bl[j] = bh[j] = 0;
                for (int len = n; len > 1;) {
                    const int half = len >> 1;
#pragma unroll
                    for (int j = 0; j < EPT; ++j) {
                        bl[j] = s_ord[bl[j] + half] < kl[j] ? bl[j] + half : bl[j];
                        bh[j] = s_ord[bh[j] + half] <= kh[j] ? bh[j] + half : bh[j];
                    }
                    len -= half;
                }
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    if (ok[j]) {
                        lo[j] = (int32_t)(ls0 + bl[j] + (s_ord[bl[j]] < kl[j] ? 1 : 0));
                        hi[j] = (int32_t)(ls0 + bh[j] + (s_ord[bh[j]] <= kh[j] ? 1 : 0));
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            if (hi[j] < lo[j]) hi[j] = lo[j];
            own += hi[j] > lo[j] ? (long long)(hi[j] - lo[j]) : 0;
        }
        long long total;
        long long run = block_inclusive_scan<NT>(own, s_ws, total) - own;
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            run += hi[j] > lo[j] ? (long long)(hi[j] - lo[j]) : 0;
            s_incl[t * EPT + j] = run;
            s_lo[t * EPT + j] = lo[j];
        }
        __syncthreads();
        // append the chunk's pairs to the queue, evaluating every full queue
        for (long long q = 0; q < total;) {
            const int take = (int)min((long long)(NT - qn), total - q);
            if (t < take) {
                const long long p = q + t;
                // the slot holding pair p: first i with s_incl[i] > p
                int i0 = 0, i1 = CH - 1;
                while (i0 < i1) {
                    const int mid = (i0 + i1) >> 1;
                    if (s_incl[mid] > p)
                        i1 = mid;
                    else
                        i0 = mid + 1;
                }
                const long long excl = i0 > 0 ? s_incl[i0 - 1] : 0;
                const long long k = (long long)s_lo[i0] + (p - excl);
                double z0 = 2.0;  // beyond the poles: no candidate
                int kk = (int)k;
                if (k < 0 || k >= a.L) {  // corrupt caller ranges: skip the pair
                    atomicOr(a.status, kStatusScratch);
                    kk = -1;
                } else {
                    z0 = staged ? from_ord(s_ord[k - ls0]) : a.lat_z[k];
                }
                s_qe[qn + t] = c * CH + (i0 % EPT) * NT + i0 / EPT;
                s_qk[qn + t] = kk;
                s_qz[qn + t] = z0;
            }
            qn += take;
            q += take;
            __syncthreads();
            if (qn == NT) {
                // entries whose latitude was out of range carry kk = -1 and
                // z0 = 2, a height beyond the poles: s^2 < 0, no hit
                eval_queue<Mode>(a, NT, s_qe, s_qk, s_qz);
                qn = 0;
                __syncthreads();
            }
        }
    }
    if (qn > 0) eval_queue<Mode>(a, qn, s_qe, s_qk, s_qz);
}

template <int Mode>
static cudaError_t launch_mode(int threads, int ept, const FusedArgs &a, unsigned grid,
                               cudaStream_t s) {
    if (threads == 128) {
        if (ept == 1)
            fused_kernel<Mode, 128, 1><<<grid, 128, 0, s>>>(a);
        else if (ept == 2)
            fused_kernel<Mode, 128, 2><<<grid, 128, 0, s>>>(a);
        else
            fused_kernel<Mode, 128, 4><<<grid, 128, 0, s>>>(a);
    } else {
        if (ept == 1)
            fused_kernel<Mode, 256, 1><<<grid, 256, 0, s>>>(a);
        else if (ept == 2)
            fused_kernel<Mode, 256, 2><<<grid, 256, 0, s>>>(a);
        else
            fused_kernel<Mode, 256, 4><<<grid, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// threads per block 128 or 256; edges per thread and chunk (the shape's
// pairs_per_lane field) 1, 2 or 4
cudaError_t launch_fused(int mode, const RaggedShape &sh, const FusedArgs &a, int sm_count,
                         cudaStream_t s) {
    const int threads = sh.threads <= 128 ? 128 : 256;
    const int ept = sh.pairs_per_lane >= 4 ? 4 : (sh.pairs_per_lane >= 2 ? 2 : 1);
    const unsigned grid = (unsigned)(sm_count * sh.blocks_per_sm);
    switch (mode) {
        case kDirect: return launch_mode<kDirect>(threads, ept, a, grid, s);
        case kEftFp64: return launch_mode<kEftFp64>(threads, ept, a, grid, s);
        case kEftFf32: return launch_mode<kEftFf32>(threads, ept, a, grid, s);
        case kWideInt: return launch_mode<kWideInt>(threads, ept, a, grid, s);
        default: return launch_mode<kEftFp64Printed>(threads, ept, a, grid, s);
    }
}

}  // namespace sphx
