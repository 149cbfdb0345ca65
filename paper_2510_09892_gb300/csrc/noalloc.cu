// Ragged call without any allocation (sphx_intersect_ragged_noalloc).
//
// Some callers must not allocate device memory on their call path: plugins
// whose host framework owns the device memory budget (a cudaMalloc behind its
// back can fail, or break its accounting), and latency-critical loops in which
// cudaMalloc's implicit device synchronisation is not acceptable. For them the
// scratch of the ragged sequence (candidate ranges, their prefix sum, scan
// block sums, the work counter and a status word) lives in one file-scope
// device array of fixed size, which every GPU that loads this library holds
// until the process exits. The kernels are the ones sphx_intersect_ragged
// launches, with unordered (atomic) compaction and the default launch shape.
//
// In host code the array's name only stands for the symbol: its device
// address is looked up with cudaGetSymbolAddress, once per device, with that
// device current, on the first call made on the device.
#include <mutex>

#include "common.cuh"

namespace sphx {
namespace {

constexpr int64_t kNoAllocMaxEdges = SPHX_NOALLOC_MAX_EDGES;
// the scan writes one block sum per scan_blocks_const(E) block (plus the
// total); its tile size is the one ragged.cu's scan kernels use (common.cuh)
constexpr int64_t kMaxScanBlocks = scan_blocks_const(kNoAllocMaxEdges);
static_assert(kMaxScanBlocks * kScanTile >= kNoAllocMaxEdges,
              "block-sum area too small for the largest accepted batch");

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// layout of the scratch array (byte offsets, each 256-byte aligned)
constexpr size_t kOffOffsets = 0;  // int64[E + 1]
constexpr size_t kOffBlockSums = align256(kOffOffsets + (kNoAllocMaxEdges + 1) * 8);  // int64[nb + 1]
constexpr size_t kOffCounters = align256(kOffBlockSums + (kMaxScanBlocks + 1) * 8);   // u64[4]
constexpr size_t kOffStatus = align256(kOffCounters + 4 * 8);                          // u32
constexpr size_t kOffLo = align256(kOffStatus + 4);                                    // int32[E]
constexpr size_t kOffHi = align256(kOffLo + kNoAllocMaxEdges * 4);                     // int32[E]
constexpr size_t kScratchBytes = align256(kOffHi + kNoAllocMaxEdges * 4);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_base[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// device address of the scratch array and the SM count, for the current device
sphx_status scratch_for_current(unsigned char **base, int *sms) {
    int dev = 0;
    SPHX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return SPHX_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        SPHX_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        int n = 0;
        SPHX_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        g_sms[dev] = n > 0 ? n : 1;
        g_base[dev] = static_cast<unsigned char *>(p);
    }
    *base = g_base[dev];
    *sms = g_sms[dev];
    return SPHX_OK;
}

}  // namespace
}  // namespace sphx

using namespace sphx;

extern "C" sphx_status sphx_intersect_ragged_noalloc(const double *A, const double *B,
                                                     const int64_t *edge_offsets, int32_t M,
                                                     int64_t E, const double *lat_z,
                                                     const int64_t *lat_offsets, int64_t L,
                                                     sphx_mode mode, sphx_hit *out,
                                                     int64_t out_cap, int64_t *out_total,
                                                     sphx_stream stream) {
    if (M < 1 || E < 0 || L < 0 || L > INT32_MAX || out_cap < 0) return SPHX_ERR_INVALID_ARG;
    if (E > kNoAllocMaxEdges) return SPHX_ERR_INVALID_ARG;  // beyond the fixed scratch
    if (mode == SPHX_MODE_ADAPTIVE) return SPHX_ERR_UNSUPPORTED;
    if ((int)mode < 0 || (int)mode > 4) return SPHX_ERR_INVALID_ARG;
    if (!out_total || (out_cap > 0 && !out)) return SPHX_ERR_INVALID_ARG;
    if (E > 0 && (!A || !B || !edge_offsets || !lat_z || !lat_offsets)) return SPHX_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(out) & 15u) || (reinterpret_cast<uintptr_t>(out_total) & 7u))
        return SPHX_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (E == 0) {
        SPHX_CUDA(cudaMemsetAsync(out_total, 0, sizeof(int64_t), s));
        return SPHX_OK;
    }
    unsigned char *base = nullptr;
    int sms = 1;
    sphx_status st = scratch_for_current(&base, &sms);
    if (st != SPHX_OK) return st;
    long long *offsets = reinterpret_cast<long long *>(base + kOffOffsets);
    long long *block_sums = reinterpret_cast<long long *>(base + kOffBlockSums);
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(base + kOffCounters);
    unsigned *status = reinterpret_cast<unsigned *>(base + kOffStatus);
    int32_t *lo = reinterpret_cast<int32_t *>(base + kOffLo);
    int32_t *hi = reinterpret_cast<int32_t *>(base + kOffHi);

    // the array keeps the previous call's contents: clear what must start at zero
    SPHX_CUDA(cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), s));
    SPHX_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), s));
    SPHX_CUDA(cudaMemsetAsync(out_total, 0, sizeof(int64_t), s));
    SPHX_CUDA(launch_candidates(A, B, edge_offsets, M, E, lat_z, L, lat_offsets, lo, hi, sms, s));
    SPHX_CUDA(launch_scan(lo, hi, E, block_sums, offsets, s));
    RaggedArgs a{};
    a.A = A;
    a.B = B;
    a.lat_z = lat_z;
    a.lo = lo;
    a.offsets = offsets;
    a.E = E;
    a.L = L;
    a.out = out;
    a.cap = out_cap;
    a.out_total = reinterpret_cast<unsigned long long *>(out_total);
    a.counters = counters;
    a.ring = nullptr;  // unordered compaction only
    a.ring_slots = 1;
    a.status = status;
    RaggedShape sh;
    sh.compaction = SPHX_COMPACT_ATOMIC;
    SPHX_CUDA(launch_ragged((int)mode, sh, a, sms, s));
    return SPHX_OK;
}

extern "C" sphx_status sphx_noalloc_sync_status(sphx_stream stream) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    SPHX_CUDA(cudaStreamSynchronize(s));
    unsigned char *base = nullptr;
    int sms = 1;
    sphx_status st = scratch_for_current(&base, &sms);
    if (st != SPHX_OK) return st;
    unsigned *status = reinterpret_cast<unsigned *>(base + kOffStatus);
    unsigned h = 0;
    SPHX_CUDA(cudaMemcpy(&h, status, sizeof h, cudaMemcpyDeviceToHost));
    SPHX_CUDA(cudaMemset(status, 0, sizeof h));
    if (h & (kStatusScratch | kStatusInvalid)) return SPHX_ERR_INVALID_ARG;
    if (h & kStatusCapacity) return SPHX_ERR_CAPACITY;
    return SPHX_OK;
}
