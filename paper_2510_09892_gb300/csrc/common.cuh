// Internal definitions shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sphx.h"

namespace sphx {

// device status word bits (OR-ed by kernels, read by sphx_sync_status)
enum : unsigned { kStatusCapacity = 1u, kStatusTimeout = 2u, kStatusScratch = 4u, kStatusInvalid = 8u };

// bound on the ordered compaction's look-back spin: each iteration is one L2
// read plus a 64 ns sleep (~0.5 us), so the wait gives up after about a second
constexpr long long kSpinLimit = 2000000;

void set_cuda_error(cudaError_t e);

#define SPHX_CUDA(call)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) {                         \
            ::sphx::set_cuda_error(e_);                  \
            return SPHX_ERR_CUDA;                        \
        }                                                \
    } while (0)

// launch shape of the ragged intersection kernel
struct RaggedShape {  // defaults: the fastest fused shape on both GB300 workloads
    int threads = 256;
    int blocks_per_sm = 4;
    int pairs_per_lane = 4;  // for the fused kernel: edges per thread and chunk
    int compaction = SPHX_COMPACT_AUTO;  // FUSED until autotuned
    int use_graph = 1;
    bool operator<(const RaggedShape &o) const {
        return std::tie(threads, blocks_per_sm, pairs_per_lane, compaction, use_graph) <
               std::tie(o.threads, o.blocks_per_sm, o.pairs_per_lane, o.compaction, o.use_graph);
    }
};

// scratch buffers of one ragged argument set
struct RaggedScratch {
    int32_t *lo = nullptr, *hi = nullptr;  // computed candidate ranges (E each)
    long long *offsets = nullptr;          // exclusive scan of hi - lo, E + 1
    long long *block_sums = nullptr;       // per scan block, nb + 1
    unsigned long long *ring = nullptr;    // look-back ring (ORDERED)
    unsigned long long *counters = nullptr;  // [0] chunk ticket, [1] output cursor
    int64_t E = -1, nb = 0, ring_slots = 0;
};

// argument block of the persistent ragged kernel
struct RaggedArgs {
    const double *A = nullptr, *B = nullptr, *lat_z = nullptr;
    const int32_t *lo = nullptr;
    const long long *offsets = nullptr;  // E + 1 entries: exclusive scan of candidate counts
    int64_t E = 0, L = 0;
    sphx_hit *out = nullptr;
    int64_t cap = 0;
    unsigned long long *out_total = nullptr;
    unsigned long long *counters = nullptr;  // [0] chunk ticket
    unsigned long long *ring = nullptr;      // look-back ring (ORDERED)
    int64_t ring_slots = 1;                  // power of two
    unsigned *status = nullptr;
    int hold_first = 0;            // failure injection (tests): chunk 0 never publishes its
                                   // prefix, so the look-back of chunk 1 waits out its limit
};

// argument block of the fused ragged kernel (fused.cu)
struct FusedArgs {
    const double *A = nullptr, *B = nullptr, *lat_z = nullptr;
    const int64_t *edge_offsets = nullptr, *lat_offsets = nullptr;
    const int32_t *lo_in = nullptr, *hi_in = nullptr;  // caller's ranges, or null
    int M = 0;
    int64_t E = 0, L = 0;
    sphx_hit *out = nullptr;
    int64_t cap = 0;
    unsigned long long *out_total = nullptr;
    unsigned long long *counters = nullptr;  // [0] chunk ticket
    unsigned *status = nullptr;
};

// exclusive scan of the candidate counts (ragged.cu): edges per scan block,
// and the number of blocks (each writes one block sum) for E edges
constexpr int kScanThreads = 256, kScanItems = 16;
constexpr int64_t kScanTile = int64_t(kScanThreads) * kScanItems;
constexpr int64_t scan_blocks_const(int64_t E) { return (E + kScanTile - 1) / kScanTile; }

// ragged.cu
int64_t scan_blocks_for(int64_t E);
cudaError_t launch_candidates(const double *A, const double *B, const int64_t *edge_offsets,
                              int M, int64_t E, const double *lat_z, int64_t L,
                              const int64_t *lat_offsets, int32_t *lo, int32_t *hi,
                              int sm_count, cudaStream_t s);
cudaError_t launch_scan(const int32_t *lo, const int32_t *hi, int64_t E, long long *block_sums,
                        long long *offsets, cudaStream_t s);
cudaError_t launch_ragged(int mode, const RaggedShape &sh, const RaggedArgs &a, int sm_count,
                          cudaStream_t s);
// dense.cu: the dense call on page-locked host arrays read in place
sphx_status dense_host_inplace(const double *A, const double *B, const double *z0, int64_t n,
                               double *out_pts, int32_t *out_count, sphx_mode mode,
                               cudaStream_t s);
// fused.cu
cudaError_t launch_fused(int mode, const RaggedShape &sh, const FusedArgs &a, int sm_count,
                         cudaStream_t s);

// Process-wide tuning cache (runtime.cu): launch shapes found by the
// autotuners, keyed by device name, call, mode and a size class, shared by
// every context of the process and, when SPHX_TUNE_CACHE names a file, kept
// there as JSON across processes.
struct TuneEntry {
    int threads = 0, blocks_per_sm = 0, pairs_per_lane = 0, compaction = 0, waves = 0;
    double ms = 0.0;
};
bool tune_lookup(const std::string &key, TuneEntry &e);
void tune_store(const std::string &key, const TuneEntry &e);
std::string tune_device_name();  // of the current device
// grid of the dense kernels: waves x one wave of resident blocks (default 1)
int dense_waves(int mode);
void set_dense_waves(int mode, int waves);

// device staging of the host-buffer dense call: kHostSlots chunks in flight,
// one stream each (copy in, kernel, copy out stay in order on a slot's
// stream). Each copy costs several microseconds of set-up, so the arcs go in
// as few chunks as keep both copy directions and the kernels overlapped: one
// per slot, up to kHostMaxChunk arcs each. Measured on GB300 with pageable
// buffers of 2x10^7 arcs: 3 x 2^19 arcs 30 GB/s, 6 x 2^20 78 GB/s, 4 x 2^21
// 152 GB/s (page-locked ones: 142 and 320 GB/s for the first and the last).
constexpr int kHostSlots = 4;
constexpr int64_t kHostMaxChunk = int64_t(1) << 21;  // arcs per chunk, at most
struct HostStaging {
    int64_t cap = 0;  // arcs per slot the buffers hold
    double *A[kHostSlots] = {}, *B[kHostSlots] = {}, *z[kHostSlots] = {}, *P[kHostSlots] = {};
    int32_t *C[kHostSlots] = {};
    cudaStream_t s[kHostSlots] = {};
    cudaEvent_t done[kHostSlots] = {};
    cudaEvent_t start = nullptr;
};

struct GraphKey {
    std::vector<uintptr_t> v;
    bool operator<(const GraphKey &o) const { return v < o.v; }
};

}  // namespace sphx

struct sphx_context {
    int device = 0;
    int sm_count = 0;
    unsigned *status = nullptr;  // device status word
    cudaStream_t capture_stream = nullptr;
    sphx::RaggedScratch scratch;
    bool tuned = false;          // tuning fixed by sphx_set_tuning / autotune
    sphx::RaggedShape shape;
    std::map<sphx::GraphKey, cudaGraphExec_t> graphs;
    sphx::HostStaging host;
    long long *band_block_sums = nullptr;  // band ranges' prefix sum: per scan block
    int32_t *band_lists = nullptr;         // band areas: the three cell lists (3 x band_faces)
    unsigned long long *band_counts = nullptr;  // their lengths
    int64_t band_faces = 0;                // cells these buffers serve
    unsigned long long *zonal_acc = nullptr;  // zonal sums: 4 words per band
    int64_t zonal_bands = 0;
    double *unit_nodes = nullptr;  // band areas: the mesh nodes normalised (3 x unit_node_cap)
    int64_t unit_node_cap = 0;
    std::mutex mu;
};

namespace sphx {
// runtime.cu: per-context scratch of the band-area calls (grown on demand)
sphx_status ensure_band_scratch(sphx_context *ctx, int64_t faces);
sphx_status ensure_zonal_scratch(sphx_context *ctx, int64_t bands);
sphx_status ensure_unit_nodes(sphx_context *ctx, int64_t nodes);
}  // namespace sphx
