// Band areas of spherical cells and zonal sums: the zonal-mean step that
// Sec. 1 names as the use of arc-latitude intersections.
//
//  1. band_range_kernel   one thread per cell: the height range of its arcs
//                         (ranges.cuh) and its winding number around the
//                         z-axis give the bands [lo, hi) it can meet; the
//                         ragged call's prefix sum turns the counts into
//                         output offsets.
//  2. band_partition_kernel sorts the cells into three lists, so that every
//     kernel below sees uniform warps:
//     fan_area_kernel     cells inside one band: the band area is the cell's
//                         own area, a fan of spherical triangles (Van
//                         Oosterom and Strackee's excess).
//     pair_area_kernel    cells cut by one latitude: the fan above its two
//                         crossings (Eq. 2.2) plus the sliver between the
//                         closing chord and the latitude arc; the part below
//                         is the cell's fan minus that.
//     band_area_kernel    every other cell, by the boundary integral. In
//                         longitude and height the area element is
//                         dlambda dz, so by Green's theorem a region's area is
//                         the boundary integral of lambda dz; the latitude
//                         pieces of the boundary of (cell ∩ band) have dz = 0.
//                         Each arc is cut at its crossings with the latitudes
//                         (Eq. 2.2 by the chosen mode), and each piece p -> q
//                         adds lambda_p (z_q - z_p) + dl z_q - T to the band
//                         holding its midpoint: dl is its longitude step and
//                         T = 2 atan(K h) the signed area between it and the
//                         equator, with h = tan(dl / 2) from the xy cross and
//                         dot products and K = (t_p + t_q) / (1 + t_p t_q),
//                         t = tan(latitude / 2). lambda is unwrapped along the
//                         cell from its first node off the poles; a cell
//                         around a pole adds 2 pi times each band's share of
//                         the height from that node to the pole (the cut
//                         across which lambda jumps by 2 pi). Crossings come
//                         in order along the arc without a sort: slot 0 of
//                         Eq. 2.2 crosses upwards along the arc and slot 1
//                         downwards, so a rising run takes the slot-0 hits of
//                         ascending latitudes and a falling run the slot-1
//                         hits of descending ones (an arc that passes its
//                         highest or lowest point is split there).
//  3. zonal_sum_kernel    per band, sum of field * area and of area, in
//                         128-bit fixed point with 64-bit integer atomics (per
//                         block in shared memory, then once per block in
//                         global memory), so the result does not depend on the
//                         order of the additions.
#include <cuda_runtime.h>

#include "areas.cuh"
#include "common.cuh"
#include "intersect.cuh"
#include "ranges.cuh"

namespace sphx {

constexpr int kAreaThreads = 128;
constexpr int64_t kSmemLat = 2048;  // latitudes (and their radii) staged in shared memory up to this count
constexpr int kZonalThreads = 256;
constexpr int64_t kSmemBands = 3072;  // bands accumulated in shared memory up to this count
__global__ void band_range_kernel(Mesh m, int32_t *__restrict__ band_lo,
                                  int32_t *__restrict__ band_hi) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < m.n_faces;
         f += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = 0;
        int64_t s, e;
        if (m.L >= 2 && cell_span(m, f, s, e) && e > s) {
            double zmin = 2.0, zmax = -2.0, wind = 0.0;
            bool ok = true, any = false;
            double a[3], b[3];
            ok = node_at(m, s, a);
            for (int64_t i = s; i < e && ok; ++i) {
                if (!(ok = node_at(m, i + 1 < e ? i + 1 : s, b))) break;
                double zl, zh;
                if (z_range_fp32(a, b, zl, zh) || z_range_fp64(a, b, zl, zh)) {
                    zmin = fmin(zmin, zl);
                    zmax = fmax(zmax, zh);
                    any = true;
                }
                // the winding number needs each step only to well within pi:
                // FP32; arcs from or to a pole step no longitude
                const float ax = (float)a[0], ay = (float)a[1], bx = (float)b[0], by = (float)b[1];
                if ((ax != 0.0f || ay != 0.0f) && (bx != 0.0f || by != 0.0f))
                    wind += (double)atan2f(ax * by - ay * bx, ax * bx + ay * by);
                a[0] = b[0];
                a[1] = b[1];
                a[2] = b[2];
            }
            if (ok && any) {
                const double w = rint(wind / kTwoPi);
                if (w >= 1.0) zmax = 1.0;
                if (w <= -1.0) zmin = -1.0;
                if (!(zmax < m.lat[0] || zmin > m.lat[m.L - 1])) {
                    int64_t klo = upper_bound_ord(m.lat, m.L, ord64(zmin)) - 1;
                    int64_t khi = upper_bound_ord_from(m.lat, m.L, klo + 1, ord64(zmax)) - 1;
                    klo = klo < 0 ? 0 : klo;
                    khi = khi > m.L - 2 ? m.L - 2 : khi;
                    if (khi >= klo) {
                        lo = (int32_t)klo;
                        hi = (int32_t)(khi + 1);
                    }
                }
            }
        }
        band_lo[f] = lo;
        band_hi[f] = hi;
    }
}

// Cells are split in three lists (warp-aggregated appends, so warps stay
// uniform): 0, cells that lie inside one band other than the first and the
// last (their widened height range does, so nothing was clamped), whose band
// area is the cell's own area; 2, cells in two such bands, cut by one
// latitude; 1, the others.
__global__ void band_partition_kernel(const int32_t *__restrict__ band_lo,
                                      const int32_t *__restrict__ band_hi, int64_t F, int64_t L,
                                      int32_t *__restrict__ lists, unsigned long long *counts) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; base < F;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = base + lane;
        int64_t klo = 0, nb = 0;
        if (f < F) {
            klo = band_lo[f];
            nb = (int64_t)band_hi[f] - klo;
        }
        const bool one = f < F && nb == 1 && klo > 0 && klo < L - 2;
        const bool two = f < F && nb == 2 && klo > 0 && klo + 1 < L - 2;
        const bool other = f < F && nb > 0 && !one && !two;
#pragma unroll
        for (int w = 0; w < 3; ++w) {
            const bool mine = w == 0 ? one : (w == 1 ? other : two);
            const unsigned bal = __ballot_sync(0xffffffffu, mine);
            if (!bal) continue;
            unsigned long long at = 0;
            if (lane == __ffs(bal) - 1) at = atomicAdd(counts + w, (unsigned long long)__popc(bal));
            at = __shfl_sync(0xffffffffu, at, __ffs(bal) - 1);
            if (mine) lists[w * F + (int64_t)at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)f;
        }
    }
}

// fan_area over the one-band list; a cell the fan does not take is appended
// to the other list, which band_area_kernel (launched after this kernel)
// works through
__global__ void __launch_bounds__(kAreaThreads, 8)
    fan_area_kernel(Mesh m, const long long *__restrict__ offsets, double *__restrict__ areas,
                    int64_t cap, int32_t *__restrict__ lists,
                    unsigned long long *__restrict__ counts) {
    const int64_t n = (int64_t)counts[0];
    const int lane = threadIdx.x & 31;
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + lane;
        bool far = false;
        int64_t f = -1;
        if (i < n) {
            f = lists[i];
            far = fan_area(m, f, offsets, areas, cap);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, far);
        if (bal) {
            unsigned long long at = 0;
            if (lane == __ffs(bal) - 1) at = atomicAdd(counts + 1, (unsigned long long)__popc(bal));
            at = __shfl_sync(0xffffffffu, at, __ffs(bal) - 1);
            if (far) lists[m.n_faces + (int64_t)at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)f;
        }
    }
}

// every node as a unit vector (unit(): the same arithmetic the area routines
// apply to a node when they read it), once per node instead of once per cell
// that uses the node
__global__ void unit_nodes_kernel(const double *__restrict__ nodes, int64_t n,
                                  double *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v[3] = {nodes[3 * i], nodes[3 * i + 1], nodes[3 * i + 2]};
        double u[3];
        unit(v, u);
        out[3 * i] = u[0];
        out[3 * i + 1] = u[1];
        out[3 * i + 2] = u[2];
    }
}

// pair_area over the two-band list; a cell it does not cover is appended to
// the other list (taken by band_area_kernel, launched after this kernel).
// Four resident blocks per SM (at most 128 registers, a few bytes of spills):
// its FP64 chains need the warps; measured on GB300 on the cubed sphere
// N = 1024, 3.23 -> 3.02 ms for the whole band-area call against the
// unbounded 146 registers (3 blocks); 5, 6 and 8 blocks gave the same 3.0 ms
template <int Mode>
__global__ void __launch_bounds__(kAreaThreads, 4)
    pair_area_kernel(Mesh m, const int32_t *__restrict__ band_lo,
                     const long long *__restrict__ offsets, double *__restrict__ areas, int64_t cap,
                     int32_t *__restrict__ lists, unsigned long long *__restrict__ counts) {
    extern __shared__ double s_lat[];
    const double *lat = m.lat;
    if (m.L <= kSmemLat) {
        for (int64_t i = threadIdx.x; i < m.L; i += blockDim.x) s_lat[i] = m.lat[i];
        __syncthreads();
        lat = s_lat;
    }
    const int64_t n = (int64_t)counts[2];
    const int lane = threadIdx.x & 31;
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + lane;
        bool back = false;
        int64_t f = -1;
        if (i < n) {
            f = lists[2 * m.n_faces + i];
            back = pair_area<Mode>(m, f, band_lo, offsets, areas, cap, lat);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, back);
        if (bal) {
            unsigned long long at = 0;
            if (lane == __ffs(bal) - 1) at = atomicAdd(counts + 1, (unsigned long long)__popc(bal));
            at = __shfl_sync(0xffffffffu, at, __ffs(bal) - 1);
            if (back) lists[m.n_faces + (int64_t)at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)f;
        }
    }
}

template <int Mode>
__global__ void __launch_bounds__(kAreaThreads, 3)
    band_area_kernel(Mesh m, const int32_t *__restrict__ band_lo,
                     const int32_t *__restrict__ band_hi, const long long *__restrict__ offsets,
                     double *__restrict__ areas, int64_t cap, const int32_t *__restrict__ list,
                     const unsigned long long *__restrict__ count) {
    extern __shared__ double s_lat[];  // L latitudes, then their radii
    const double *lat = m.lat, *rho_lat = nullptr;
    if (m.L <= kSmemLat) {
        for (int64_t i = threadIdx.x; i < m.L; i += blockDim.x) {
            const double z = m.lat[i];
            s_lat[i] = z;
            s_lat[m.L + i] = rho_of_lat(z);
        }
        __syncthreads();
        lat = s_lat;
        rho_lat = s_lat + m.L;
    }
    const int64_t n = (int64_t)*count;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        green_cell<Mode>(m, list[i], band_lo, band_hi, offsets, areas, cap, lat, rho_lat);
}

// ---- zonal sums in 128-bit fixed point (to_fixed, from_fixed: areas.cuh) ------------
// (hi, lo) += (vhi, vlo) modulo 2^128 with two 64-bit atomics: each wrap of
// the low word carries once into the high word, whatever the order
__device__ __forceinline__ void add128(unsigned long long *acc, unsigned long long vlo,
                                       unsigned long long vhi) {
    if (vlo == 0ull && vhi == 0ull) return;
    const unsigned long long old = atomicAdd(acc, vlo);
    const unsigned long long up = vhi + (old + vlo < old ? 1ull : 0ull);
    if (up) atomicAdd(acc + 1, up);
}


__global__ void __launch_bounds__(kZonalThreads)
    zonal_sum_kernel(const int32_t *__restrict__ band_lo, const int32_t *__restrict__ band_hi,
                     const long long *__restrict__ offsets, int64_t F,
                     const double *__restrict__ areas, const double *__restrict__ field,
                     int64_t n_bands, unsigned long long *__restrict__ acc, int use_smem,
                     unsigned *status) {
    extern __shared__ unsigned long long s_acc[];
    unsigned long long *tgt = acc;
    if (use_smem) {
        for (int64_t i = threadIdx.x; i < 4 * n_bands; i += blockDim.x) s_acc[i] = 0ull;
        __syncthreads();
        tgt = s_acc;
    }
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t klo = band_lo[f];
        const int64_t nb = (int64_t)band_hi[f] - klo;
        if (nb <= 0) continue;
        const long long off = offsets[f];
        const double fv = field[f];
        for (int64_t j = 0; j < nb; ++j) {
            const int64_t k = klo + j;
            if (k < 0 || k >= n_bands || off < 0) {
                atomicOr(status, kStatusInvalid);
                break;
            }
            const double A = areas[off + j];
            unsigned long long lo, hi;
            if (to_fixed(fv * A, lo, hi))
                add128(tgt + 4 * k, lo, hi);
            else
                atomicOr(status, kStatusInvalid);
            if (to_fixed(A, lo, hi))
                add128(tgt + 4 * k + 2, lo, hi);
            else
                atomicOr(status, kStatusInvalid);
        }
    }
    if (use_smem) {
        __syncthreads();
        for (int64_t i = threadIdx.x; i < 2 * n_bands; i += blockDim.x)
            add128(acc + 2 * i, s_acc[2 * i], s_acc[2 * i + 1]);
    }
}

__global__ void zonal_finish_kernel(const unsigned long long *__restrict__ acc, int64_t n_bands,
                                    double *__restrict__ out_fa, double *__restrict__ out_a) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_bands;
         k += (int64_t)gridDim.x * blockDim.x) {
        out_fa[k] = from_fixed(acc[4 * k], acc[4 * k + 1]);
        out_a[k] = from_fixed(acc[4 * k + 2], acc[4 * k + 3]);
    }
}

// ---- launchers -------------------------------------------------------------------
template <int Mode>
static cudaError_t launch_areas_mode(const Mesh &m, const int32_t *lo, const int32_t *hi,
                                     const long long *off, double *areas, int64_t cap,
                                     int32_t *lists, unsigned long long *counts, int sm_count,
                                     cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int64_t need = (m.n_faces + 255) / 256;
    band_partition_kernel<<<(unsigned)std::min<int64_t>(need, (int64_t)sm_count * 8), 256, 0, s>>>(
        lo, hi, m.n_faces, m.L, lists, counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fan_area_kernel, kAreaThreads, 0);
    if (e != cudaSuccess) return e;
    int64_t grid = std::min<int64_t>((m.n_faces + kAreaThreads - 1) / kAreaThreads,
                                     (int64_t)std::max(per_sm, 1) * sm_count);
    fan_area_kernel<<<(unsigned)grid, kAreaThreads, 0, s>>>(m, off, areas, cap, lists, counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem1 = m.L <= kSmemLat ? (size_t)m.L * sizeof(double) : 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_area_kernel<Mode>, kAreaThreads,
                                                      smem1);
    if (e != cudaSuccess) return e;
    grid = std::min<int64_t>((m.n_faces + kAreaThreads - 1) / kAreaThreads,
                             (int64_t)std::max(per_sm, 1) * sm_count);
    pair_area_kernel<Mode><<<(unsigned)grid, kAreaThreads, smem1, s>>>(m, lo, off, areas, cap, lists,
                                                                        counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = m.L <= kSmemLat ? 2 * (size_t)m.L * sizeof(double) : 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, band_area_kernel<Mode>, kAreaThreads,
                                                      smem);
    if (e != cudaSuccess) return e;
    grid = std::min<int64_t>((m.n_faces + kAreaThreads - 1) / kAreaThreads,
                             (int64_t)std::max(per_sm, 1) * sm_count);
    band_area_kernel<Mode><<<(unsigned)grid, kAreaThreads, smem, s>>>(
        m, lo, hi, off, areas, cap, lists + m.n_faces, counts + 1);
    return cudaGetLastError();
}

}  // namespace sphx

using namespace sphx;

namespace {

bool valid_mesh(sphx_context *ctx, const double *nodes, int64_t n_nodes,
                const int64_t *face_offsets, const int32_t *face_nodes, int64_t n_face_nodes,
                int64_t n_faces, const double *lat_z, int64_t n_lat) {
    // cells and nodes are indexed by int32 (node indices, the cell lists)
    return ctx && n_faces >= 0 && n_faces <= INT32_MAX && n_nodes >= 0 && n_nodes <= INT32_MAX &&
           n_face_nodes >= 0 && n_lat >= 2 && n_lat <= INT32_MAX &&
           (n_faces == 0 || (nodes && face_offsets && face_nodes)) && lat_z;
}

Mesh make_mesh(sphx_context *ctx, const double *nodes, int64_t n_nodes,
               const int64_t *face_offsets, const int32_t *face_nodes, int64_t n_face_nodes,
               int64_t n_faces, const double *lat_z, int64_t n_lat) {
    Mesh m;
    m.nodes = nodes;
    m.n_nodes = n_nodes;
    m.face_offsets = face_offsets;
    m.face_nodes = face_nodes;
    m.n_face_nodes = n_face_nodes;
    m.n_faces = n_faces;
    m.lat = lat_z;
    m.L = n_lat;
    m.status = ctx->status;
    return m;
}

}  // namespace

extern "C" sphx_status sphx_band_ranges(sphx_context *ctx, const double *nodes, int64_t n_nodes,
                                        const int64_t *face_offsets, const int32_t *face_nodes,
                                        int64_t n_face_nodes, int64_t n_faces,
                                        const double *lat_z, int64_t n_lat, int32_t *band_lo,
                                        int32_t *band_hi, int64_t *area_offsets,
                                        sphx_stream stream) {
    if (!valid_mesh(ctx, nodes, n_nodes, face_offsets, face_nodes, n_face_nodes, n_faces, lat_z,
                    n_lat) ||
        !area_offsets || (n_faces > 0 && (!band_lo || !band_hi)))
        return SPHX_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> g(ctx->mu);
    SPHX_CUDA(cudaSetDevice(ctx->device));
    if (n_faces == 0) {
        SPHX_CUDA(cudaMemsetAsync(area_offsets, 0, sizeof(int64_t), s));
        return SPHX_OK;
    }
    sphx_status st = ensure_band_scratch(ctx, n_faces);
    if (st != SPHX_OK) return st;
    const Mesh m =
        make_mesh(ctx, nodes, n_nodes, face_offsets, face_nodes, n_face_nodes, n_faces, lat_z, n_lat);
    const int64_t grid = std::min<int64_t>((n_faces + 255) / 256, (int64_t)ctx->sm_count * 8);
    band_range_kernel<<<(unsigned)grid, 256, 0, s>>>(m, band_lo, band_hi);
    SPHX_CUDA(cudaGetLastError());
    SPHX_CUDA(launch_scan(band_lo, band_hi, n_faces, ctx->band_block_sums,
                          reinterpret_cast<long long *>(area_offsets), s));
    return SPHX_OK;
}

extern "C" sphx_status sphx_band_areas(sphx_context *ctx, const double *nodes, int64_t n_nodes,
                                       const int64_t *face_offsets, const int32_t *face_nodes,
                                       int64_t n_face_nodes, int64_t n_faces,
                                       const double *lat_z, int64_t n_lat,
                                       const int32_t *band_lo, const int32_t *band_hi,
                                       const int64_t *area_offsets, sphx_mode mode,
                                       double *areas, int64_t areas_cap, sphx_stream stream) {
    if (!valid_mesh(ctx, nodes, n_nodes, face_offsets, face_nodes, n_face_nodes, n_faces, lat_z,
                    n_lat) ||
        areas_cap < 0 || (n_faces > 0 && (!band_lo || !band_hi || !area_offsets)) ||
        (areas_cap > 0 && !areas))
        return SPHX_ERR_INVALID_ARG;
    if (n_faces == 0) return SPHX_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> g(ctx->mu);
    SPHX_CUDA(cudaSetDevice(ctx->device));
    sphx_status st = ensure_band_scratch(ctx, n_faces);
    if (st != SPHX_OK) return st;
    if ((st = ensure_unit_nodes(ctx, n_nodes)) != SPHX_OK) return st;
    Mesh m =
        make_mesh(ctx, nodes, n_nodes, face_offsets, face_nodes, n_face_nodes, n_faces, lat_z, n_lat);
    if (n_nodes > 0) {
        const int64_t grid = std::min<int64_t>((n_nodes + 255) / 256, (int64_t)ctx->sm_count * 8);
        unit_nodes_kernel<<<(unsigned)grid, 256, 0, s>>>(nodes, n_nodes, ctx->unit_nodes);
        SPHX_CUDA(cudaGetLastError());
    }
    m.unit_nodes = ctx->unit_nodes;
    const long long *off = reinterpret_cast<const long long *>(area_offsets);
    cudaError_t e;
    switch (mode) {
        case SPHX_MODE_DIRECT_FP64:
            e = launch_areas_mode<kDirect>(m, band_lo, band_hi, off, areas, areas_cap, ctx->band_lists,
                                 ctx->band_counts, ctx->sm_count, s);
            break;
        case SPHX_MODE_EFT_FP64:
            e = launch_areas_mode<kEftFp64>(m, band_lo, band_hi, off, areas, areas_cap, ctx->band_lists,
                                 ctx->band_counts, ctx->sm_count, s);
            break;
        case SPHX_MODE_EFT_FF32:
            e = launch_areas_mode<kEftFf32>(m, band_lo, band_hi, off, areas, areas_cap, ctx->band_lists,
                                 ctx->band_counts, ctx->sm_count, s);
            break;
        case SPHX_MODE_EFT_FP64_PRINTED:
            e = launch_areas_mode<kEftFp64Printed>(m, band_lo, band_hi, off, areas, areas_cap, ctx->band_lists,
                                 ctx->band_counts, ctx->sm_count, s);
            break;
        case SPHX_MODE_WIDE_INT:
            e = launch_areas_mode<kWideInt>(m, band_lo, band_hi, off, areas, areas_cap, ctx->band_lists,
                                 ctx->band_counts, ctx->sm_count, s);
            break;
        case SPHX_MODE_ADAPTIVE:
            return SPHX_ERR_UNSUPPORTED;
        default:
            return SPHX_ERR_INVALID_ARG;
    }
    SPHX_CUDA(e);
    return SPHX_OK;
}

extern "C" sphx_status sphx_zonal_sums(sphx_context *ctx, const int32_t *band_lo,
                                       const int32_t *band_hi, const int64_t *area_offsets,
                                       int64_t n_faces, const double *areas, const double *field,
                                       int64_t n_lat, double *out_fa, double *out_a,
                                       sphx_stream stream) {
    if (!ctx || n_faces < 0 || n_lat < 2 || !out_fa || !out_a ||
        (n_faces > 0 && (!band_lo || !band_hi || !area_offsets || !areas || !field)))
        return SPHX_ERR_INVALID_ARG;
    const int64_t n_bands = n_lat - 1;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> g(ctx->mu);
    SPHX_CUDA(cudaSetDevice(ctx->device));
    sphx_status st = ensure_zonal_scratch(ctx, n_bands);
    if (st != SPHX_OK) return st;
    unsigned long long *acc = ctx->zonal_acc;
    SPHX_CUDA(cudaMemsetAsync(acc, 0, 4 * n_bands * sizeof(unsigned long long), s));
    if (n_faces > 0) {
        const int use_smem = n_bands <= kSmemBands ? 1 : 0;
        const size_t smem = use_smem ? (size_t)(4 * n_bands) * sizeof(unsigned long long) : 0;
        if (smem > 48 * 1024)
            SPHX_CUDA(cudaFuncSetAttribute(zonal_sum_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int64_t grid =
            std::min<int64_t>((n_faces + kZonalThreads - 1) / kZonalThreads, (int64_t)ctx->sm_count * 2);
        zonal_sum_kernel<<<(unsigned)grid, kZonalThreads, smem, s>>>(
            band_lo, band_hi, reinterpret_cast<const long long *>(area_offsets), n_faces, areas,
            field, n_bands, acc, use_smem, ctx->status);
        SPHX_CUDA(cudaGetLastError());
    }
    const int64_t g2 = std::min<int64_t>((n_bands + 255) / 256, 1024);
    zonal_finish_kernel<<<(unsigned)g2, 256, 0, s>>>(acc, n_bands, out_fa, out_a);
    SPHX_CUDA(cudaGetLastError());
    return SPHX_OK;
}
