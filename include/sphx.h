/*
 * sphx -- great-circle arc x constant-latitude intersection on the GPU.
 *
 * C ABI of libsphx.so. Every compute call is stream ordered and returns once
 * its work is enqueued; pointers are caller-owned device pointers unless a
 * comment says "host". Errors found before a launch come back as the return
 * value and nothing is launched; errors found on the device (output capacity,
 * a bounded wait that ran out) are recorded in the context's device status
 * word and reported by sphx_sync_status().
 *
 * The problem (Sec. 1.2 of Chen, Ullrich, Panetta, "Fast and Accurate
 * Intersections on a Sphere", arXiv 2510.09892): an arc is the shorter great
 * circle arc between two FP64 points x1, x2 (not necessarily of unit norm:
 * the formula only uses the direction of n = x1 x x2); a latitude is the plane
 * z = z0. The candidate points are Eq. 2.2,
 *   P = ( -(z0 nx nz +- s ny) / |n_xy|^2, -(z0 ny nz -+ s nx) / |n_xy|^2, z0 ),
 *   s = sqrt(|n_xy|^2 - |n|^2 z0^2),
 * they exist iff |n_xy|^2 >= |n|^2 z0^2 (two when strict, Sec. 2), and a
 * candidate is a hit iff it lies on the arc, decided as (x1 x P).n >= 0 and
 * (P x x2).n >= 0 (Sec. 2 only asks for the point to lie between the endpoints).
 * Root slot 0 is the upper sign (the alpha* <= 0 root that Algorithm 8,
 * AccuX, returns); slot 1 the lower sign. A tangent point (s = 0) is one hit
 * in slot 0.
 */
#ifndef SPHX_H
#define SPHX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* a cudaStream_t (NULL = the legacy default stream) */
typedef struct CUstream_st *sphx_stream;

typedef enum {
    SPHX_OK = 0,
    SPHX_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or enum: nothing launched */
    SPHX_ERR_CUDA = 2,        /* a CUDA runtime call failed (see sphx_last_cuda_error) */
    SPHX_ERR_CAPACITY = 3,    /* ragged output needed more records than out_cap */
    SPHX_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    SPHX_ERR_NOMEM = 5,       /* scratch allocation failed */
    SPHX_ERR_UNSUPPORTED = 6  /* no sm_103a device, or a feature not built */
} sphx_status;

/* How the candidate points are evaluated. */
typedef enum {
    /* Eq. 2.2 translated directly into FP64 (Sec. 4): plain cross product,
       sums of squares, sqrt and two divisions, no FMA contraction. */
    SPHX_MODE_DIRECT_FP64 = 0,
    /* AccuX (Algorithm 8) in FP64 with error-free transformations, both
       roots, each AccuDOP pair renormalised by one TwoSum so that the
       compensation terms stay below u times their leading parts (needed by
       SumOfSquaresC for arcs much shorter than 1e-8 rad or nearly antipodal).
       Error <= 4 ulp per component of the correctly rounded exact point. */
    SPHX_MODE_EFT_FP64 = 1,
    /* Float-float tail on an exact core (the paper has no such variant; its
       Sec. 9 names reduced precision as future work): the steps whose
       cancellation the error analysis of Sec. 4 and 6.1 is about -- the
       cross product of nearly coincident or antipodal endpoints (exact),
       |n_xy|^2, |n|^2 and s^2 (128-bit) -- run on 32-bit integer limbs as in
       SPHX_MODE_WIDE_INT; the square root, 1 / |n_xy|^2 and the point
       Eq. 2.2 in float-float (pairs of FP32, TwoSum / FMA TwoProd) on the
       FP32 pipe; the on-arc test as in SPHX_MODE_WIDE_INT. Error
       |P~ - P| <= 2^-44 sqrt(1 - z0^2) for every arc (near tangency and the
       poles included), hit counts those of the exact core. */
    SPHX_MODE_EFT_FF32 = 2,
    /* Algorithm 8 exactly as printed (no renormalisation after AccuDOP), for
       comparison; loses accuracy on very short and near-antipodal arcs. */
    SPHX_MODE_EFT_FP64_PRINTED = 3,
    /* Eq. 2.2 in software floating point with 32-bit integer limbs: n from
       exact products of the inputs, |n_xy|^2, |n|^2 and s^2 with 128-bit
       mantissas (the cancelling steps of Sec. 4 and 6.1), the square root,
       numerators and the division by |n_xy|^2 with 96-bit mantissas; the
       on-arc test in FP32 on offsets from the endpoints. Same bound as
       SPHX_MODE_EFT_FP64 (<= 4 ulp per component of the correctly rounded
       exact point), computed on the integer pipe, which GB300 runs 32 times
       faster than its FP64 pipe. */
    SPHX_MODE_WIDE_INT = 4,
    /* The adaptive filter (Sec. 9): Eq. 2.2 in plain FP64 (FMA cross
       products, one correctly rounded sqrt and division per coordinate) with
       a running forward error bound. A lane is kept when the bound proves its
       hit count (sign of s^2, both on-arc signs) and every point component
       within the 4-ulp gate (4 ulp of the correctly rounded value where
       |P_c| >= 2^-20 sqrt(1 - z0^2), 4 u sqrt(1 - z0^2) absolute below);
       otherwise the lane is re-evaluated as in SPHX_MODE_WIDE_INT (tangency,
       near-endpoint and degenerate arcs, inputs outside [2^-100, 2^100]).
       Every result therefore meets the SPHX_MODE_EFT_FP64 bound. Dense and
       host-buffer calls only (the others return SPHX_ERR_UNSUPPORTED). */
    SPHX_MODE_ADAPTIVE = 5
} sphx_mode;

/* Output compaction scheme of the ragged call. */
typedef enum {
    SPHX_COMPACT_AUTO = 0,    /* autotuned choice among FUSED and ATOMIC, else FUSED */
    SPHX_COMPACT_ATOMIC = 1,  /* one atomicAdd per warp: record order unspecified */
    SPHX_COMPACT_ORDERED = 2, /* decoupled look-back: records in (edge, lat, root) order */
    SPHX_COMPACT_FUSED = 3    /* one persistent kernel: candidate ranges, pair queue in shared
                                 memory, evaluation and one atomicAdd per warp; no range, prefix
                                 sum or scratch passes over HBM; record order unspecified */
} sphx_compaction;

typedef struct sphx_context sphx_context;

/* One compacted hit of the ragged call: 32 bytes. */
typedef struct {
    int64_t edge; /* global edge index into A, B */
    int32_t lat;  /* index into the concatenated lat_z array */
    int32_t root; /* 0 or 1: root slot of Eq. 2.2 as above */
    double x, y;  /* P_x, P_y; P_z is lat_z[lat] */
} sphx_hit;

/* Launch-shape overrides for the ragged path (0 = autotuned / default). */
typedef struct {
    int32_t threads_per_block; /* 64..1024, multiple of 32 */
    int32_t blocks_per_sm;     /* persistent grid = blocks_per_sm x SM count */
    int32_t pairs_per_lane;    /* ATOMIC, ORDERED: candidate pairs a lane takes per claimed
                                  chunk (1, 2, 4); FUSED: edges per thread per chunk (1, 2, 4) */
    int32_t compaction;        /* sphx_compaction */
    int32_t use_graph;         /* 1: capture the ragged launch sequence in a CUDA graph */
} sphx_tuning;

/* Create a context on `device` (made current). The context owns the scratch
   of the ragged call, its device status word, the tuning cache and the CUDA
   graphs. Returns SPHX_ERR_UNSUPPORTED if the device is not compute 10.3. */
sphx_status sphx_create(sphx_context **ctx, int device);
void sphx_destroy(sphx_context *ctx);

/* Dense call: arc i = (A[i], B[i]) against latitude z0[i], i < n.
   A, B: device, n x 3 row-major FP64 (a torch (n, 3) tensor), 16-byte aligned.
   z0: device, n FP64. out_pts: device, n x 2 x 3 FP64, slot r of arc i at
   out_pts[6i + 3r .. 6i + 3r + 2]; slots without a hit are NaN.
   out_count: device, n int32: number of hits 0..2, or -1 when the arc is
   degenerate (computed n = 0) or lies on the equator with z0 = 0 (coincident
   circles). Non-finite inputs give count 0. n = 0 is a no-op.
   Allocates nothing; safe to capture in a CUDA graph. */
sphx_status sphx_intersect_gca_constlat(const double *A, const double *B, const double *z0,
                                        int64_t n, double *out_pts, int32_t *out_count,
                                        sphx_mode mode, sphx_stream stream);

/* The adaptive mode with a caller's gate and its statistics: as
   sphx_intersect_gca_constlat with mode SPHX_MODE_ADAPTIVE, except that the
   filter keeps a lane when its bound proves each point component within
   gate_ulps ulp (gate_ulps u sqrt(1 - z0^2) for components below
   2^-20 sqrt(1 - z0^2)); 4 is the mode's own gate. gate_ulps in [1, 2^26],
   else SPHX_ERR_INVALID_ARG. Re-evaluated lanes are correctly rounded from
   96 bits whatever the gate. Atomically adds to *fallback_count (device
   uint64, 8-byte aligned, may be NULL) the number of arcs the filter handed
   to the integer-limb form. Stream ordered; allocates nothing. */
sphx_status sphx_intersect_gca_constlat_adaptive(const double *A, const double *B,
                                                 const double *z0, int64_t n, double *out_pts,
                                                 int32_t *out_count, double gate_ulps,
                                                 unsigned long long *fallback_count,
                                                 sphx_stream stream);

/* Dense call on HOST buffers (same problem and layouts as
   sphx_intersect_gca_constlat; A, B, z0, out_pts, out_count are host
   pointers, best page-locked). When all five are page-locked memory the device
   maps (unified addressing; over NVLink-C2C on GB300), the kernel reads and
   writes them in place, with no staging copies. Otherwise the arcs go through
   the context's device staging in four chunks (of at most 2097152 arcs; more
   chunks beyond that), each on its own stream of the context, so that the
   copies in both directions overlap the kernels. The staging (108 B per arc of a chunk, per
   stream) is allocated when a call needs more than the last and kept.
   The work starts after the work already enqueued on `stream` but does not
   hold `stream` back: successive calls on one context overlap (one call's
   results going out while the next call's inputs come in). The host outputs
   are complete once sphx_host_join(ctx, stream) has been enqueued and
   `stream` has synchronised. Returns after enqueuing. The host buffers must
   stay valid until then. Calls on one context must come from one host thread
   at a time. */
sphx_status sphx_intersect_gca_constlat_host(sphx_context *ctx, const double *A, const double *B,
                                             const double *z0, int64_t n, double *out_pts,
                                             int32_t *out_count, sphx_mode mode,
                                             sphx_stream stream);

/* Make `stream` wait for every sphx_intersect_gca_constlat_host call
   enqueued on `ctx` so far (their copies out included). Returns after
   enqueuing. */
sphx_status sphx_host_join(sphx_context *ctx, sphx_stream stream);

/* Intersection of two great circle arcs, pair i = (A1[i], A2[i]) and
   (B1[i], B2[i]): three cross products followed by a normalisation (Sec. 1)
   (Sec. 9 names it as a use of the accurate cross product). The circles meet
   at +-v / |v|, v = (a1 x a2) x (b1 x b2); a point is a hit iff it lies on
   both closed minor arcs, decided as in the latitude call. A1, A2, B1, B2:
   device, n x 3 row-major FP64, 16-byte aligned. out_pts: device,
   n x 2 x 3 FP64: slot 0 holds +v / |v|, slot 1 -v / |v|, NaN without a hit.
   out_count: device, n int32: 0 or 1 (2 only for arcs meeting at both
   antipodes' boundaries), -1 when an arc's normal is 0 or both arcs lie on
   one great circle; non-finite inputs give 0. mode: SPHX_MODE_WIDE_INT
   (integer limbs: the normals exact, v and |v|^2 with 128-bit mantissas,
   v / |v| rounded to nearest from 96 bits), SPHX_MODE_EFT_FP64 (renormalised
   AccuDOP normals, each v_i one compensated 6-term dot product, FP64
   normalisation) or SPHX_MODE_DIRECT_FP64; the others return
   SPHX_ERR_UNSUPPORTED. Allocates nothing; stream ordered. */
sphx_status sphx_intersect_gca_gca(const double *A1, const double *A2, const double *B1,
                                   const double *B2, int64_t n, double *out_pts,
                                   int32_t *out_count, sphx_mode mode, sphx_stream stream);

/* The intermediate pairs of Algorithm 8 (SPHX_MODE_EFT_FP64), for the
   error analysis of App. A: for arc i, 16 doubles at out_mid[16 i]:
   n[3] and their compensation terms en[3] (AccuDOP), S2, s2 (|n_xy|^2 as a
   pair), S3, s3 (|n|^2), ss, ess (s^2), sb, es (AccSqrt), X (root 0's
   x-coordinate numerator, P_x = -X / S2), 0. Quantities past the point where
   an arc stops (degenerate, no candidate) are 0. Device pointers, layouts as
   in sphx_intersect_gca_constlat; stream ordered. */
sphx_status sphx_accux_intermediates(const double *A, const double *B, const double *z0,
                                     int64_t n, double *out_mid, sphx_stream stream);

/* Candidate latitude ranges of a ragged batch (step a11 of the hot path):
   for each edge e of mesh m, [lo[e], hi[e]) indexes lat_z (global indices)
   and covers every latitude of mesh m inside the edge's z-range (the endpoint
   z's and, when the arc passes it, the arc's apex |n_xy| / |n|, Sec. 2),
   widened so that no hit is lost to rounding: by 2^-19 when both endpoints
   have unit norm (the range is then computed in FP32, whose error stays three
   times below the widening; for endpoints at most 2^-9 apart from their
   heights alone, since such an arc rises at most its sagitta, 0.31 |x2 - x1|^2,
   above them), by 1e-13 otherwise (FP64). lat_z must be sorted
   ascending within each mesh. Sizes as in sphx_intersect_ragged.
   lo, hi: device int32[E]. */
sphx_status sphx_candidate_ranges(const double *A, const double *B, const int64_t *edge_offsets,
                                  int32_t M, int64_t E, const double *lat_z,
                                  const int64_t *lat_offsets, int64_t L, int32_t *lo,
                                  int32_t *hi, sphx_stream stream);

/* Ragged call: M meshes; mesh m owns edges [edge_offsets[m], edge_offsets[m+1])
   of A, B (device, E x 3 FP64) and latitudes [lat_offsets[m], lat_offsets[m+1])
   of lat_z (device, L FP64, ascending within each mesh). edge_offsets and
   lat_offsets are device int64[M + 1] starting at 0 and ending at E and L.
   Every edge is tested against every latitude of its mesh in its z-range:
   edge_lat_lo / edge_lat_hi (device int32[E], global latitude indices) give
   those ranges, or both NULL to compute them (sphx_candidate_ranges).
   Hits are written as sphx_hit records to out (device, out_cap records);
   *out_total (device int64) receives the number of hits. If it exceeds
   out_cap, only out_cap records are written and sphx_sync_status() reports
   SPHX_ERR_CAPACITY. Degenerate pairs (count -1 in the dense call) give no
   record. Scratch comes from the context (allocated on the first call for a
   given size, then reused); the launch sequence is captured in a CUDA graph
   on the first call with a given argument set and replayed afterwards.
   Calls on one context must not overlap in time. The ordered compaction's
   look-back waits at most about 2e6 sleeps of 64 ns per chunk; one that runs
   out records SPHX_ERR_TIMEOUT (the records are then incomplete) and the
   call still ends. Failure injection for tests, read from the environment on
   each call: SPHX_FAULT=alloc makes a scratch allocation fail (ERR_NOMEM),
   SPHX_FAULT=lookback makes the first chunk withhold its prefix so that the
   look-back runs out (ERR_TIMEOUT from sphx_sync_status). */
sphx_status sphx_intersect_ragged(sphx_context *ctx, const double *A, const double *B,
                                  const int64_t *edge_offsets, int32_t M, int64_t E,
                                  const double *lat_z, const int64_t *lat_offsets, int64_t L,
                                  const int32_t *edge_lat_lo, const int32_t *edge_lat_hi,
                                  sphx_mode mode, sphx_hit *out, int64_t out_cap,
                                  int64_t *out_total, sphx_stream stream);

/* ---- band areas of spherical cells (the zonal-mean step) -----------------
   Sec. 1 names zonal means as the use that makes arc-latitude intersections
   matter; the paper gives no algorithm for this step, so these calls are this
   library's design around its intersections.

   Mesh arguments, shared by the three calls below:
     nodes         device, n_nodes x 3 FP64 (row-major): node directions, any
                   nonzero length;
     face_offsets  device int64[n_faces + 1]: cell f is the node list
                   face_nodes[face_offsets[f] .. face_offsets[f + 1]);
     face_nodes    device int32[n_face_nodes]: node indices
                   (n_nodes and n_faces below 2^31).
   A cell is a simple spherical polygon whose consecutive nodes (and the last
   and the first) are joined by minor great circle arcs, counter-clockwise
   seen from outside the sphere, with at most one pole in its interior (a pole
   may be a node). lat_z: device, n_lat >= 2 FP64, strictly ascending, in
   [-1, 1]; band k (0 <= k < n_lat - 1) is z_k <= z <= z_{k+1}. Parts of a
   cell outside [z_0, z_{n_lat-1}] are in no band. Cells whose offsets or node
   indices fall outside these arrays get no bands, and sphx_sync_status()
   reports SPHX_ERR_INVALID_ARG. */

/* Bands each cell can meet: band_lo[f] <= k < band_hi[f] (device int32[n_faces]
   each), from the cell's height range (arc endpoints and, where an arc passes
   it, its highest or lowest point, widened by 1e-13; up to the pole for a cell
   around a pole), and area_offsets (device int64[n_faces + 1]), the exclusive
   prefix sum of band_hi - band_lo: the area of cell f in band k goes to
   areas[area_offsets[f] + k - band_lo[f]], and area_offsets[n_faces] is the
   number of entries. Scratch for the prefix sum comes from ctx: calls on one
   context must not overlap in time (as for sphx_intersect_ragged). Stream
   ordered. */
sphx_status sphx_band_ranges(sphx_context *ctx, const double *nodes, int64_t n_nodes,
                             const int64_t *face_offsets, const int32_t *face_nodes,
                             int64_t n_face_nodes, int64_t n_faces, const double *lat_z,
                             int64_t n_lat, int32_t *band_lo, int32_t *band_hi,
                             int64_t *area_offsets, sphx_stream stream);

/* Area of every cell in every band of its range (layout of sphx_band_ranges;
   areas: device FP64[areas_cap]). Each arc is cut where it crosses the
   latitudes in its height range, the crossings computed by `mode` as in
   sphx_intersect_gca_constlat (Eq. 2.2: slot 0 crosses upwards along the
   arc, slot 1 downwards). In longitude and height the area element is
   dlambda dz, so a region's area is the boundary integral of lambda dz (Green);
   the latitude pieces of the boundary have dz = 0, and every arc piece adds
   [lambda z] minus the integral of z dlambda along it (the signed area between
   the piece and the equator, in closed form) to the band it lies in, lambda
   unwrapped along the cell from its first node off the poles. A cell around a
   pole adds 2 pi times each band's share of the height between that node and
   the pole. Areas are FP64 with an absolute error of a few units of rounding
   times (the sum over the cell's arcs of their longitude spans plus the
   cell's height range). Entries past
   areas_cap are not written (sphx_sync_status() reports SPHX_ERR_CAPACITY).
   Cells inside one band (other than the first and the last) get their own
   area, a fan of spherical triangles (Van Oosterom and Strackee's excess);
   cells cut by one latitude get the fan above their two crossings plus the
   sliver under the latitude arc; the rest take the boundary integral. The
   cell lists and a normalised copy of the nodes (24 B per node, made once per
   call) live in ctx's scratch (allocated when a call needs more, then kept;
   calls on one context must not overlap in time). mode: any sphx_mode but
   SPHX_MODE_ADAPTIVE (SPHX_ERR_UNSUPPORTED). Stream ordered. */
sphx_status sphx_band_areas(sphx_context *ctx, const double *nodes, int64_t n_nodes,
                            const int64_t *face_offsets, const int32_t *face_nodes,
                            int64_t n_face_nodes, int64_t n_faces, const double *lat_z,
                            int64_t n_lat, const int32_t *band_lo, const int32_t *band_hi,
                            const int64_t *area_offsets, sphx_mode mode, double *areas,
                            int64_t areas_cap, sphx_stream stream);

/* Zonal sums: for every band k, out_fa[k] = sum over cells of field[f] *
   A[f, k] and out_a[k] = sum of A[f, k] (device FP64[n_lat - 1] each); the
   zonal mean is out_fa / out_a. field: device FP64[n_faces]. Each term is
   rounded once to a multiple of 2^-80 and summed exactly in 128-bit fixed
   point, so the sums do not depend on the order the GPU adds them in
   (bitwise reproducible); the results are the exact sums rounded to FP64.
   Terms of magnitude 2^46 or more, or non-finite, are left out and
   sphx_sync_status() reports SPHX_ERR_INVALID_ARG. band_lo, band_hi,
   area_offsets and areas are those sphx_band_ranges and sphx_band_areas
   wrote (the call reads areas where the offsets point). Scratch comes from
   ctx: calls on one context must not overlap in time. Stream ordered. */
sphx_status sphx_zonal_sums(sphx_context *ctx, const int32_t *band_lo, const int32_t *band_hi,
                            const int64_t *area_offsets, int64_t n_faces, const double *areas,
                            const double *field, int64_t n_lat, double *out_fa, double *out_a,
                            sphx_stream stream);

/* Largest edge count sphx_intersect_ragged_noalloc accepts. */
#define SPHX_NOALLOC_MAX_EDGES 262144

/* The ragged call for callers that must not allocate device memory on their
   call path. The paper has no counterpart: this is a property of the library,
   not of the method. Examples are plugins whose host framework owns the
   device memory budget (a cudaMalloc behind its back can fail, or break that
   framework's accounting) and latency-critical loops that cannot afford
   cudaMalloc's implicit device synchronisation.
   Arguments and results are those of sphx_intersect_ragged. There is no
   context and no caller-given ranges (they are always computed). Output
   order is unspecified (unordered compaction).
   Scratch: a fixed device array of about 4.2 MB inside this library, holding
   room for SPHX_NOALLOC_MAX_EDGES edges. Every GPU that loads the library
   holds it until the process exits.
   E > SPHX_NOALLOC_MAX_EDGES returns SPHX_ERR_INVALID_ARG and launches
   nothing. Nothing is allocated: no cudaMalloc, no cudaFree, no allocating
   library routine.
   The first call on a device looks up the array's device address (with that
   device current). Make that first call before any stream capture.
   All calls share the one array. The counters that must start at zero are
   cleared by each call, on its stream. Calls that overlap on the GPU (other
   streams, other host threads) race on the array and must be serialised by
   the caller.
   A capacity overflow shows as *out_total > out_cap (only out_cap records
   are written). The kernels' other findings (a candidate latitude index
   outside the batch, from corrupt offsets) are recorded in a status word in
   the same array: sphx_noalloc_sync_status reads it. */
sphx_status sphx_intersect_ragged_noalloc(const double *A, const double *B,
                                          const int64_t *edge_offsets, int32_t M, int64_t E,
                                          const double *lat_z, const int64_t *lat_offsets,
                                          int64_t L, sphx_mode mode, sphx_hit *out,
                                          int64_t out_cap, int64_t *out_total, sphx_stream stream);

/* Device status of the allocation-free call (the paper has no counterpart).
   Synchronises `stream`, reads the status word that the kernels of the last
   sphx_intersect_ragged_noalloc call on the current device set, and clears
   it. Returns SPHX_OK, SPHX_ERR_CAPACITY (more hits than out_cap) or
   SPHX_ERR_INVALID_ARG (a candidate outside the batch, from inconsistent
   offsets), or SPHX_ERR_CUDA. Allocates nothing. Each call of
   sphx_intersect_ragged_noalloc clears the word first, so this reports the
   latest call only; calls that overlap on the GPU race on it as on the rest
   of the array. */
sphx_status sphx_noalloc_sync_status(sphx_stream stream);

/* Synchronise `stream`, read and clear the context's device status word.
   Returns SPHX_OK, SPHX_ERR_CAPACITY or SPHX_ERR_TIMEOUT (or SPHX_ERR_CUDA). */
sphx_status sphx_sync_status(sphx_context *ctx, sphx_stream stream);

/* Fix (tuning != NULL) or release (NULL) the ragged launch shape. */
sphx_status sphx_set_tuning(sphx_context *ctx, const sphx_tuning *tuning);
/* Read the tuning the next ragged call will use. */
sphx_status sphx_get_tuning(sphx_context *ctx, sphx_tuning *tuning);

/* Autotune the ragged launch shape on the given batch (same arguments as
   sphx_intersect_ragged): times each candidate shape with CUDA events and
   keeps the fastest for this context. Synchronises `stream`. If ms_out is not
   NULL (host), it receives the best time in milliseconds. The trial runs
   write out and *out_total; any status they raise (such as a capacity
   overflow) is cleared before returning.
   The result is also kept in the process-wide tuning cache under (device
   name, mode, the context's requested compaction, floor(log2) of E, of L / M
   and of M). When the cache already holds that key (found by any context of
   the process, or read from the file SPHX_TUNE_CACHE names), its shape is
   applied to ctx without any trial run and ms_out receives the time stored
   with it. With SPHX_TUNE_CACHE set, every new entry is written to that file
   (JSON, one entry per line). */
sphx_status sphx_autotune_ragged(sphx_context *ctx, const double *A, const double *B,
                                 const int64_t *edge_offsets, int32_t M, int64_t E,
                                 const double *lat_z, const int64_t *lat_offsets, int64_t L,
                                 sphx_mode mode, sphx_hit *out, int64_t out_cap,
                                 int64_t *out_total, sphx_stream stream, double *ms_out);

/* Autotune the dense call's grid for `mode`: 1, 2, 4 or 8 waves of resident
   blocks striding over the tiles of 128 arcs, each timed with CUDA events on
   the given arrays (arguments as sphx_intersect_gca_constlat, which the
   trials call and whose outputs they overwrite). The fastest applies to every
   later dense call of `mode` in the process (the dense call has no context)
   and goes into the tuning cache under (device name, mode, floor(log2 n)); a
   cached entry is applied without trial runs. Synchronises `stream`. ms_out
   (host, may be NULL) receives the best time in milliseconds. */
sphx_status sphx_autotune_dense(const double *A, const double *B, const double *z0, int64_t n,
                                double *out_pts, int32_t *out_count, sphx_mode mode,
                                sphx_stream stream, double *ms_out);

/* Entries the autotuners took from the tuning cache (hits) and found by
   trial runs (sweeps) since the process started or the last clear. */
sphx_status sphx_tuning_cache_stats(int64_t *hits, int64_t *sweeps);
/* Drop the process-wide tuning cache (a file named by SPHX_TUNE_CACHE is read
   again on next use) and reset the dense grids to one wave. */
sphx_status sphx_tuning_cache_clear(void);

/* Peak probe of the current device, written to *rate (host); synchronises
   the device. pipe = 0: FP32 FMA, 1: FP64 FMA, in floating-point operations
   per second (an FMA counts 2); pipe = 2: 32-bit integer multiply-adds per
   second. Independent chains, 8 per thread, 8 blocks of 256 threads per SM. */
sphx_status sphx_probe_fma_rate(int pipe, double *rate);

/* Error text of a status; the last CUDA error string seen by the library. */
const char *sphx_status_string(sphx_status status);
const char *sphx_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPHX_H */
