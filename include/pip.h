/*
 * pip.h -- C ABI of libpip, a GB300 (sm_103a) implementation of the Voronoi
 * point-inclusion test for convex polygons of Zengin & Sezer,
 * "A Novel Point Inclusion Test for Convex Polygons Based on Voronoi
 * Tessellations" (arXiv 2007.15385).
 *
 * The method (Sec. 3-4 of the paper): each convex polygon becomes a set of
 * Voronoi generators -- the centroid p0 (Eq. 3-4, Alg. 3) and its mirror p_k
 * across every edge line (Eq. 8, Alg. 4) -- and a point x is inside when no
 * outer generator is nearer than p0 (Eq. 1, Alg. 5).  Squaring (Eq. 10-11)
 * and expanding turns the test for edge k into the affine sign test
 *     s_k(x) = t_k - x . w_k >= 0,   w_k = 2 (p_k - p0),
 *     t_k = |p_k - o|^2 - |p0 - o|^2,                    (x relative to o)
 * taken over all edges.  The library evaluates it in float32 on the GPU with
 * a rigorous per-point error bound, and re-decides the few points inside the
 * bound exactly, so its answers equal exact closed-polygon membership.
 *
 * Conventions shared by every call:
 *   - Vertices and points are interleaved xy pairs of float32 (PIP_F32) or
 *     int32 (PIP_I32).  Integer vertices must lie in [-2^24, 2^24].
 *   - A polygon has 3..64 vertices in either orientation; edge k joins
 *     vertex k-1 and vertex k (cyclic).
 *   - The boundary is closed (Eq. 1 uses <=): a point on an edge is inside.
 *     A point with a NaN or infinite coordinate is outside.
 *   - Every device pointer is owned by the caller unless stated otherwise;
 *     the library owns only what pip_prepare allocates inside a pip_tables.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls that do not say "synchronizes" only enqueue work and
 *     return; they allocate nothing and can be captured in a CUDA graph.
 *   - Host-detectable argument errors return PIP_E_INVALID_ARG before any
 *     work is enqueued.  Launch failures return PIP_E_CUDA.  Problems found on
 *     the device (a bad polygon) are recorded in the tables and reported by
 *     pip_get_status.
 */
#ifndef PIP_H
#define PIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIP_OK = 0,
    PIP_E_INVALID_ARG = 1, /* null/misaligned pointer, bad size, n outside 3..64 */
    PIP_E_DEGENERATE = 2,  /* repeated consecutive vertex, zero area, or a centroid
                              that is not safely interior (Eq. 4 / Eq. 8 divide by 0) */
    PIP_E_NONCONVEX = 3,   /* turns both ways, folds back, or winds more than once */
    PIP_E_NONFINITE = 4,   /* NaN or infinite vertex coordinate */
    PIP_E_CUDA = 5,        /* a CUDA runtime call failed */
    PIP_E_TIMEOUT = 6,     /* a bounded device-side wait ran out (see pip_selftest_wait_timeout) */
    PIP_E_CAPACITY = 7     /* more points than the capacity given to pip_prepare */
} pip_status;

typedef enum { PIP_F32 = 0, PIP_I32 = 1 } pip_dtype;

/* pip_test output selection (bit flags) */
enum { PIP_MASK = 1, PIP_FIRST_HIT = 2, PIP_CULL = 4, PIP_EARLY_EXIT = 8, PIP_DISC = 16 };

/* Opaque: device tables built from a batch of polygons (generators,
 * coefficients, bounds, validation results) plus the refine workspace. */
typedef struct pip_tables pip_tables;

/*
 * pip_prepare -- convert polygons into Voronoi generator tables
 * (Eq. 3-4 / Alg. 3 centroid, Eq. 8 / Alg. 4 generators, and the expanded
 * Eq. 11 coefficients).  One warp per polygon, in fp64.
 *
 *   d_vertices        device, [total_vertices][2] of `vdtype`, 8-byte aligned.
 *   d_vertex_offsets  device, int32 [num_polygons + 1], non-decreasing,
 *                     offsets[0] = 0, offsets[num_polygons] = total_vertices.
 *   num_polygons      >= 1.
 *   total_vertices    the last offset (the host states it so that nothing
 *                     has to be read back).
 *   max_points        the largest num_points any later pip_test call on these
 *                     tables will pass (sizes the refine queue), >= 0.
 *   out               receives the new tables; owned by the caller, released
 *                     with pip_destroy.
 *
 * The vertices are copied; the caller's buffers may be freed afterwards.
 * Allocates device memory (cudaMalloc), so it must not be called while a
 * stream is being captured.  With one polygon it also synchronizes `stream`
 * once, to keep a host copy of the polygon's coefficients that pip_test then
 * passes to its kernel as launch parameters.  Per-polygon validation runs on the device; an
 * invalid polygon contains no point, and pip_get_status reports the worst
 * problem.  Returns PIP_OK, PIP_E_INVALID_ARG or PIP_E_CUDA.
 */
pip_status pip_prepare(const void *d_vertices, pip_dtype vdtype,
                       const int32_t *d_vertex_offsets, int32_t num_polygons,
                       int32_t total_vertices, int64_t max_points, void *stream,
                       pip_tables **out);

/*
 * pip_prepare_p0 -- pip_prepare with another inner generator.  Any point
 * strictly inside the polygon may serve as p0 (Sec. 3): the mirrored
 * generators and the test's results are then the same closed-polygon
 * membership, only the float32 coefficients and their error bound change.
 *
 *   p0_kind   PIP_P0_CENTROID (Eq. 3-4, what pip_prepare takes),
 *             PIP_P0_VERTEX_MEAN (the mean of the polygon's vertices), or
 *             PIP_P0_GIVEN (d_p0)
 *   d_p0      device double [num_polygons][2], 16-byte aligned, absolute
 *             coordinates; read only for PIP_P0_GIVEN (may be NULL otherwise)
 *
 * A p0 that is not clearly inside every edge line (or not finite) makes the
 * polygon PIP_E_DEGENERATE, as pip_get_status reports.  Everything else as
 * pip_prepare.
 */
enum { PIP_P0_CENTROID = 0, PIP_P0_VERTEX_MEAN = 1, PIP_P0_GIVEN = 2 };
pip_status pip_prepare_p0(const void *d_vertices, pip_dtype vdtype, const int32_t *d_vertex_offsets,
                          int32_t num_polygons, int32_t total_vertices, int64_t max_points, int32_t p0_kind,
                          const double *d_p0, void *stream, pip_tables **out);

/*
 * pip_test -- Voronoi inclusion (Alg. 5 with the squared-distance form of
 * Eq. 10-11), bit-exact against exact closed-polygon membership.
 *
 *   d_points          device, [num_points][2] of `pdtype`, 8-byte aligned
 *                     (16-byte alignment takes the vectorised path).
 *   num_points        0 <= num_points <= max_points of pip_prepare.
 *   d_point_offsets   NULL: every point meets every polygon.  With one
 *                     polygon this is the streaming single-polygon test; with
 *                     several it is the all-pairs test.
 *                     non-NULL: device int64 [num_polygons + 1]; polygon j
 *                     owns points [offs[j], offs[j+1]) (own-polygon batch),
 *                     offs[num_polygons] = num_points.
 *   mode              PIP_MASK and/or PIP_FIRST_HIT (first hit only when
 *                     d_point_offsets is NULL); PIP_CULL may be added for
 *                     the all-pairs test: a polygon is skipped for a warp's
 *                     points when none lies in its vertex bounding box and
 *                     within its outer disc (see PIP_DISC), the points are
 *                     decided inside without the edges when all of them lie
 *                     in its inner disc, and a block stops once each of its
 *                     points has a candidate.
 *                     Same results, less work; not the paper's full-work
 *                     timing convention (Sec. 6.2).  Ignored otherwise.
 *                     PIP_EARLY_EXIT may be added for one polygon or an
 *                     own-polygon batch (16-byte aligned points): the
 *                     sequential test's early break (Sec. 5), warp-uniform --
 *                     edges are taken in groups of four spread around the
 *                     polygon and a warp stops once all its points are
 *                     decided outside.  Same results, less work; not the
 *                     full-work convention either.  Ignored by the exact
 *                     integer batch path and the all-pairs test.
 *                     PIP_DISC may be added for one polygon or an
 *                     own-polygon batch (16-byte aligned points; not
 *                     together with PIP_EARLY_EXIT, which is
 *                     PIP_E_INVALID_ARG): in the Voronoi picture the polygon
 *                     is the cell of p0 (Eq. 1), which holds the disc about
 *                     p0 of half the distance to the nearest generator (the
 *                     distance to the nearest edge line, Eq. 8) and lies in
 *                     the disc about p0 through its farthest vertex.  The
 *                     kernel takes both discs about o = float32(p0) (radii:
 *                     the least distance from o to an edge line, the largest
 *                     to a vertex), with float32 thresholds on |p - o|^2
 *                     that cover its rounding (pip_export_tables' h_disc): a
 *                     point inside the inner disc is decided inside, one
 *                     outside the outer disc outside, without their edges;
 *                     the others take the full test (filter, exact refine).
 *                     Same results, less work; not the full-work convention.
 *                     Ignored by the exact integer batch path (integer
 *                     polygons with integer points) and the all-pairs test.
 *   d_mask            device uint32 [ceil(num_points / 32)]; bit (i % 32) of
 *                     word (i / 32) is 1 when point i is inside its polygon
 *                     (own-polygon batch) or inside at least one polygon
 *                     (otherwise).  Bits past num_points are written as 0.
 *   d_first_hit       device int32 [num_points]: the lowest polygon index
 *                     whose closed polygon holds point i, or -1.  May be NULL
 *                     when PIP_FIRST_HIT is not requested.
 *
 * Points whose float32 result lies within the error bound are queued on the
 * device and re-decided in fp64 and then exactly (int64 for PIP_I32 inputs,
 * floating-point expansions for PIP_F32) by a second kernel.  No host
 * synchronisation; graph-capturable.  Calls on the same tables must not run
 * concurrently (they share the refine queue).
 */
pip_status pip_test(const pip_tables *t, const void *d_points, pip_dtype pdtype,
                    int64_t num_points, const int64_t *d_point_offsets, int mode,
                    uint32_t *d_mask, int32_t *d_first_hit, void *stream);

/*
 * pip_test_host -- pip_test on host buffers: the paper has no counterpart to
 * this call; it serves callers whose points live in host memory.  Mask only,
 * with d_point_offsets NULL (one polygon, or "inside any polygon" for
 * several).  The points move to the caller's device staging buffer in
 * `pieces` pieces (1..64, each a multiple of 128 points but the last) on a
 * copy stream the tables own; piece i is tested on `stream` once its copy has
 * landed, and its mask words go back to h_mask on `stream`, so that copying
 * piece i + 1 overlaps testing and reading back piece i.  One cudaMemcpyAsync
 * per piece and direction.
 *
 *   h_points     host, [num_points][2] of `pdtype`; page-locked
 *                (cudaHostAlloc / cudaHostRegister) for the copies to overlap
 *   d_points     device staging, [num_points][2], 16-byte aligned
 *   d_mask       device staging, uint32 [ceil(num_points / 32)], 16-byte aligned
 *   h_mask       host, uint32 [ceil(num_points / 32)], the result
 *   num_points   0 <= num_points <= max_points of pip_prepare
 *
 * Enqueues only: h_mask is complete once `stream` has finished the work
 * queued before return (synchronize it).  The first call on a set of tables
 * creates its copy stream and events (released by pip_destroy), so make it
 * before any stream capture.  Calls on the same tables must not overlap.
 * Returns PIP_OK, PIP_E_INVALID_ARG, PIP_E_CAPACITY or PIP_E_CUDA.
 */
pip_status pip_test_host(pip_tables *t, const void *h_points, pip_dtype pdtype, int64_t num_points, void *d_points,
                         uint32_t *d_mask, uint32_t *h_mask, int32_t pieces, void *stream);

/*
 * pip_margin -- signed Voronoi margin in length units.  Edge k is the set of
 * points equidistant from p0 and p_k (Eq. 2); the signed distance of x from
 * that bisector is (|x - p0|^2 - |x - p_k|^2) / (2 |p_k - p0|), and the margin
 * is the largest of these over k: > 0 outside, <= 0 inside.  float32, with
 * error at most a few float32 ulps of the coordinates involved.
 *
 *   d_points, num_points, d_point_offsets: as in pip_test.  With
 *   d_point_offsets NULL and several polygons, the result is the smallest
 *   margin over all polygons.
 *   d_margin          device float [num_points].
 * No host synchronisation; graph-capturable.
 */
pip_status pip_margin(const pip_tables *t, const void *d_points, pip_dtype pdtype,
                      int64_t num_points, const int64_t *d_point_offsets, float *d_margin,
                      void *stream);

/*
 * pip_get_status -- synchronizes `stream`, then returns the worst polygon
 * status found by pip_prepare (PIP_OK if every polygon is valid) and, in
 * *refine_count (may be NULL), how many points the last pip_test call sent
 * to the refine step.
 */
pip_status pip_get_status(const pip_tables *t, void *stream, int64_t *refine_count);

/* Per-polygon statuses: copies int32 [num_polygons] to host memory (synchronizes). */
pip_status pip_get_polygon_status(const pip_tables *t, int32_t *h_status, void *stream);

/*
 * pip_export_tables -- copies the prepared tables to host memory
 * (synchronizes); any pointer may be NULL to skip that table.
 *   h_g0     double [num_polygons][2]   centroid p0 (Eq. 4)
 *   h_gk     double [total_vertices][2] mirrored generators p_k (Eq. 8)
 *   h_coef   float [total_vertices][4]  (w_x, w_y, t, 0) of edge k, in
 *                                       coordinates relative to h_origin
 *   h_origin float [num_polygons][2]    o = float32(p0)
 *   h_bound  float [num_polygons][2]    (beta0, beta1): |error of s_k| <=
 *                                       beta0 + beta1 * max(|x|, |y|)
 *   h_disc   float [num_polygons][2]    (tin, tout), the disc bounds of
 *                                       PIP_DISC on d2 = fl(x x + fl(y y)),
 *                                       x = float32(p - o): d2 < tin only
 *                                       strictly inside, d2 > tout only
 *                                       strictly outside; (0, -inf) for an
 *                                       invalid polygon
 */
pip_status pip_export_tables(const pip_tables *t, double *h_g0, double *h_gk, float *h_coef,
                             float *h_origin, float *h_bound, float *h_disc, void *stream);

/* Releases the tables (synchronizes the device first).  NULL is a no-op. */
void pip_destroy(pip_tables *t);

/*
 * Kernel timing, for benchmarks.  pip_timing(t, 1) makes every later pip_test
 * on `t` record CUDA events on its stream around its bulk kernel and around
 * its refine kernel (up to 4096 calls are kept); pip_timing(t, 0) stops.
 * Creating the events synchronizes the device, so call it outside capture.
 * pip_timing_read synchronizes, returns the number of timed calls and the
 * summed milliseconds of the bulk and refine kernels, and starts over.
 */
pip_status pip_timing(pip_tables *t, int enable);
pip_status pip_timing_read(pip_tables *t, int32_t *calls, double *bulk_ms, double *refine_ms);

/*
 * Tile shapes of the pipelined single-polygon kernel (the path pip_test takes
 * for one polygon, no point offsets and 16-byte aligned points): each variant
 * is (points per lane per stage, ring stages).  pip_autotune_stream times
 * every variant `reps` times with CUDA events on the caller's own inputs
 * (synchronizes; not during capture), keeps the fastest in the tables and
 * returns it with its mean milliseconds.  pip_set_stream_variant picks one
 * directly (for a cached tuning result).  The disc filter (PIP_DISC) runs at
 * the chosen shape as well.
 */
int32_t pip_stream_variant_count(void);
pip_status pip_set_stream_variant(pip_tables *t, int32_t variant);
pip_status pip_autotune_stream(pip_tables *t, const void *d_points, pip_dtype pdtype,
                               int64_t num_points, uint32_t *d_mask, int32_t reps, void *stream,
                               int32_t *best_variant, float *best_ms);

/*
 * Tile shapes of the pipelined own-polygon batch kernel (the path pip_test
 * takes with point offsets and 16-byte aligned points): each variant is
 * (points per lane, ring stages); an item of work is 224 x points per lane
 * points of one polygon.  pip_autotune_batch times every variant `reps` times
 * with CUDA events on the caller's own batch (d_point_offsets as in pip_test;
 * synchronizes, not during capture), keeps the fastest in the tables and
 * returns it with its mean milliseconds per pip_test call.
 */
int32_t pip_batch_variant_count(void);
pip_status pip_set_batch_variant(pip_tables *t, int32_t variant);
pip_status pip_autotune_batch(pip_tables *t, const void *d_points, pip_dtype pdtype,
                              int64_t num_points, const int64_t *d_point_offsets, uint32_t *d_mask,
                              int32_t reps, void *stream, int32_t *best_variant, float *best_ms);

/*
 * pip_set_tuning_cache -- the paper has no counterpart; a JSON file where the
 * autotuners keep their choices.  With a path set, pip_autotune_stream and
 * pip_autotune_batch first look up the key (kernel, GPU name, polygons,
 * vertices, points, vertex and point types): a hit sets that tile shape and
 * returns its recorded time without any timing run or synchronisation; a miss
 * times the variants as usual and records the winner (the file is rewritten
 * whole, through a temporary file and a rename).  NULL or "" turns the cache
 * off (the default).  The path is copied; process-wide.
 */
pip_status pip_set_tuning_cache(const char *path);

/* Number of polygons / vertices held by the tables. */
int32_t pip_num_polygons(const pip_tables *t);
int32_t pip_total_vertices(const pip_tables *t);

const char *pip_status_string(pip_status s);

/* ------------------------------------------------------------------------
 * Same-chip comparators (the paper's reference tests, Sec. 2.1-2.2, and the
 * unbatched fp64 form of Alg. 5).  Single polygon or own-polygon batch
 * (d_point_offsets as in pip_test; NULL needs num_polygons == 1), mask
 * output as in pip_test, float polygons and float points only (integer
 * tables return PIP_E_INVALID_ARG).  They are NOT exact: each decides in its
 * own precision, as the paper's listings do.
 *
 * They run in the Voronoi test's own frame, so that the methods differ only
 * in their per-edge arithmetic: with one polygon and 16-byte aligned points,
 * sign of offset and ray crossing take the pipelined single-polygon kernel
 * (edges as launch parameters, bulk-copy ring, ballot packing); an own-polygon
 * batch takes the pipelined batch kernel with the offsets read on the device
 * (no host synchronisation, graph-capturable) and needs 16-byte aligned
 * points (PIP_E_INVALID_ARG otherwise).  The fp64 form of one polygon, and
 * one polygon's unaligned points, take a register-streaming kernel.  Calls on
 * the same tables must not overlap each other or pip_test (they share the
 * work-item table).  Edge k's LHS - RHS = q_y dV_x - q_x dV_y - RHS is formed
 * as one two-FMA affine form of the point, from dV and RHS rounded to float32
 * at pip_prepare.
 * ------------------------------------------------------------------------ */

/* Alg. 2 (sign of offset) in float32: inside when every edge's
 * "LHS < RHS" flag is the same. */
pip_status pip_test_sign_of_offset(const pip_tables *t, const float *d_points,
                                   int64_t num_points, const int64_t *d_point_offsets,
                                   uint32_t *d_mask, void *stream);

/* Alg. 1 (ray crossing, +x ray) in float32; an odd crossing count is inside. */
pip_status pip_test_ray_crossing(const pip_tables *t, const float *d_points,
                                 int64_t num_points, const int64_t *d_point_offsets,
                                 uint32_t *d_mask, void *stream);

/* Alg. 5 literally in fp64: M_0 <= M_k for all k with M the squared distances
 * to the fp64 generators; no error bound, no refine. */
pip_status pip_test_voronoi_fp64(const pip_tables *t, const float *d_points,
                                 int64_t num_points, const int64_t *d_point_offsets,
                                 uint32_t *d_mask, void *stream);

/* ------------------------------------------------------------------------
 * Differentiable collision penalty (motion-planning use of the margin):
 *
 *   L = sum_pose sum_point softplus(-m(R(theta)^T (p - t)) / tau)
 *
 * with m the Voronoi margin of pip_margin (the signed distance from the Eq. 2
 * bisectors), of one convex footprint given in its body frame.  The gradient
 * flows through the margin's maximising edge (lowest index among ties), the
 * mirrored generators (Eq. 8) and the centroid (Eq. 3-4) to the vertices, and
 * through the rigid transform to the poses.  Each call rebuilds the
 * generators from the vertices (nothing is carried from forward to
 * backward).  The bulk margins are float32; for every (pose, point) pair
 * with a nonzero gradient the backward pass re-decides the argmax edge and
 * re-evaluates its margin in float-float arithmetic (exact point offset,
 * two-part fp64-derived coefficients), so that dL/dm carries no float32
 * margin error.  Per-edge sums go to per-thread float32 shared-memory slots
 * for up to 16 edges (a fixed order, reproducible) and to per-warp slots by
 * shared-memory atomics above (order not fixed); each block adds them in
 * fp64, and the per-block partials are added in fp64 in a fixed order.
 *
 *   d_vertices   device float [num_vertices][2], 3..64 vertices, 8-byte aligned
 *   d_poses      device float [num_poses][3] = (t_x, t_y, theta)
 *   d_points     device float [num_points][2], 8-byte aligned
 *   tau          > 0, in the units of the coordinates
 *   d_workspace  device, >= pip_penalty_workspace_bytes(...) bytes, 256-byte
 *                aligned, owned by the caller; nothing is allocated
 *   d_loss       device double [1]
 *   d_grad_loss  device float [1] (the upstream dL_total/dL) or NULL for 1
 *   d_grad_vertices device double [num_vertices][2];  d_grad_poses device double [num_poses][3]
 *
 *   flags        0, or PIP_PENALTY_CULL: the pairs provably beyond 120 tau of
 *                every edge line (a disc about the pose's centroid, from
 *                the largest angle between consecutive edge normals and the
 *                largest centroid-to-edge distance) are left out before
 *                their margin is formed.  Their float32 softplus term and
 *                gradient are exactly 0, so the results are those of the
 *                full pass up to the order of the float32 partial sums;
 *                less work, not the full-work timing convention.  Other
 *                bits: PIP_E_INVALID_ARG.
 *
 * An invalid footprint (see pip_prepare) gives loss 0 and zero gradients.
 * No host synchronisation.
 * ------------------------------------------------------------------------ */
enum { PIP_PENALTY_CULL = 1 };
size_t pip_penalty_workspace_bytes(int32_t num_vertices, int32_t num_poses, int64_t num_points);
pip_status pip_penalty_forward(const float *d_vertices, int32_t num_vertices, const float *d_poses,
                               int32_t num_poses, const float *d_points, int64_t num_points, float tau,
                               double *d_loss, int32_t flags, void *d_workspace, size_t workspace_bytes,
                               void *stream);
pip_status pip_penalty_backward(const float *d_vertices, int32_t num_vertices, const float *d_poses,
                                int32_t num_poses, const float *d_points, int64_t num_points, float tau,
                                const float *d_grad_loss, double *d_grad_vertices, double *d_grad_poses,
                                int32_t flags, void *d_workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------
 * pip_test_single_noalloc -- the paper has no counterpart to this call; it
 * exists for callers that cannot allocate device memory when they test
 * points: a fixed-rate control loop (a vehicle's collision check) that cannot
 * absorb cudaMalloc's latency and implicit synchronisation, or a plug-in
 * whose host application owns the device memory pool or a fixed memory
 * budget.  It does what pip_prepare + pip_test + pip_destroy do for ONE
 * polygon and a mask, with the same exact result, but allocates nothing: its
 * scratch (the polygon's tables and the refine queue, about 4 MiB) is one
 * static device array that every GPU loading this library holds until the
 * process exits.
 *
 *   d_vertices    device, [num_vertices][2] of `vdtype`, 8-byte aligned.
 *   num_vertices  3..64.
 *   d_points      device, [num_points][2] of `pdtype`, 8-byte aligned.
 *   num_points    0 .. 1048576 (2^20); more returns PIP_E_CAPACITY and
 *                 enqueues nothing.
 *   d_mask        device uint32 [ceil(num_points / 32)], as in pip_test.
 *   d_status      device int32 [1] or NULL: receives the polygon's status
 *                 (PIP_OK or the pip_prepare code; an invalid polygon
 *                 contains no point).
 *
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one scratch array and it
 * keeps the last call's contents (each call clears its own counters first):
 * calls that overlap on the GPU -- on different streams, or from host threads
 * without ordering -- race on it and must not be issued.  The looked-up
 * address is kept for the life of the process: after cudaDeviceReset on a
 * device, do not call this entry point on that device again.
 * ------------------------------------------------------------------------ */
pip_status pip_test_single_noalloc(const void *d_vertices, pip_dtype vdtype, int32_t num_vertices,
                                   const void *d_points, pip_dtype pdtype, int64_t num_points,
                                   uint32_t *d_mask, int32_t *d_status, void *stream);

/* ------------------------------------------------------------------------
 * pip_rasterize -- pixel coverage of the prepared polygons (the screen-space
 * use of the inclusion test, Sec. 1: each pixel's membership decided by a
 * point inclusion test at its centre).  Pixel (c, r), 0 <= c < width,
 * 0 <= r < height, has the float32 centre
 *     (fmaf((float)c, dx, x0), fmaf((float)r, dy, y0))
 * (one rounding each); the results are those of pip_test's all-pairs test on
 * those centres, bit-exact (closed polygons, fp64 / exact refine).
 *
 *   width, height   1 .. 2^24 each, width * height <= max_points of pip_prepare
 *   x0, y0, dx, dy  finite, dx > 0, dy > 0, the last centre finite
 *   d_first_hit     device int32 [height][width] (row-major) or NULL: the
 *                   lowest polygon index whose closed polygon holds the
 *                   pixel's centre (front to back), or -1
 *   d_mask          device uint32 [height][ceil(width / 32)] or NULL (not
 *                   both NULL): bit (c % 32) of word r * ceil(width / 32) +
 *                   c / 32 is 1 when some polygon holds pixel (c, r); bits
 *                   past width are 0
 *   d_workspace     device, >= pip_raster_workspace_bytes(num_polygons,
 *                   width, height) bytes (a tile x polygon bitmask),
 *                   16-byte aligned, owned by the caller
 *
 * Shares the tables' refine queue and candidate keys with pip_test (calls on
 * the same tables must not overlap).  No allocation, no host
 * synchronisation; graph-capturable.  PIP_E_CAPACITY when width * height
 * exceeds max_points, PIP_E_INVALID_ARG for a bad grid or buffer.
 * ------------------------------------------------------------------------ */
size_t pip_raster_workspace_bytes(int32_t num_polygons, int32_t width, int32_t height);
pip_status pip_rasterize(const pip_tables *t, int32_t width, int32_t height, float x0, float y0, float dx,
                         float dy, int32_t *d_first_hit, uint32_t *d_mask, void *d_workspace,
                         size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------
 * pip_fma_peak -- the paper has no counterpart to this call; it measures the
 * float32 FMA throughput of the current GPU, the denominator of the FP32
 * roofline that the dense all-pairs test and the penalty are reported
 * against.  Launches blocks_per_sm x #SM blocks of 256 threads, each thread
 * running 8 independent FMA chains for `iters` x 16 steps; the caller times
 * the launch (CUDA events on `stream`) and divides *fmas by the time.
 *
 *   d_sink       device float [sink_floats], sink_floats >= blocks x 256; the
 *                kernel never actually writes it (a guarded store that keeps
 *                the work from being optimised away)
 *   fmas         receives the number of FMAs the launch performs
 * Returns PIP_OK, PIP_E_INVALID_ARG or PIP_E_CUDA.
 * ------------------------------------------------------------------------ */
pip_status pip_fma_peak(int32_t blocks_per_sm, int32_t iters, float *d_sink, int64_t sink_floats, void *stream,
                        int64_t *fmas);

/* ------------------------------------------------------------------------
 * pip_selftest_wait_timeout -- the paper has no counterpart to this call; it
 * exercises the failure path that every pipelined kernel takes when one of
 * its waits never completes (a lost producer or consumer).
 *
 * Launches one CTA that starts a 4 KiB bulk copy into shared memory, then
 * waits on an mbarrier phase that nothing completes, bounded by
 * `limit_cycles` SM cycles (1 .. 2^31; the kernels' own limit is 2e9, about
 * a second).  When the limit runs out the kernel records PIP_E_TIMEOUT in the
 * tables' error word, waits (again bounded) for its own copy to land and
 * returns: no trap, no fault, the context stays usable.  The next
 * pip_get_status returns PIP_E_TIMEOUT once and clears the word.
 *
 *   t         tables from pip_prepare (only the error word is written)
 *   d_scratch device, >= 4096 bytes, 16-byte aligned (the copy's source)
 * Returns PIP_OK when the launch was queued, PIP_E_INVALID_ARG or PIP_E_CUDA.
 * ------------------------------------------------------------------------ */
pip_status pip_selftest_wait_timeout(pip_tables *t, const void *d_scratch, int64_t limit_cycles,
                                     void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PIP_H */
