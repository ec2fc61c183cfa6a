/* grca.h — C ABI of the GB300-native GRCA ray caster (libgrca.so).
 *
 * GRCA (Gajmer Ray-Casting Algorithm) answers, per frame, the problem of
 * Sec. 1.1 (Eq. brute): for every ray of every spinning LiDAR, the closest
 * triangle it intersects and its distance.  It inverts the question — which
 * rays can each triangle hit — and needs no acceleration structure: each
 * (triangle, LiDAR) pair is moved into the emitter frame, its elevation and
 * azimuth extent is bounded against the channel cones/plane (Sec. 3.2-3.7)
 * and the azimuth grid, optional range culling is applied (App. A.4.1), the
 * candidate (channel, ray) spans are expanded, each candidate gets a
 * watertight ray-triangle test and a per-ray closest-hit reduction keeps
 * (distance, triangle id) (App. A.4.1 Step 5, Sec. A.5.2).
 *
 * Conventions (all entry points):
 *   - Return a grca_status: GRCA_OK (0) or a negative error code; no
 *     exception crosses the ABI.  grca_status_string() names each code.
 *   - All device work is asynchronous on the caller's `stream` (a
 *     cudaStream_t passed as void*; NULL = legacy default stream).  Errors
 *     raised by device work (queue capacity overflow) are reported by
 *     grca_get_stats() on that stream.
 *   - One context per host thread; a context is bound to one CUDA device.
 *     Its casts share the context's work buffers (keys, queues, tables), so
 *     they run in the order issued on one stream; casts on different streams
 *     must be ordered by the caller (events or synchronisation).
 *   - World frame: any right-handed frame; sensor axes f (forward), r (right),
 *     u (up) are orthonormal in it.  Azimuth increases from f toward r
 *     ("clockwise seen from above", Sec. 3.1), elevation upward from the
 *     f-r plane.
 *   - Rays of a cast are laid out sensor-major in `sensor_ids` order, then
 *     channel (ascending elevation), then ray (ascending azimuth): global ray
 *     index g = O_n + j * n_rays_n + i (App. A.4.1, Step 5).
 */
#ifndef GRCA_H
#define GRCA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grca_ctx grca_ctx; /* opaque; created and owned by the library */
typedef int32_t grca_status;

enum {
    GRCA_OK = 0,
    GRCA_ERR_INVALID_ARG = -1, /* null pointer, bad size, bad sensor, unsorted table ... */
    GRCA_ERR_OOM = -2,         /* device or host allocation failed */
    GRCA_ERR_CUDA = -3,        /* a CUDA runtime call failed (see grca_last_cuda_error) */
    GRCA_ERR_CAPACITY = -4,    /* a device work queue overflowed; results of that cast are invalid */
    GRCA_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
    GRCA_ERR_NOT_READY = -6    /* no triangles uploaded, or no sensors */
};

/* Where a host-API buffer lives. */
enum { GRCA_MEM_HOST = 0, GRCA_MEM_DEVICE = 1 };

/* grca_cast flags. */
enum {
    /* FP32 tests, then FP64 re-tests of every ray flagged by the FP32 pass
     * (a candidate within the FP32 error bound of an edge, a t whose FP32
     * error bound is large, or two hits on one ray whose FP32 distances are
     * within the tie band).  Off: plain FP32 path. */
    GRCA_CAST_FP64_RECHECK = 1u << 0,
    /* Keep only triangles facing the sensor: n = (v1-v0)x(v2-v0) with
     * n.(o - v0) > 0 (reading of App. A.4.1 Step 1, sign fixed to the
     * usual outward-normal convention). */
    GRCA_CAST_CULL_BACKFACE = 1u << 1,
    /* Debug: no culling, every ray against every triangle (small scenes). */
    GRCA_CAST_BRUTE = 1u << 2,
    /* Capture the frame's kernel sequence into a CUDA graph and replay it on
     * later casts with the same shape, flags and buffers. */
    GRCA_CAST_GRAPH = 1u << 3,
    /* Debug: append every tested (ray, triangle) candidate to the dump buffer
     * set by grca_set_debug_dump (for superset checks of the culling). */
    GRCA_CAST_DUMP_CANDIDATES = 1u << 4,
    /* Lossy apparent-area cull (App. A.4.1 Step 1, Eq. apparent_area): skip a
     * (triangle, sensor) pair when (A_T (c-o).n^)^2 < eps_A^2 |c-o|^6, with
     * A_T the area, c the centroid and n^ the unit normal; eps_A =
     * grca_options.area_eps (default 1e-6, the paper's value).  Drops true
     * hits on small, far or edge-on triangles by design. */
    GRCA_CAST_LOSSY_AREA = 1u << 5,
    /* Turn off the group-level cull (GACP-T_g, Sec. 10.1.1).  That cull is
     * lossless and runs by default whenever some sensor of the cast has a
     * finite d_max: each 32-triangle group's box (kept current by uploads
     * and vertex updates) is tested against every sensor's range and channel
     * window before any per-triangle work.  For debugging and A/B timing. */
    GRCA_CAST_NO_GROUP_CULL = 1u << 6,
    /* Trace the static triangles through the culls even when a static
     * hierarchy exists (grca_build_static): for A/B timing and debugging. */
    GRCA_CAST_NO_STATIC_BVH = 1u << 7,
    /* grca_cast_host only (other calls reject it): return once the frame is
     * enqueued instead of once its results are on the host.  The results are
     * copied to the host arrays on a stream of the context's own, after the
     * frame; grca_host_wait tells when they are there.  Until then the host
     * arrays must not be read and the host source `xyz_dynamic` must stay
     * unchanged.  The next frame on the context runs meanwhile (only its key
     * decode waits for this copy-out), so a caller that alternates two pairs
     * of host arrays overlaps each frame's copy-out with the next frame. */
    GRCA_CAST_HOST_ASYNC = 1u << 8,
    /* Test every candidate even where its ray already holds a closer hit.
     * By default an FP32+recheck cast drops, before its test setup, a
     * (triangle, sensor) pair of at most 4 candidate rays when every one of
     * those rays already holds a certain hit closer than the pair's distance
     * lower bound (nearest vertex minus longest edge) by more than the tie
     * band (counted in grca_stats.pairs_occluded), and drops single
     * candidates of large pairs the same way in their per-channel test pass.
     * None of the dropped tests could change the result, so the output is
     * the same bits either way.  For A/B timing and debugging. */
    GRCA_CAST_NO_OCCLUSION = 1u << 9
};

/* Context options (all fields 0 = library default). */
typedef struct {
    uint64_t big_pair_capacity;  /* pairs deferred to the per-channel span pass (default 4M, 112 B each) */
    uint64_t chunk_capacity;     /* test chunks in the work queue (default 32M, 16 B each) */
    uint64_t recheck_capacity;   /* (ray, triangle) pairs queued for FP64 re-test (default 8M, 16 B each) */
    uint32_t inline_max;         /* candidates per pair tested inline by the culling pass (default 16) */
    uint32_t chunk_rays;         /* rays per test chunk (default 64) */
    uint32_t cull_block;         /* threads per culling block (default 256) */
    uint32_t cull_blocks_per_sm; /* resident culling blocks per SM (default 4) */
    uint64_t survivor_capacity;  /* max (triangle, sensor) pairs passing the elevation cull per cast
                                    (default 256M, 8 B each; the queue grows to n_tris * n_sensors up to it) */
    double area_eps;             /* eps_A of GRCA_CAST_LOSSY_AREA (default 1e-6) */
} grca_options;

/* One spinning LiDAR (Sec. 3.1, Eq. ray_dir and the centred angle grid).
 *   origin, f, r, u : position and orthonormal axes, FP64, world frame.
 *   elev_rad        : n_channels elevations in radians, strictly ascending,
 *                     |elev| < pi/2.  Copied by the library.
 *   n_rays, theta0, dtheta : azimuth grid theta_i = theta0 + i*dtheta,
 *                     i in [0, n_rays); n_rays*dtheta <= 2*pi (+1e-9).  When
 *                     n_rays*dtheta == 2*pi (to 1e-9) the grid closes the
 *                     circle and spans wrap around it.
 *   d_min, d_max    : a hit counts only if d_min <= t <= d_max (per-hit
 *                     reading of the range filter of App. A.4.1); d_max may
 *                     be +inf.  0 <= d_min <= d_max.
 * Limits: n_channels <= 1024, n_rays <= 32768, at most 64 sensors per cast. */
typedef struct {
    double origin[3];
    double f[3];
    double r[3];
    double u[3];
    const double* elev_rad;
    uint32_t n_channels;
    uint32_t n_rays;
    double theta0;
    double dtheta;
    double d_min;
    double d_max;
} grca_sensor_desc;

/* Counters of the last cast (valid after grca_get_stats, which syncs). */
typedef struct {
    uint64_t pairs;           /* (triangle, sensor) pairs visited = n_sensors * n_tris */
    uint64_t pairs_live;      /* pairs whose candidate span is non-empty */
    uint64_t survivors;       /* pairs that passed the elevation (channel-span) cull */
    uint64_t candidates;      /* (channel, ray) candidates in the pair spans */
    uint64_t candidates_inline; /* of which tested inline by the culling pass */
    uint64_t big_pairs;       /* pairs deferred to the per-channel span pass */
    uint64_t chunks;          /* test chunks emitted by that pass */
    uint64_t tests;           /* ray-triangle tests run (candidates dropped as occluded are not tested) */
    uint64_t hits;            /* certain FP32 hits those tests found */
    uint64_t uncertain;       /* FP32 tests sent to the FP64 re-test */
    uint64_t ties;            /* tie events between FP32 hits on one ray */
    uint64_t flagged_rays;    /* rays resolved by the FP64 re-test */
    uint64_t recheck_pairs;   /* queued (ray, triangle) pairs kept by the filter and re-tested in FP64
                                 (besides the re-test of each flagged ray's FP32 winner) */
    uint64_t group_culled;    /* pairs skipped whole by the group-level cull (GACP-T_g) */
    uint64_t bvh_node_visits; /* static-hierarchy node visits, one per warp of 32 rays (hybrid casts) */
    uint64_t bvh_tests;       /* ray-triangle pre-tests on static leaves (hybrid casts) */
    uint64_t n_rays;          /* rays in the last cast */
    uint32_t device_error;    /* bit mask of device-side errors (0 = none) */
    uint32_t reserved;
    /* FP64 re-test queue by cause, FP32+recheck casts only.  queued_*: (ray,
     * triangle) entries the FP32 pass queued; kept_*: of those, the entries
     * the filter kept because they may still beat or tie the ray's final FP32
     * winner (their rays are the flagged rays).  Causes: edge = the ray passes
     * within the FP32 error bound of an edge of the triangle; t = inside with
     * margin but the error bound of the FP32 distance is above the accepted
     * relative bound; range = the distance lies within its error bound of
     * d_min or d_max; orient = the sign of (v0-o).n is within its error bound;
     * tie = two certain FP32 hits on one ray within the tie band (both
     * triangles queued). */
    uint64_t queued_edge, queued_t, queued_range, queued_orient, queued_tie;
    uint64_t kept_edge, kept_t, kept_range, kept_orient, kept_tie;
    /* queued entries of cause t whose distance was re-evaluated in
     * double-float FP32 arithmetic (bounded to the accepted relative error)
     * before the filter; the settled ones are committed as certain hits or
     * dropped as misses and are never kept. */
    uint64_t t_refined;
    /* live pairs (FP32+recheck casts, at most 4 candidate rays) dropped
     * before their test setup because every candidate ray already held a
     * certain hit closer than the pair's distance lower bound (nearest
     * vertex minus longest edge) by more than the tie band: none of their
     * tests could change the result.  Counted in pairs_live as well. */
    uint64_t pairs_occluded;
} grca_stats;

/* Create a context on CUDA device `device`.  `opt` may be NULL.
 * *out receives the context (owned by the library; free with grca_destroy).
 * Returns GRCA_ERR_INVALID_ARG for a null `out` or bad options (a culling
 * block size that is not a multiple of 32 in [32, 256], a chunk size above
 * 4096, a capacity above 2^32 - 1), GRCA_ERR_CUDA if the device cannot be
 * used and GRCA_ERR_OOM if a work buffer cannot be allocated. */
grca_status grca_create(grca_ctx** out, int device, const grca_options* opt);

/* Free every device and host buffer of the context.  NULL is a no-op. */
void grca_destroy(grca_ctx* ctx);

/* Register a sensor (Sec. 3.1).  The description and its elevation table are
 * copied.  *out_sensor_id receives a dense id (0, 1, ...).  Returns
 * GRCA_ERR_INVALID_ARG unless: 1 <= n_channels <= 1024 and 1 <= n_rays <=
 * 32768; f, r, u orthonormal to 1e-9 and the origin finite; elevations
 * finite, strictly ascending and below pi/2 in magnitude; dtheta > 0 with
 * n_rays * dtheta <= 2 pi and |theta0| <= 4 pi; 0 <= d_min <= d_max with
 * d_min finite (d_max may be +inf). */
grca_status grca_create_sensor(grca_ctx* ctx, const grca_sensor_desc* desc, int32_t* out_sensor_id);

/* Move a sensor: new origin and orthonormal axes (FP64, world frame); the
 * next cast uses them.  Returns GRCA_ERR_INVALID_ARG for an unknown id, a
 * non-finite origin or axes that are not orthonormal to 1e-9. */
grca_status grca_set_sensor_pose(grca_ctx* ctx, int32_t sensor_id, const double origin[3], const double f[3],
                                 const double r[3], const double u[3]);

/* (Re)define the scene: n_tris unindexed FP32 triangles, layout [n][3][3]
 * (triangle, vertex, xyz), world frame.  `where` = GRCA_MEM_HOST or
 * GRCA_MEM_DEVICE tells where `xyz` lives.  The library copies the data into
 * a device buffer it owns (asynchronous on `stream`; a host source must stay
 * valid until the stream reaches the copy).  Triangle ids are 0..n_tris-1. */
grca_status grca_upload_triangles(grca_ctx* ctx, const float* xyz, uint32_t n_tris, int where, void* stream);

/* Overwrite triangles [first_tri, first_tri + n_tris) with new vertices
 * (same layout), e.g. the dynamic part of the scene every frame; `where` and
 * the lifetime of a host source as for grca_upload_triangles.  Touching a
 * triangle of the static hierarchy (grca_build_static) makes it stale until
 * rebuilt; group boxes of the touched groups are refreshed by the next cast
 * that needs them.  Returns GRCA_ERR_INVALID_ARG for a range outside the
 * uploaded set. */
grca_status grca_update_vertices(grca_ctx* ctx, const float* xyz, uint32_t first_tri, uint32_t n_tris, int where,
                                 void* stream);

/* Cast one frame for the listed sensors (Sec. 1.1 problem statement).
 *   out_dist : DEVICE pointer, one float per ray: distance t of the closest
 *              hit, +inf on a miss (Sec. A.5.1).
 *   out_tri  : DEVICE pointer, one uint32 per ray: triangle id, 0xFFFFFFFF on
 *              a miss.  Ties in distance go to the lower id.
 * Both arrays hold sum over sensors of n_channels*n_rays entries in the
 * layout above and are owned by the caller.  `flags` = GRCA_CAST_*. */
grca_status grca_cast(grca_ctx* ctx, const int32_t* sensor_ids, uint32_t n_sensors, float* out_dist,
                      uint32_t* out_tri, uint32_t flags, void* stream);

/* Triangle-sharded casts (several GPUs, each holding a slice of the
 * triangles).  The closest hit over the union of the slices is the minimum,
 * over the slices, of each slice's closest hit (Sec. 1.1, Eq. brute: the
 * result is a minimum over triangles), so a frame is cast per slice and the
 * per-ray (distance, id) keys are combined by a u64 MIN across the GPUs
 * (the caller's collective; keys are < 2^63, so a signed int64 MIN gives the
 * same result).  Protocol per frame, the same sensors and flags on every
 * shard, each shard holding triangles with global ids tri_base + local id:
 *   1. grca_cast_shard: the FP32 pass over this GPU's slice (with the
 *      double-float re-evaluation of t); keys_out receives one u64 key per
 *      ray, (FP32 bits of t) << 32 | global triangle id, 0x7F800000FFFFFFFF
 *      for a miss.
 *   2. keys_min = MIN over the shards of those keys.  Without
 *      GRCA_CAST_FP64_RECHECK, keys_min is final: go to 5.
 *   3. grca_flag_shard: the FP64 re-test's filter against keys_min; flags_out
 *      receives one byte per ray, 1 where this shard holds a queued candidate
 *      that may beat or tie keys_min, or an FP32 winner other than keys_min's
 *      triangle within the tie band of it.  flags_any = MAX over the shards.
 *   4. grca_resolve_shard: every ray with flags_any set is settled in FP64 by
 *      each shard holding a candidate within the tie band (the shard of
 *      keys_min's triangle included); keys_out receives this shard's keys,
 *      the FP64 ones where settled.  keys_final = MIN over the shards.
 *   5. grca_decode_keys (any shard): distances and global ids of the keys.
 * The result equals a single-GPU cast of the whole triangle set with the
 * same flags: the re-test sees the same candidates.
 * Flags: as grca_cast except GRAPH, BRUTE, DUMP_CANDIDATES and HOST_ASYNC
 * (GRCA_ERR_INVALID_ARG).  Key arrays (int64 / u64) and flag arrays (one
 * byte) are DEVICE arrays of the cast's ray count.  Steps 3-5 use the work
 * buffers of the context's last grca_cast_shard (GRCA_ERR_NOT_READY without
 * one; step 4 also needs step 3, and reads keys_min again: keep it until
 * then); no other cast may run on the context in between. */
grca_status grca_cast_shard(grca_ctx* ctx, const int32_t* sensor_ids, uint32_t n_sensors, uint32_t tri_base,
                            uint64_t* keys_out, uint32_t flags, void* stream);
grca_status grca_flag_shard(grca_ctx* ctx, const uint64_t* keys_min, uint8_t* flags_out, void* stream);
grca_status grca_resolve_shard(grca_ctx* ctx, const uint8_t* flags_any, uint64_t* keys_out, void* stream);
grca_status grca_decode_keys(grca_ctx* ctx, const uint64_t* keys, float* out_dist, uint32_t* out_tri, void* stream);

/* Same as grca_cast with HOST output arrays: the frame's vertices
 * (`xyz_dynamic`, n_dynamic triangles starting at first_dynamic, HOST;
 * pinned memory gives the fastest copy) are copied in, the results copied
 * back into the host arrays, and the call returns once they are there
 * (end-to-end frame; with GRCA_CAST_HOST_ASYNC, once the frame is enqueued).
 * When the dynamic triangles are the tail of the set
 * (first_dynamic + n_dynamic = uploaded count, first_dynamic > 0), their copy
 * runs on an internal stream while the elevation cull works through the
 * triangles before them.  Returns GRCA_ERR_INVALID_ARG for a range outside
 * the uploaded set. */
grca_status grca_cast_host(grca_ctx* ctx, const int32_t* sensor_ids, uint32_t n_sensors, const float* xyz_dynamic,
                           uint32_t first_dynamic, uint32_t n_dynamic, float* out_dist_host,
                           uint32_t* out_tri_host, uint32_t flags, void* stream);

/* Block until at most `max_pending` grca_cast_host calls with
 * GRCA_CAST_HOST_ASYNC still have results on their way to the host (0: all
 * of them are there); casts complete in call order.  At most 8 such casts
 * are in flight: a ninth call first waits for the oldest.  Returns
 * GRCA_ERR_CUDA if a copy failed, GRCA_ERR_INVALID_ARG for a null context. */
grca_status grca_host_wait(grca_ctx* ctx, uint32_t max_pending);

/* Time the launch-parameter candidates (culling block shape: 128 or 256
 * threads, 2 to 32 blocks per SM; inline candidate limit 4 to 1024; chunk
 * size 32 to 256 rays) by coordinate descent on the current scene for these
 * sensors and flags, and keep the fastest for later casts of the same shape.
 * The result does not depend on these parameters.  Runs casts
 * into the given output buffers; synchronous.  *out_ms (nullable) receives
 * the best frame time. */
grca_status grca_autotune(grca_ctx* ctx, const int32_t* sensor_ids, uint32_t n_sensors, float* out_dist,
                          uint32_t* out_tri, uint32_t flags, void* stream, float* out_ms);

/* The launch configuration a cast of these sensors with these flags would
 * use now (tuned by grca_autotune for this cast shape, else the context's
 * default): out[0] inline candidate limit, out[1] chunk size in rays,
 * out[2] culling block size, out[3] culling blocks per SM.  Returns
 * GRCA_ERR_INVALID_ARG for bad ids, counts or flags. */
grca_status grca_get_launch_config(grca_ctx* ctx, const int32_t* sensor_ids, uint32_t n_sensors, uint32_t flags,
                                  int32_t out[4]);

/* Hybrid static/dynamic pipeline (Sec. 7): build a bounding-volume hierarchy
 * over triangles [0, n_static) of the uploaded set (binned SAH on the host,
 * once; blocks until done).  Casts then trace those triangles through the
 * hierarchy, one GPU thread per ray, and the rest through the culls; both
 * sides commit into the same closest-hit keys, so the merge is the key
 * minimum on the GPU and the result is the same as without the hierarchy.
 * A cast falls back to the culls for every triangle when the static
 * triangles were uploaded or updated after the build, when a sensor's
 * farthest scene point is more than ~1.25 scene diagonals away, or with the
 * BRUTE, LOSSY_AREA, DUMP_CANDIDATES or NO_STATIC_BVH flags.  n_static = 0
 * drops the hierarchy.  Returns GRCA_ERR_INVALID_ARG if n_static exceeds
 * the uploaded count and GRCA_ERR_CAPACITY if the tree would be deeper than
 * the traversal stack (64). */
grca_status grca_build_static(grca_ctx* ctx, uint32_t n_static, void* stream);

/* Non-spinning and patterned sensors (App. A.3, animated ray-mask images):
 * an on/off mask over the sensor's channel x ray grid.  `bits` holds
 * ceil(n_channels*n_rays/32) uint32 words; bit (q & 31) of word q >> 5, with
 * q = j*n_rays + i, set = ray (j, i) fires.  Rays that do not fire report a
 * miss (+inf, 0xFFFFFFFF) at their usual, stable output index.  `where` =
 * GRCA_MEM_HOST (copied before return) or GRCA_MEM_DEVICE (copied on
 * `stream`; the source may be reused once that stream reaches the copy).
 * bits = NULL removes the mask.  Call again between casts to animate it.
 * Returns GRCA_ERR_INVALID_ARG for a bad id or `where`. */
grca_status grca_set_ray_mask(grca_ctx* ctx, int32_t sensor_id, const uint32_t* bits, int where, void* stream);

/* Horizontal angular noise (App. A.1, Eq. noise_search): per-ray azimuths
 * theta[i] (radians, n_rays host doubles, copied) that replace theta0 +
 * i*dtheta, each strictly within dtheta of its nominal value so that the
 * search window of a ray stays its nominal index +-1.  Spans widen by the
 * largest perturbation; the ray tests use the perturbed directions.
 * theta = NULL restores the uniform grid.  Returns GRCA_ERR_INVALID_ARG when
 * a value is not finite or lies dtheta or more from its nominal azimuth.
 * (Per-channel vertical noise needs no call: give the perturbed, still
 * ascending elevations as the sensor's elevation table.) */
grca_status grca_set_sensor_azimuths(grca_ctx* ctx, int32_t sensor_id, const double* theta);

/* Range noise (App. A.1, applied after output conversion): each hit
 * distance of the sensor gets sigma * z added, with z = sqrt(-2 ln u1)
 * cos(2 pi u2) (Box and Muller, 1958), u1 = (hi24(a) + 1) / 2^24,
 * u2 = hi24(b) / 2^24, a = splitmix64(seed + 2q), b = splitmix64(seed + 2q + 1),
 * q = j*n_rays + i the ray's index within the sensor, hi24 the top 24 bits
 * and splitmix64 the output function of SplitMix64 (Steele, Lea and Flood,
 * 2014) for the state x: mix(x + 0x9E3779B97F4A7C15).  z is evaluated in
 * FP32.  sigma = 0 turns it off; change the seed per frame for fresh noise.
 * Returns GRCA_ERR_INVALID_ARG for a bad id or a negative or non-finite sigma. */
grca_status grca_set_range_noise(grca_ctx* ctx, int32_t sensor_id, double sigma, uint64_t seed);

/* Allocation-free cast of one sensor.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc (for example
 * code running inside an allocator or memory-pool callback, a plugin whose
 * host forbids device allocations after start-up, or a real-time loop that
 * must not wait on the driver's allocator).  It needs no context and
 * allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * Its scratch memory (per-ray closest-hit keys, ray tables, counters) is one
 * fixed device array of about 2.4 MB inside the library, present on every
 * GPU that loads the library until the process exits.
 *   sensor   : checked as by grca_create_sensor (read during the call only).
 *   tris     : DEVICE pointer, n_tris FP32 triangles [n][3][3], 16-byte
 *              aligned (else GRCA_ERR_INVALID_ARG); read up to its last
 *              float only, so the buffer needs no padding.
 *   out_dist, out_tri : DEVICE arrays of n_channels*n_rays entries, same
 *              layout and miss convention as grca_cast.
 *   flags    : 0 or GRCA_CAST_CULL_BACKFACE; the plain FP32 test is used.
 * Limits: n_channels <= 256, n_rays <= 32768, n_channels*n_rays <= 262144;
 * larger sizes return GRCA_ERR_CAPACITY, other bad arguments
 * GRCA_ERR_INVALID_ARG.
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Every call on a device shares the one
 * array (each call resets what must start empty): calls that overlap on the
 * GPU (different streams, or different host threads) race and corrupt each
 * other's results.
 * Errors: the return value reports argument errors and this call's kernel
 * launch errors (an error left by an earlier launch is cleared first).  No
 * device-side error can arise: every candidate span is tested inline, so the
 * call has no work queue that could overflow.  Spans are not split across
 * threads here, so a triangle that covers many rays (ground under the sensor)
 * is tested by one thread and lengthens the call; grca_cast balances such
 * pairs over many threads. */
grca_status grca_cast_noalloc(const grca_sensor_desc* sensor, const float* tris, uint32_t n_tris, float* out_dist,
                              uint32_t* out_tri, uint32_t flags, void* stream);

/* Debug dump for GRCA_CAST_DUMP_CANDIDATES: a DEVICE buffer of `capacity`
 * (global ray id, triangle id) uint32 pairs and a DEVICE uint32 counter
 * (caller zeroes it).  Pass NULLs to detach. */
grca_status grca_set_debug_dump(grca_ctx* ctx, uint32_t* pairs, uint64_t capacity, uint32_t* counter);

/* Counters and device error bits of the last cast; synchronizes `stream`.
 * Returns GRCA_ERR_CAPACITY if a work queue overflowed in that cast. */
grca_status grca_get_stats(grca_ctx* ctx, grca_stats* out, void* stream);

/* Number of kernels the last cast launched (or replayed in its graph), plus
 * the group-bound kernels that vertex uploads and updates launched since the
 * cast before it. */
uint32_t grca_last_launch_count(grca_ctx* ctx);

/* Per-kernel timing with CUDA events (tracing aid).  While enabled, casts
 * are launched without graph replay and each kernel of the frame is
 * bracketed by two events recorded on the cast's stream.  Enabling or
 * disabling resets the totals. */
grca_status grca_profile_enable(grca_ctx* ctx, int enable);

/* Totals since grca_profile_enable: for kernel k < min(max, *n_out) of the
 * frame sequence (k_init, k_cull_a, k_cull_b, k_expand, k_test, k_bvh,
 * k_refine, k_recheck_filter, k_recheck_rays, k_recheck_pairs, k_decode),
 * its name (static string), number of launches and
 * summed device time in ms.  Synchronizes with the recorded events.
 * *n_out receives the number of kernel kinds. */
grca_status grca_profile_read(grca_ctx* ctx, uint32_t max, const char** names, uint64_t* launches,
                              double* total_ms, uint32_t* n_out);

/* Static description of a status code. */
const char* grca_status_string(grca_status status);

/* Text of the last CUDA error seen by this context ("" if none). */
const char* grca_last_cuda_error(grca_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GRCA_H */
