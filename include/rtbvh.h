/*
 * rtbvh -- closest-hit and any-hit ray queries against triangulated scenes
 * through a BVH whose splits use the hybrid surface-area + distance cost of
 * Wang et al., "An Improved Ray Tracing Acceleration Algorithm Based on
 * Bounding Volume Hierarchies" (arXiv 2208.10008).  GB300 (sm_103a) only.
 *
 * Conventions for every entry point
 *  - Return 0 (RT_OK) on success, a negative RT_E* code on failure;
 *    rt_last_error() then gives a message (thread-local, valid until the
 *    next call from the same thread).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it and the call returns without waiting,
 *    unless the comment says "synchronous".  Inputs must not change and
 *    outputs must not be read until the stream has reached the call.
 *  - Buffers named *_dev are device pointers owned by the caller.  Handles
 *    (rt_scene, rt_session) are owned by the library and freed by their
 *    *_destroy call.
 *  - Triangle ids are input order: triangle i is tris[9i .. 9i+8].  The
 *    library's internal reordering is never visible.
 *  - A scene's calls must be issued from one host thread at a time; calls on
 *    different scenes may run concurrently.
 */
#ifndef RTBVH_H
#define RTBVH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT_OK 0
#define RT_EINVAL (-1)     /* bad argument (null handle, negative size, bad params) */
#define RT_ENOMEM (-2)     /* device or host allocation failed */
#define RT_ENOTBUILT (-3)  /* trace on a scene whose BVH has not been built */
#define RT_ETIMEOUT (-4)   /* a bounded device wait ran out (status word set) */
#define RT_ECUDA (-5)      /* a CUDA runtime call failed */
#define RT_EBUSY (-6)      /* resource in use (session admission) */
#define RT_EINTERNAL (-7)  /* a device-side consistency check failed */

typedef struct rt_scene_s* rt_scene;
typedef struct rt_session_s* rt_session;

/* One ray, 32 bytes, 16-byte aligned arrays.  Points o + t d with
 * tmin < t < tmax are on the ray.  d need not be unit length; t is in units
 * of |d|.  A ray with a non-finite component, or tmax <= tmin, misses. */
typedef struct {
  float ox, oy, oz, tmin;
  float dx, dy, dz, tmax;
} rt_ray;

/* Closest-hit result, 16 bytes.  Miss: t = +inf, tri = -1, u = v = 0.
 * (u, v) are the barycentric weights of vertices 1 and 2 of the hit
 * triangle (the point is (1-u-v) v0 + u v1 + v v2). */
typedef struct {
  float t;
  int32_t tri;
  float u, v;
} rt_hit;

/* Build parameters (Sec. II.B-C).  Split cost of children A, B of node C:
 *   alpha (S(A)/S(C) k_A t_i + S(B)/S(C) k_B t_i) + (1 - alpha) d^2 + t_trav
 * (Eq. 2; Eq. 1 when alpha = 1) with S the AABB surface area (Eq. 3 boxes),
 * k the triangle counts and d^2 = (d_A^2 + d_B^2)/2, d_X the distance from
 * the centre of X's AABB to `source`.  dist_norm = 1 replaces d^2 by
 * d^2 / diag(C)^2 * k_C t_i (scale-free); dist_norm = 2 by
 * (k_A d_A^2 + k_B d_B^2) / diag(C)^2 * t_i (scale-free, each child's
 * distance weighted by its triangles, as the SAH term weights its area);
 * 0 keeps the paper's raw m^2.
 * A node becomes a leaf when it holds at most max_leaf triangles. */
typedef struct {
  float alpha;      /* [0, 1] */
  float t_i;        /* > 0 */
  float t_trav;     /* >= 0 (never changes a split; kept for the cost report) */
  float source[3];  /* ray source point of Eq. 2 */
  int32_t max_leaf; /* 1 .. 15 */
  int32_t bins;     /* candidate planes per axis + 1: 4 .. 32 */
  int32_t width;    /* children per traversal node: 4 */
  int32_t dist_norm;/* 0, 1 or 2 */
  float range;      /* ray action range around `source` (Sec. II.B): > 0 builds over only the
                       triangles whose box lies within range of the source (no point of a path of
                       total length <= range is farther away, at any reflection order); 0 (or
                       +inf): all triangles.  Rays traced against such a tree must keep their
                       whole path within range of the source. */
  int32_t quantize; /* 1: also write the 64-byte traversal nodes (children's planes as bytes
                       on a per-axis power-of-two grid, rounded outward) that
                       RT_QUANTIZED_NODES walks; 0: only the 128-byte float nodes */
} rt_build_params;

/* Trace flags */
#define RT_NO_FP64_RETEST 1u /* skip the float64 re-test of flagged rays (diagnostics) */
#define RT_COUNT_STATS 2u    /* count nodes visited / triangles tested per ray */
#define RT_QUANTIZED_NODES 4u /* walk the 64-byte quantised nodes (the scene's last build had
                                 quantize = 1); the same hits, half the node bytes */

typedef struct {
  uint32_t flags;
  const int32_t* skip_tri_dev; /* nullable; per-ray triangle id to ignore (-1 = none),
                                  e.g. the triangle a reflected ray leaves from */
  uint32_t* stats_dev;         /* nullable; with RT_COUNT_STATS, per ray [nodes, tris] */
  int32_t* n_flagged_dev;      /* nullable; receives the number of rays the float32 pass
                                  flagged for the float64 re-test */
  int32_t block;               /* rays per CTA of the float32 walk (ray tile): 64, 128 or
                                  256; 0 = 128.  Results do not depend on it. */
  int32_t stack;               /* depth of the walk's per-ray stack: 16, 32 or 64; 0 = 64.
                                  A ray whose stack would overflow is finished by the
                                  float64 pass, so results do not depend on it. */
} rt_trace_params;

/* Build report (rt_bvh_info). */
typedef struct {
  int64_t n_tri;          /* triangles in the scene */
  int64_t n_bvh2_internal;/* binary internal nodes (Sec. II.C tree) */
  int64_t n_leaves;       /* leaves */
  int64_t n_wide;         /* traversal nodes */
  int32_t depth2;         /* depth of the binary tree (root = 1) */
  int32_t depth_wide;     /* depth of the traversal tree (root = 1) */
  int32_t max_leaf_size;  /* largest leaf */
  int32_t status;         /* device status word, 0 = ok */
  double build_ms;        /* device time of the last build (events) */
  int64_t n_built;        /* triangles in the tree (n_tri unless the build had a range) */
} rt_bvh_info_t;

/* Library version (major*10000 + minor*100 + patch). */
int rt_version(void);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all scenes, all threads).  Reading it twice around a region gives the
 * launches made inside it.  Never fails. */
uint64_t rt_launch_count(void);

/* Message of the last failed call on this thread ("" if none). */
const char* rt_last_error(void);

/* Copy a triangle soup into a new scene (Sec. II.A: buildings as triangular
 * facets).  tris: n_tri * 9 floats, vertex k of triangle i at
 * tris[9i + 3k .. 9i + 3k + 2]; a host pointer (is_device_ptr = 0; pageable
 * or pinned) or a device pointer (1).  The caller may free `tris` once the
 * stream has reached the call.  n_tri may be 0 (every ray then misses).
 * Errors: RT_EINVAL (out == NULL, n_tri < 0 or > 2^27), RT_ENOMEM,
 * RT_ECUDA. */
int rt_scene_upload(const float* tris, int64_t n_tri, int is_device_ptr, void* stream,
                    rt_scene* out);

/* Free a scene and every device buffer it owns (synchronous). */
int rt_scene_destroy(rt_scene scene);

/* Replace the vertex data of an existing scene with n_tri triangles (same
 * layout as rt_scene_upload).  The BVH must be rebuilt before tracing.
 * Errors: RT_EINVAL, RT_ENOMEM, RT_ECUDA. */
int rt_scene_update(rt_scene scene, const float* tris, int64_t n_tri, int is_device_ptr,
                    void* stream);

/* Build (or rebuild) the scene's BVH on the device (Sec. II.B-C, Fig. 2):
 * per-triangle AABBs (Eq. 3), scene bounds, a top-down split of every node
 * by the minimum of the Eq. 2 cost over `bins`-1 candidate planes on each
 * axis (nodes of at most 32 triangles: over the splits of the Morton order
 * of their box centres), leaves of at most max_leaf triangles, then a
 * collapse of the binary tree into `width`-ary traversal nodes.
 * Asynchronous: no host synchronisation, so it can be captured in a CUDA
 * graph once the scene's buffers exist (the first build of a scene
 * allocates them).  Errors: RT_EINVAL (bad params), RT_ENOMEM, RT_ECUDA. */
int rt_bvh_build(rt_scene scene, const rt_build_params* params, void* stream);

/* Instrumentation, with no counterpart in the paper: record the CUDA events
 * ev_begin and ev_end (cudaEvent_t passed as void*) on the build stream just
 * before and just after the split kernel (the recursion of Fig. 2, the
 * build's longest kernel) of every later rt_bvh_build of this scene, so
 * that the caller can time that kernel alone (cudaEventElapsedTime).  Both
 * NULL stops it.  Inside a stream capture the records become event-record
 * nodes of the graph.  The events stay the caller's and must outlive the
 * builds that record them.  Errors: RT_EINVAL (scene NULL, or only one of
 * the two events given). */
int rt_scene_set_split_events(rt_scene scene, void* ev_begin, void* ev_end);

/* Autotuner result (rt_autotune). */
typedef struct {
  int32_t max_leaf;   /* chosen leaf size */
  int32_t bins;       /* chosen bins per axis */
  int32_t block;      /* chosen ray tile of the walk (rt_trace_params.block) */
  int32_t n_tried;    /* configurations timed */
  float build_ms;     /* device time of one build with the choice */
  float trace_ms;     /* device time of one trace of the sample with the choice */
  float score_ms;     /* build_weight * build_ms + trace_ms */
  float default_score_ms; /* the same for width 4, max_leaf 4, bins 16, block 128, stack 64 */
  int32_t width;      /* chosen traversal node width (rt_build_params.width) */
  int32_t stack;      /* chosen stack depth of the walk (rt_trace_params.stack) */
} rt_tune_result;

/* Autotuner of the build and walk parameters (no counterpart in the paper),
 * in two stages: first the tree, width in {4, 8} x max_leaf in {2, 4, 6, 8}
 * x bins in {8, 16, 32} (alpha, t_i, t_trav, source, dist_norm, range kept
 * from `base`), each build timed and the closest-hit walk of the n_rays
 * sample rays (device pointer) timed with the default tile and stack; then,
 * on the chosen tree, the walk's ray tile in {64, 128, 256} x stack depth in
 * {16, 32, 64}.  Every timing is the median of 5 CUDA-event timings, each
 * after an untimed 256 MB write that evicts the L2 (cold-cache ranking); the
 * choice minimises build_weight * build_ms + trace_ms (build_weight = builds
 * per traced sample: 1 when the scene is rebuilt for every batch, 0 when it
 * is built once and traced many times).  Every configuration gives the same
 * hits (the hit rule does not depend on the tree or the walk).  On return
 * the scene holds the BVH built with the choice (never quantised).
 * Synchronous.  Allocates and frees one n_rays hit buffer and the 256 MB
 * eviction buffer (without it, when it cannot be had, the timings are
 * warm-cache).  Errors: RT_EINVAL (NULL arguments, n_rays < 1,
 * build_weight < 0, bad base params), RT_ENOMEM, RT_ECUDA. */
int rt_autotune(rt_scene scene, const rt_build_params* base, const rt_ray* rays_dev, int64_t n_rays,
                float build_weight, rt_tune_result* out, void* stream);

/* Instrumentation (no counterpart in the paper): enqueue one launch that
 * reads the device buffer buf_dev (`bytes`, a multiple of 16, 16-byte
 * aligned; small enough to stay in the L2, e.g. 24 MB) `reps` times with
 * 16-byte loads cached in the L2 only.  Timing it with events on `stream`
 * gives the L2 read bandwidth, bytes * reps / time, the ceiling of a walk
 * whose nodes and triangles stay in the L2.  sink_dev (nullable, one word
 * per block: 4 x the SM count) is written only to keep the loads; the buffer's
 * contents do not matter.  Errors: RT_EINVAL, RT_ECUDA. */
int rt_probe_l2_read(const void* buf_dev, int64_t bytes, int32_t reps, uint32_t* sink_dev, void* stream);

/* Test hooks (no counterpart in the paper): make failures happen on purpose,
 * without faulting the device, so that the error paths can be tested.
 * Process-wide; value 0 turns a hook off.
 *   RT_DEBUG_SPIN_LIMIT    polls a build's work-queue wait may make without
 *                          progress before it gives up (default 2^24)
 *   RT_DEBUG_PHANTOM_TASK  every later build counts this many subtree tasks
 *                          that are never published: its warps wait for them
 *                          until the spin limit, the build ends with the
 *                          timeout status (rt_bvh_info: RT_ETIMEOUT)
 *   RT_DEBUG_PHANTOM_ITEM  the same for big-node chunk items
 *   RT_DEBUG_FAIL_ALLOC    the value-th device allocation from now fails
 *                          (RT_ENOMEM) without calling the allocator
 * Errors: RT_EINVAL (unknown hook or negative value). */
#define RT_DEBUG_SPIN_LIMIT 1
#define RT_DEBUG_PHANTOM_TASK 2
#define RT_DEBUG_PHANTOM_ITEM 3
#define RT_DEBUG_FAIL_ALLOC 4
int rt_debug_inject(int hook, int64_t value);

/* Synchronous: wait for the stream, then report the built tree.  Counting
 * the traversal nodes reachable from the root takes a temporary device array
 * of their child references (16 bytes per node slot, 32 for 8-wide nodes),
 * read back to the host.  Errors: RT_EINVAL, RT_ENOTBUILT, RT_ENOMEM,
 * RT_ECUDA; RT_ETIMEOUT when a work-queue wait of the build ran out
 * (status 1); RT_EINTERNAL when the device status word reports a failed
 * check (info->status says which). */
int rt_bvh_info(rt_scene scene, void* stream, rt_bvh_info_t* info);

/* Synchronous: copy the binary tree (Sec. II.C, Fig. 1) to host arrays in
 * the neutral form used by the tests: node i has children child[2i],
 * child[2i+1] (>= 0: node index; < 0: leaf -1-l), leaf l covers
 * prims[leaf_first[l] .. + leaf_count[l]), prims holds triangle ids, node
 * 0 is the root (or leaf 0 when there is no internal node).  Array sizes
 * come from rt_bvh_info: child 2*n_bvh2_internal, leaf arrays n_leaves,
 * prims n_tri.  boxes (nullable) receives 12 floats per internal node: the
 * AABBs (lo xyz, hi xyz) of its two children. */
int rt_bvh_export(rt_scene scene, void* stream, int32_t* child, int64_t* leaf_first,
                  int64_t* leaf_count, int32_t* prims, float* boxes);

/* Closest hit for n rays (Sec. III.B, Fig. 4): descend through the boxes
 * the ray meets within [tmin, min(tmax, best t)], test the leaf triangles
 * and keep the nearest hit with tmin < t < tmax (ties: lowest triangle id).
 * The float32 pass flags rays whose answer its error bounds cannot settle
 * (a triangle edge or a second hit within the bound, a hit near tmin or
 * tmax); those are traced again in float64 with the same hit rule as the
 * reference definition (Moller-Trumbore, inclusive edges).
 * rays_dev: n rt_ray (16-byte aligned); hits_dev: n rt_hit.  n may be 0.
 * Errors: RT_EINVAL, RT_ENOTBUILT, RT_ENOMEM (first use of a larger n
 * grows the scene's re-test queue), RT_ECUDA. */
int rt_trace_closest(rt_scene scene, const rt_ray* rays_dev, int64_t n, rt_hit* hits_dev,
                     const rt_trace_params* params, void* stream);

/* Any hit for n rays: occluded_dev[i] = 1 when some triangle is hit with
 * tmin < t < tmax, else 0 (visibility between two points: o = p0,
 * d = p1 - p0, tmin = 0, tmax = 1).  Same flagging and float64 re-test as
 * rt_trace_closest.  Errors as rt_trace_closest. */
int rt_trace_any(rt_scene scene, const rt_ray* rays_dev, int64_t n, uint8_t* occluded_dev,
                 const rt_trace_params* params, void* stream);

/* Closest hit with HOST buffers: rays_host and hits_host are host memory
 * (pinned for overlap; pageable works but serialises).  The library copies
 * rays in chunks to device staging buffers and traces them, overlapping the
 * copies of one chunk with the tracing of another.  When hits_host is
 * 16-byte aligned page-locked memory mapped into the device's address space
 * (cudaHostAlloc / cudaMallocHost / a mapped registration, as reported by
 * cudaPointerGetAttributes), the walk writes the hit records straight into
 * it; otherwise hits go to device staging buffers and are copied back.
 * Synchronous with respect to the host buffers: on return, hits_host is
 * filled.  Of params (nullable) flags and block are used; skip_tri_dev and
 * stats_dev must be NULL and n_flagged_dev is not written.
 * Errors as rt_trace_closest. */
int rt_trace_closest_host(rt_scene scene, const rt_ray* rays_host, int64_t n, rt_hit* hits_host,
                          const rt_trace_params* params, void* stream);

/* Launch direction sets (Sec. III.A). */
#define RT_RAYS_FIBONACCI 0 /* param = number of rays N: z_i = 1 - (2i+1)/N, azimuth i pi (3 - sqrt 5);
                               launched in band order (rt_launch_index) */
#define RT_RAYS_ICOSPHERE 1 /* param = level L: vertices of the icosahedron with every edge cut into
                               f = 2^L, 10 f^2 + 2 rays; order: 12 corners, edge points, face points
                               row by row; launched in tile order (rt_launch_index) */

/* Number of rays of a launch (RT_RAYS_FIBONACCI: param; RT_RAYS_ICOSPHERE:
 * 10 * 4^param + 2); -1 for an invalid kind or param.  Never touches the GPU. */
int64_t rt_ray_count(int kind, int64_t param);

/* Fill rays_dev with the launch of Sec. III.A from `origin`: unit
 * directions (float32, formed with the azimuth reduced exactly in integer
 * arithmetic for RT_RAYS_FIBONACCI; the planar subdivision point normalised
 * for RT_RAYS_ICOSPHERE), tmin / tmax as given.  capacity must be at least
 * rt_ray_count(kind, param).  Icosphere levels 0..12.  Slot s holds
 * direction rt_launch_index(kind, param, s): rays come in band (Fibonacci)
 * or tile (icosphere) order, so that the 32 rays of a warp are neighbouring
 * directions.
 * Errors: RT_EINVAL, RT_ECUDA. */
int rt_gen_rays(int kind, const float* origin, int64_t param, float tmin, float tmax, rt_ray* rays_dev,
                int64_t capacity, void* stream);

/* Index, in the order of the RT_RAYS_* definitions, of the direction that
 * rt_gen_rays (and every batch or session launch) writes to slot `slot`;
 * -1 for an invalid kind, param or slot.  RT_RAYS_FIBONACCI with N rays:
 * w = the largest Fibonacci number (1, 2, 3, 5, 8, ...; w >= 2) with
 * w^2 <= 80 N, and c = the one of the two Fibonacci numbers before w that
 * has an even index (F_1 = F_2 = 1); slot b w + t with (b + 1) w <= N holds
 * direction b w + (t c mod w), which walks the w consecutive spiral points
 * of band b in order of azimuth; every later slot holds its own direction.
 * RT_RAYS_ICOSPHERE: corners and edge points keep their slots; each face's
 * interior (rows i = 1 .. f-2 of f-1-i points) is cut into bands of 8 rows,
 * and a band lists the columns all 8 rows hold as tiles of 8 rows x 4
 * columns (row by row inside a tile), then the rest of its rows row by row;
 * odd bands (counted from 0) list the rest first and the tiles from the last
 * to the first; the rows after the last full band follow row by row.  Never
 * touches the GPU. */
int64_t rt_launch_index(int kind, int64_t param, int64_t slot);

/* Specular bounce (Sec. III.B: a ray that meets a facet generates a
 * reflected ray) with compaction.  For every ray i whose hit has tri >= 0
 * and remaining range tmax - t > 0, in input order, writes the next ray
 * (o + t d, 0, d - 2 (d.n) n, tmax - t), n the unit geometric normal
 * (v1 - v0) x (v2 - v0) of the hit triangle, to out_rays_dev; the hit
 * triangle to out_skip_dev (pass it as skip_tri_dev when tracing the new
 * rays: a reflected ray never meets the facet it leaves); i to out_src_dev
 * (nullable); the number written to *out_count_dev (device int).  Output
 * arrays hold n entries.  Allocates per-scene scratch on first use of a
 * larger n.  Errors: RT_EINVAL, RT_ENOMEM, RT_ECUDA. */
int rt_reflect(rt_scene scene, const rt_ray* rays_dev, const rt_hit* hits_dev, int64_t n,
               rt_ray* out_rays_dev, int32_t* out_skip_dev, int32_t* out_src_dev,
               int32_t* out_count_dev, void* stream);

/* ---- reception (Sec. III.C, Eq. 4) ---------------------------------- */
typedef struct rt_rxset_s* rt_rxset;

/* One received path segment: the ray's index in the rays passed, the
 * receiver's index, the path length l from the source to the foot of the
 * perpendicular from the receiver (Eq. 4's l) and the receiver's distance
 * to the ray there. */
typedef struct {
  int32_t ray;
  int32_t rx;
  float l;
  float dist;
} rt_rx_record; /* 16 B */

typedef struct {
  float delta;         /* angle between adjacent rays at the source, radians (Eq. 4) */
  float range0;        /* the paths' initial ray action range; l = (range0 - tmax) + t* */
  int32_t max_records; /* capacity of out_dev, in records */
  int32_t reserved;    /* 0 */
  unsigned long long* stats_dev; /* nullable, device [2]: grid cells visited and receiver
                                    entries tested, summed over the rays (added to, not zeroed) */
  const float* delta_ray_dev;    /* nullable, device [n]: each ray's own delta (rays of
                                    transmitters launched with different counts); a value
                                    beyond the set's r_max * sqrt(3) / range0 is taken as that */
} rt_receive_params;

/* Receivers: rx_host = m * 3 floats (x, y, z), copied to the device into a
 * uniform grid in which every receiver is entered into each cell its largest
 * receiving sphere (radius r_max) overlaps.  Synchronous.  Errors:
 * RT_EINVAL (NULL, m outside 1..2^26, r_max not positive and finite,
 * non-finite position), RT_ENOMEM, RT_ECUDA. */
int rt_rxset_create(const float* rx_host, int32_t m, float r_max, rt_rxset* out);

/* Free a receiver set (synchronous). */
int rt_rxset_destroy(rt_rxset rs);

/* Receiving-sphere test of Sec. III.C (Eq. 4) for the path segments of n
 * rays: ray i covers t in [tmin, tend), tend = min(hits[i].t, tmax) (a
 * miss: tmax), and receives at receiver p when the foot of the
 * perpendicular from p, t* = (p - o).d / (d.d), lies in [tmin, tend) and
 * |p - (o + t* d)| <= l delta / sqrt(3) with l = (range0 - tmax) + t*
 * (every bounce leaves the remaining range in tmax; directions have unit
 * length, as rt_gen_rays and rt_reflect make them).  Each (ray, receiver)
 * pair is reported once, in no particular order, as an rt_rx_record in
 * out_dev; *count_dev (device int, zeroed by the call) receives the number
 * of pairs found, which may exceed max_records (the records past it are
 * dropped).  n_dev (nullable, device int): the number of valid rays when it
 * is smaller than n (a compacted order of rt_batch_order).  Rays with a
 * non-finite component or tmax <= tmin receive nothing.  Asynchronous on
 * `stream`.  Errors: RT_EINVAL (NULL buffers, n out of range, delta or
 * range0 not positive and finite, range0 * delta / sqrt(3) > the set's
 * r_max, max_records < 0), RT_ECUDA. */
int rt_receive(rt_rxset rs, const rt_ray* rays_dev, const rt_hit* hits_dev, int64_t n, const int32_t* n_dev,
               const rt_receive_params* params, rt_rx_record* out_dev, int32_t* count_dev, void* stream);

/* ---- binding check ----------------------------------------------------- */
/* sizeof of every public struct, for bindings to check their mirrors
 * against, in this order: rt_ray, rt_hit, rt_build_params, rt_trace_params,
 * rt_bvh_info_t, rt_tune_result, rt_rx_record, rt_receive_params,
 * rt_batch_desc, rt_batch_stats, rt_request, rt_session_stats.  Writes
 * min(n, 12) values to sizes (host) and returns 12.  Needs no GPU. */
int rt_abi_struct_sizes(int64_t* sizes, int32_t n);

/* ---- batched multi-bounce tracing ------------------------------------ */
typedef struct rt_batch_s* rt_batch;

#define RT_BATCH_MAX_ORDER 8

/* Many transmitters with uneven ray counts, traced with up to max_order
 * specular reflections each (Sec. III.B: paths stop at the order limit or
 * when the ray action range tmax is used up) plus the visibility of every
 * transmitter-receiver pair (any hit on the segment). */
typedef struct {
  int32_t n_tx;
  const float* tx_pos;     /* host, n_tx * 3 */
  const int64_t* tx_param; /* host, n_tx: rays per transmitter (RT_RAYS_FIBONACCI) or level */
  int32_t dir_kind;        /* RT_RAYS_FIBONACCI or RT_RAYS_ICOSPHERE */
  int32_t max_order;       /* reflections after the direct rays: 0 .. RT_BATCH_MAX_ORDER */
  float tmax;              /* ray action range: total length of every path */
  int32_t n_rx;            /* receivers (0: no visibility pass) */
  const float* rx_pos;     /* host, n_rx * 3 */
  int32_t use_graph;       /* 1: capture the pipeline in a CUDA graph on the second run, replay after */
  int32_t ray_tile;        /* rt_trace_params.block of every walk of the batch (0 = default),
                              e.g. rt_autotune's choice */
  int32_t receive;         /* 1: receiving spheres (Sec. III.C, Eq. 4) of every order's
                              segments against the receivers (n_rx > 0) */
  int32_t max_rx_records;  /* records kept per order when receive = 1 */
  const float* rx_delta;   /* host, n_tx (nullable): delta of each transmitter's launch; NULL:
                              icosphere atan(2) / 2^level, Fibonacci sqrt(4 pi / N) */
} rt_batch_desc;

typedef struct {
  int32_t n_orders;                     /* max_order + 1 */
  int64_t rays[RT_BATCH_MAX_ORDER + 1]; /* rays traced in each order */
  int64_t segments;                     /* visibility segments (n_tx * n_rx) */
  int64_t total_rays;                   /* all orders + segments */
  int64_t visible;                      /* segments with no hit */
  int32_t flagged;                      /* float64 re-tests of the last trace (diagnostic) */
  int64_t received[RT_BATCH_MAX_ORDER + 1]; /* received pairs of each order (receive = 1) */
} rt_batch_stats;

/* Allocate everything the pipeline needs for these transmitters on `scene`
 * (whose BVH must be built before rt_batch_run): per order k a ray queue, a
 * hit array, the skip and parent-index arrays, and the visibility segments
 * d = rx - tx, t in (0, 1).  Synchronous.  Errors: RT_EINVAL, RT_ENOMEM,
 * RT_ECUDA. */
int rt_batch_create(rt_scene scene, const rt_batch_desc* desc, rt_batch* out);

/* Run the whole pipeline ordered after the work already on `stream`:
 * launch the rays of every transmitter (Sec. III.A) into one queue, trace
 * closest hits, then max_order times reflect + compact on the device
 * (rt_reflect) and trace the survivors (counts never leave the device),
 * then the visibility segments (rt_trace_any).  Work runs on the batch's
 * own stream; `stream` waits for it.  Results stay valid until the next run
 * starts.  With use_graph the second run captures the pipeline and later
 * runs replay it; the scene may be updated and rebuilt between runs (not
 * during one), and a run after a change that moved the scene's arrays or
 * changed its tree size captures the pipeline again.
 * Errors: RT_EINVAL, RT_ENOTBUILT, RT_ECUDA. */
int rt_batch_run(rt_batch batch, void* stream);

/* Synchronous: wait for `stream` and the batch, report counts. */
int rt_batch_stats_get(rt_batch batch, void* stream, rt_batch_stats* stats);

/* Device pointers of order k's rays, hits, parent indices (into order k-1;
 * NULL for k = 0) and device ray count (NULL for k = 0: every launched ray).
 * Valid until rt_batch_destroy. */
int rt_batch_order(rt_batch batch, int order, const rt_ray** rays_dev, const rt_hit** hits_dev,
                   const int32_t** src_dev, const int32_t** count_dev);

/* Device array [n_tx * n_rx] (transmitter-major): 1 = segment blocked. */
int rt_batch_visibility(rt_batch batch, const uint8_t** occluded_dev);

/* Device pointers of order k's reception records (rt_receive's layout; ray
 * indices into order k's rays) and of its device count (may exceed
 * max_rx_records; the records past it are dropped).  Errors: RT_EINVAL
 * (bad order, or the batch was created without receive). */
int rt_batch_received(rt_batch batch, int order, const rt_rx_record** records_dev, const int32_t** count_dev);

/* Free the batch (synchronous). */
int rt_batch_destroy(rt_batch batch);

/* ---- serving --------------------------------------------------------- */
/* A trace request: one transmitter's launch on a resident scene, traced
 * with up to max_order reflections (Sec. III). */
typedef struct {
  int32_t scene_id;          /* from rt_session_add_scene */
  float tx[3];               /* transmitter (ray source point) */
  int32_t dir_kind;          /* RT_RAYS_FIBONACCI or RT_RAYS_ICOSPHERE */
  int64_t param;             /* ray count or icosphere level */
  int32_t max_order;         /* 0 .. RT_BATCH_MAX_ORDER */
  float tmax;                /* ray action range */
  rt_hit* hits_host;         /* nullable: receives the closest hits of the launched rays */
  int64_t* order_counts_host;/* nullable: receives rays traced per order [max_order + 1] */
  rt_hit* const* order_hits_host; /* nullable: host array of max_order + 1 pointers; entry k
                                     (k >= 1, nullable) receives the closest hits of the
                                     order-k reflected rays, in the order of their parents
                                     (order_counts_host[k] of them; room for the launch's
                                     ray count); entry 0 is not used (see hits_host) */
  int32_t* const* order_src_host; /* nullable: like order_hits_host; entry k (k >= 1) receives
                                     the index of each order-k ray's parent among the
                                     order-(k-1) rays */
} rt_request;

typedef struct {
  int64_t submitted, completed, failed, queued, running, peak_running;
  int64_t rays;              /* rays traced by completed requests (all orders) */
  int64_t pool_bytes, peak_pool_bytes;
  double p50_ms, p99_ms, mean_ms; /* submit-to-completion latency of the last
                                     2^20 completed requests */
  double span_s;             /* first submit to last completion */
  double wait_p50_ms, wait_p99_ms; /* of the same requests: submit to admission (queue wait) */
  double run_p50_ms, run_p99_ms;   /* and admission to completion (on the device, results copied) */
} rt_session_stats;

/* Create a serving session: one device pool of pool_bytes (allocated now)
 * and max_slots concurrent requests (1..64), each on its own stream.  A
 * worker thread admits queued requests in arrival order whenever a slot is
 * free and the pool holds all of the request's buffers (rays, hits, skip and
 * parent arrays per order, re-test scratch: about n * (56 (max_order + 1) + 44)
 * bytes for n rays), so requests of uneven sizes run side by side on the
 * device.  The calling thread's current device is used.
 * Errors: RT_EINVAL, RT_ENOMEM, RT_ECUDA. */
int rt_session_create(size_t pool_bytes, int max_slots, rt_session* out);

/* Make a scene (BVH already built) available to requests; *scene_id is its
 * index.  The scene must outlive the session and must not be rebuilt while
 * requests run.  Errors: RT_EINVAL, RT_ENOTBUILT. */
int rt_session_add_scene(rt_session session, rt_scene scene, int32_t* scene_id);

/* Queue a request (the struct is copied; hits_host / order_counts_host must
 * stay valid until the request completes).  Never blocks on the device.
 * Errors: RT_EINVAL, RT_ENOMEM (the request can never fit the pool). */
int rt_session_submit(rt_session session, const rt_request* req, uint64_t* ticket);

/* *done = 1 once the request's results are in its host buffers.
 * Errors: RT_EINVAL (unknown ticket), RT_ECUDA (the request failed). */
int rt_session_poll(rt_session session, uint64_t ticket, int* done);

/* Block until the request completes, or timeout_ns (< 0: no limit).
 * Errors: RT_EINVAL, RT_ETIMEOUT, RT_ECUDA. */
int rt_session_wait(rt_session session, uint64_t ticket, int64_t timeout_ns);

/* Forget a finished request: its record is freed and the ticket is unknown
 * from then on.  Its results stay in the caller's host buffers.  A session
 * keeps every request until it is released (or the session destroyed), so
 * a long-running server releases each ticket once it has read the results.
 * Errors: RT_EINVAL (unknown ticket), RT_EBUSY (still queued or running). */
int rt_session_release(rt_session session, uint64_t ticket);

/* Counters (totals since creation) and latency percentiles. */
int rt_session_stats_get(rt_session session, rt_session_stats* stats);

/* Finish queued and running requests, stop the worker, free the pool. */
int rt_session_destroy(rt_session session);

/* Largest batch rt_trace_closest_noalloc accepts. */
#define RT_NOALLOC_MAX_RAYS 262144

/* Closest hit without any device allocation.  (An addition of this library;
 * the paper has no counterpart.)  Same arguments and results as
 * rt_trace_closest, for callers that must not let the library allocate
 * device memory: a runtime that manages all device memory through its own
 * pool, or a latency-critical stream where a cudaMalloc (which can
 * synchronise the device) would stall other work.  The scratch for the
 * float64 re-test comes from one fixed array compiled into the library
 * (10 MiB on every GPU that loads it, held until the process exits), not
 * from the scene.
 *  - n must not exceed RT_NOALLOC_MAX_RAYS; larger batches return
 *    RT_EINVAL ("split the batch").
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the one array: calls whose work overlaps on the GPU
 *    (other streams, other host threads) race with each other.  Issue them
 *    on one stream or order them with events.
 *  - The scene's BVH must already be built (building allocates), and the
 *    device the scene was uploaded on must be current (RT_EINVAL otherwise).
 *  - The array's address is looked up once per device and kept: after a
 *    device reset (cudaDeviceReset), which invalidates every scene, this
 *    call must not be used again in the same process.
 * Errors: RT_EINVAL, RT_ENOTBUILT, RT_ECUDA. */
int rt_trace_closest_noalloc(rt_scene scene, const rt_ray* rays_dev, int64_t n, rt_hit* hits_dev,
                             const rt_trace_params* params, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RTBVH_H */
