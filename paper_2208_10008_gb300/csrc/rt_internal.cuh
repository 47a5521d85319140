// Internal definitions shared by the CUDA translation units of librtbvh.
//
// Device data layout (all 16-byte aligned, in HBM):
//   tri_in    float4[3T]  input-order triangles: (v0.xyz, id) (v1.xyz, 0) (v2.xyz, 0)
//   rec       float4[2T]  build records (lo.xyz, id) (hi.xyz, morton key): the Eq. 3
//                         box of a triangle; every partition moves them so each
//                         node's records are contiguous (ping-pong pair)
//   node2     Node2[T]    binary tree of Sec. II.C / Fig. 1; internal node id =
//                         (split position - 1), a unique slot for every split
//   link2     int2[T]     (parent id, build epoch) of every binary node: the epoch
//                         marks the nodes written by the latest build
//   wide      WNode[T]    4-wide traversal nodes, one 128-byte line each, stored at
//                         the id of the binary node they are rooted at
//   tri_leaf  float4[3T]  triangles in leaf order, same packing as tri_in
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <exception>
#include <new>

#include "rtbvh.h"

namespace rt {

// Sets the calling thread's rt_last_error message; returns code.
int set_error(int code, const char* msg);

// Runs the body of a C-ABI entry point that allocates host memory: a C++
// exception (a failed allocation) becomes an error code instead of crossing
// the C ABI, where it would terminate the caller.
template <class F>
int abi_guard(F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return set_error(RT_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return set_error(RT_EINTERNAL, e.what());
  } catch (...) {
    return set_error(RT_EINTERNAL, "unexpected host exception");
  }
}

constexpr int kMaxLeaf = 15;   // leaf refs pack the count in 4 bits
constexpr int kMaxBins = 32;
constexpr int kWidth = 4;           // default children per traversal node (8 on request)
constexpr int kMicro = 32;          // nodes up to this size are finished by one warp
constexpr int kSpinLimit = 1 << 24; // bounded device waits (iterations of ~200 ns)

// Status codes written to the device status word (BuildCtl::status).
enum DevStatus : int {
  kStOk = 0,
  kStQueueTimeout = 1,   // a work-queue wait hit kSpinLimit
  kStQueueOverflow = 2,  // more tasks than queue slots (cannot happen for a valid tree)
  kStBadSplit = 3,       // a partition disagreed with its bin counts
  kStWideOverflow = 4,   // more traversal nodes than allocated
  kStBadLink = 5,        // a binary node refers to a node this build never wrote
};

// Leaf reference: -1 - (first * 16 + count); internal: >= 0.
__host__ __device__ inline int32_t leaf_ref(int32_t first, int32_t count) {
  return -1 - (first * 16 + count);
}
__host__ __device__ inline int32_t leaf_first(int32_t ref) { return (-1 - ref) >> 4; }
__host__ __device__ inline int32_t leaf_count(int32_t ref) { return (-1 - ref) & 15; }

// Binary node: the AABBs of its two children; a_lo.w / b_lo.w hold the
// child refs (int bits), a_hi.w / b_hi.w hold the children's triangle counts.
struct __align__(16) Node2 {
  float4 a_lo, a_hi, b_lo, b_hi;
};

// 4-wide traversal node, 128 bytes: child i's box in component i of the six
// float4 planes; child[i] = wide node index (>= 0), leaf ref (< 0, != INT_MIN)
// or INT_MIN for an empty slot (whose box is lo = +inf, hi = -inf).
// meta.x = binary parent of the node's root (-1 at the root), rest unused.
struct __align__(16) WNode {
  float4 lox, hix, loy, hiy, loz, hiz;
  int4 child;
  int4 meta;
};
static_assert(sizeof(WNode) == 128, "wide node must be one 128-byte line");

// 8-wide traversal node, 256 bytes (two lines): child i's box in component
// i % 4 of plane[.][i / 4]; child refs as in WNode (INT_MIN: empty slot,
// box lo = +inf, hi = -inf); meta[0].x = binary parent of the node's root.
struct __align__(16) WNode8 {
  float4 lox[2], hix[2], loy[2], hiy[2], loz[2], hiz[2];
  int4 child[2];
  int4 meta[2];
};
static_assert(sizeof(WNode8) == 256, "8-wide node must be 256 bytes");

// The same 4-wide node in 64 bytes: the children's planes as bytes on a
// per-axis grid of step 2^e from the union box's lower corner (origin).
// A plane decodes as qplane(q, e, origin); a child's decoded box contains its
// exact box (lower planes rounded down, upper ones up, checked with the
// decoding itself when the node is written), so a slab test on the decoded
// planes is conservative.  Empty slots have child ref INT_MIN.
struct __align__(16) QNode {
  float ox, oy, oz;
  int exps;              // (e_x + 128) | (e_y + 128) << 8 | (e_z + 128) << 16
  unsigned lox, hix, loy, hiy;  // byte i: child i's plane
  unsigned loz, hiz;
  int parent, pad;
  int4 child;
};
static_assert(sizeof(QNode) == 64, "quantised node must be 64 bytes");

// 2^e for e in [-126, 127] (a normal float, exact).
__device__ __forceinline__ float qscale(int e) { return __int_as_float((e + 127) << 23); }
// The value of byte q of a plane on the grid (origin, 2^e); q * 2^e is
// exact, so the one rounding is the fused add.
__device__ __forceinline__ float qplane(unsigned q, float scale, float origin) {
  return __fmaf_rn(__int_as_float(0x4B000000u | q) - 8388608.f, scale, origin);
}

// Specular bounce (Sec. III.B) of the ray (ra = origin, tmin; rb = direction,
// tmax) at its hit t on triangle (a, b, c): origin o + t d, direction
// d - 2 (d.n) n about the unit geometric normal n of (b - a) x (c - a), the
// range left tmax - t.  Every operation is rounded explicitly, so every
// kernel that bounces a ray writes the same bits.
__device__ __forceinline__ void reflect_ray(float4 ra, float4 rb, float t, float4 a, float4 b, float4 c,
                                            float4* o0, float4* o1) {
  const float e1x = __fsub_rn(b.x, a.x), e1y = __fsub_rn(b.y, a.y), e1z = __fsub_rn(b.z, a.z);
  const float e2x = __fsub_rn(c.x, a.x), e2y = __fsub_rn(c.y, a.y), e2z = __fsub_rn(c.z, a.z);
  float nx = __fsub_rn(__fmul_rn(e1y, e2z), __fmul_rn(e1z, e2y));
  float ny = __fsub_rn(__fmul_rn(e1z, e2x), __fmul_rn(e1x, e2z));
  float nz = __fsub_rn(__fmul_rn(e1x, e2y), __fmul_rn(e1y, e2x));
  const float inv = rsqrtf(__fadd_rn(__fadd_rn(__fmul_rn(nx, nx), __fmul_rn(ny, ny)), __fmul_rn(nz, nz)));
  nx = __fmul_rn(nx, inv);
  ny = __fmul_rn(ny, inv);
  nz = __fmul_rn(nz, inv);
  const float k = __fmul_rn(2.f, __fadd_rn(__fadd_rn(__fmul_rn(rb.x, nx), __fmul_rn(rb.y, ny)), __fmul_rn(rb.z, nz)));
  *o0 = make_float4(__fmaf_rn(t, rb.x, ra.x), __fmaf_rn(t, rb.y, ra.y), __fmaf_rn(t, rb.z, ra.z), 0.f);
  *o1 = make_float4(__fsub_rn(rb.x, __fmul_rn(k, nx)), __fsub_rn(rb.y, __fmul_rn(k, ny)),
                    __fsub_rn(rb.z, __fmul_rn(k, nz)), __fsub_rn(rb.w, t));
}

struct __align__(16) Task {
  int32_t begin, count, parent, side;  // parent: node2 id (-1 root); side 0/1
  float clo[3];                        // centroid bounds of the task's triangles
  int32_t depth;
  float chi[3];
  int32_t pad;
};

// A node of more than `big` triangles, split by several CTAs at once (one
// per chunk of its range): its range, centroid bounds, its chunks' count
// slots and what it reserved for its children (task slots, count slots).
struct __align__(16) TopTask {
  int32_t begin, count, parent, side;
  float clo[3];
  int32_t depth;
  float chi[3];
  int32_t nchunk;       // ceil(count / chunk)
  int32_t chunk_first;  // count slots of this task's chunks (written by its parent's chunks)
  int32_t child_slot;   // 2 task slots reserved for the children
  int32_t chunk_res;    // nchunk + 2 count slots reserved for the children's chunks
  int32_t parity;       // record buffer holding this task's range
};

// Device control block of one scene (zeroed at the start of every build).
// The words every waiting CTA polls share one 128-byte line; the pool
// counters and the tree facts, updated by atomics, sit on lines of their own.
struct BuildCtl {
  int status, status_where, epoch, wide_root;
  // chunk items of top tasks (CTA per item)
  int ti_head, ti_tail, ti_pending, pad0;
  // subtree task queue (CTA per task)
  int qa_head, qa_tail, qa_pending, pad3;
  int pad_a[20];
  // pools of one build: top task slots, count slots
  int t_slot_next, t_cnt_next, pad1, pad2;
  int pad_b[28];
  // tree facts
  int n_internal, n_leaves, depth2, max_leaf_size;
  int root_ref, pad4, pad5, pad6;
  // scene bounds, order-preserving unsigned codes, max-reduced (0 = empty):
  // [0..2] ~code(box lo), [3..5] code(box hi), [6..8] ~code(centre lo), [9..11] code(centre hi)
  unsigned sb[12];
};

// Launch geometry of a build of T triangles (host side; also sizes the buffers).
struct BuildGeom {
  int big;        // nodes of more than `big` triangles are split chunk-parallel
  int chunk;      // records per chunk (one CTA's share of a big node)
  int rpt;        // records per thread in a chunk (chunk / 256)
  int cap_t;      // top task slots
  int cap_c;      // count slots and chunk items
  int qa_cap;     // subtree queue slots
};
BuildGeom build_geometry(int64_t n_tri, int nsm);

// Per-call trace scratch: counter + queue of flagged ray indices.
struct TraceScratch {
  int* counter = nullptr;   // [0] flagged count, [1] status
  int* queue = nullptr;     // flagged ray indices
  int* cand = nullptr;      // per queue slot: 1 + kTraceCand ints
  int64_t cap = 0;
};
constexpr int kTraceCand = 8;

// Order-preserving float <-> int map for atomicMin/atomicMax on floats.
__host__ __device__ inline int ford(float f) {
#ifdef __CUDA_ARCH__
  int i = __float_as_int(f);
#else
  int i;
  memcpy(&i, &f, 4);
#endif
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__host__ __device__ inline float iford(int i) {
  int j = i >= 0 ? i : i ^ 0x7FFFFFFF;
#ifdef __CUDA_ARCH__
  return __int_as_float(j);
#else
  float f;
  memcpy(&f, &j, 4);
  return f;
#endif
}

// Host-side count of kernel launches (rt_launch_count); every launch site
// adds the number of kernels it enqueues.
void count_launches(int k);

// Test hooks of rt_debug_inject (process-wide).
struct DebugHooks {
  int spin_limit;     // 0: kSpinLimit
  int phantom_tasks;  // subtree tasks counted but never published
  int phantom_items;  // big-node chunk items counted but never published
};
DebugHooks debug_hooks();

// Launch helpers implemented in build.cu / trace.cu -----------------------
struct SceneDev;  // forward

cudaError_t launch_build(struct ::rt_scene_s* s, const rt_build_params& p, cudaStream_t st);
cudaError_t launch_trace(struct ::rt_scene_s* s, const rt_ray* rays, int64_t n, rt_hit* hits,
                         uint8_t* occl, const rt_trace_params* tp, TraceScratch& scr,
                         cudaStream_t st);
// As launch_trace, with the ray count read on the device from n_dev (<= n, the capacity).
cudaError_t launch_trace_dev(struct ::rt_scene_s* s, const rt_ray* rays, int64_t n, const int* n_dev,
                             rt_hit* hits, uint8_t* occl, const rt_trace_params* tp, TraceScratch& scr,
                             cudaStream_t st);
cudaError_t launch_gen_rays(int kind, const float* origin, long long param, float tmin, float tmax,
                            rt_ray* rays, long long count, cudaStream_t st);
// Band width w and in-band step c of the launch order of an n-ray Fibonacci
// set (host only; fib_slot uses them).
void fib_launch_order(long long n, long long* w, long long* c);

// Launch orders (slot -> direction), shared by the generators and
// rt_launch_index.

// Spiral point held by slot s of an n-point Fibonacci launch in band order:
// slot b w + t of a full band b holds point b w + (t c mod w), which walks the
// band's points in order of azimuth; the slots past the last full band hold
// their own point.
__host__ __device__ inline long long fib_slot(long long s, long long n, long long w, long long c) {
  const long long b = s / w;
  if ((b + 1) * w > n) return s;
  return b * w + (s - b * w) * c % w;
}

// A point of the icosahedron with every edge cut into f segments: corner a
// (kind 0); point i (1 .. f-1) inside edge a (kind 1); point (i, j) inside
// face a, row i (1 .. f-2) of f-1-i points, column j (1 .. f-1-i) (kind 2).
struct IcoPt {
  int kind, a;
  long long i, j;
};

// First point of face row i among the face's points listed row by row.
__host__ __device__ inline long long ico_row_start(long long i, long long f) {
  return (i - 1) * (f - 1) - (i - 1) * i / 2;
}

// Index of p in the order of RT_RAYS_ICOSPHERE: the 12 corners, the points
// inside each edge, the points inside each face row by row.
__host__ __device__ inline long long ico_index(const IcoPt& p, long long f) {
  if (p.kind == 0) return p.a;
  if (p.kind == 1) return 12 + p.a * (f - 1) + p.i - 1;
  return 12 + 30 * (f - 1) + p.a * ((f - 1) * (f - 2) / 2) + ico_row_start(p.i, f) + p.j - 1;
}

// Point held by slot s (0 <= s < 10 f^2 + 2) of an icosphere launch in tile
// order.  Corners and edge points keep their order.  A face's rows are cut
// into bands of 8 (band r: rows 8r+1 .. 8r+8); a band lists the columns all
// 8 of its rows hold as tiles of 8 rows x 4 columns (row by row inside a
// tile), the rest of its rows row by row; even bands run tiles then rest,
// odd bands rest then tiles from the last to the first, so the walk turns
// at the ends of the bands; the rows after the last full band follow row by
// row.  32 consecutive slots of a face lie in one or two neighbouring tiles.
__host__ __device__ inline IcoPt ico_slot_point(long long s, long long f) {
  if (s < 12) return IcoPt{0, (int)s, 0, 0};
  const long long ne = 30 * (f - 1);
  if (s < 12 + ne) {
    const long long r = s - 12;
    const long long e = r / (f - 1);
    return IcoPt{1, (int)e, r - e * (f - 1) + 1, 0};
  }
  const long long per_face = (f - 1) * (f - 2) / 2;
  const long long r0 = s - 12 - ne;
  const long long fc = r0 / per_face;
  const long long q = r0 - fc * per_face;
  const long long nb = (f - 2) / 8;
  // points before band b: sum over b' < b of 8f - 44 - 64 b'
  auto before = [f](long long b) { return (8 * f - 12) * b - 32 * b * b; };
  long long i, j;
  if (q >= before(nb)) {
    const long long q2 = ico_row_start(8 * nb + 1, f) + q - before(nb);
    i = 8 * nb + 1;
    while (ico_row_start(i + 1, f) <= q2) ++i;
    j = q2 - ico_row_start(i, f) + 1;
  } else {
    // the root of before(b) = q (radicand exact in integers, root in
    // float32: off by less than one band), then exact by stepping
    const long long b0 = 8 * f - 12, rad = b0 * b0 - 128 * q;
    long long r = (long long)(((float)b0 - sqrtf((float)(rad > 0 ? rad : 0))) * (1.f / 64.f));
    if (r < 0) r = 0;
    if (r > nb - 1) r = nb - 1;
    while (r > 0 && before(r) > q) --r;
    while (r + 1 < nb && before(r + 1) <= q) ++r;
    const long long u = q - before(r);
    const long long l7 = f - 9 - 8 * r;  // points in the band's last row
    const long long nblk = l7 / 4, tiles = 32 * nblk, rest = 8 * (l7 - 4 * nblk) + 28;
    const bool odd = (r & 1) != 0;
    const bool in_tiles = odd ? u >= rest : u < tiles;
    long long v = odd ? (in_tiles ? u - rest : u) : (in_tiles ? u : u - tiles);
    if (in_tiles) {
      long long blk = v / 32;
      if (odd) blk = nblk - 1 - blk;
      const long long w = v - (v / 32) * 32;
      i = 8 * r + 1 + w / 4;
      j = 4 * blk + (w & 3) + 1;
    } else {
      // row k of the rest holds (l7 - 4 nblk) + 7 - k points
      const long long e = l7 - 4 * nblk;
      long long k = 0;
      while (k < 7 && v >= e + 7 - k) {
        v -= e + 7 - k;
        ++k;
      }
      i = 8 * r + 1 + k;
      j = 4 * nblk + 1 + v;
    }
  }
  return IcoPt{2, (int)fc, i, j};
}
// Device buffers of a batch for the one-launch pipeline (launch_batch_persistent).
struct BatchLaunch {
  int max_order;
  long long n0, n_seg;
  rt_ray* rays[RT_BATCH_MAX_ORDER + 1];
  rt_hit* hits[RT_BATCH_MAX_ORDER + 1];
  int* skip[RT_BATCH_MAX_ORDER + 1];
  int* src[RT_BATCH_MAX_ORDER + 1];
  int* counts;      // [RT_BATCH_MAX_ORDER + 1]
  int* chunk;       // [n0 / 32 + 1]
  int* cta_total;   // [cta_cap]
  int cta_cap;
  const rt_ray* seg;
  uint8_t* occl;
  unsigned* bar;    // [4]
  int* status;
  int* take;        // [RT_BATCH_MAX_ORDER + 2]
  long long timeout_ns;
  TraceScratch* scr;
  // reception (Eq. 4) afterwards: every bounced ray takes its parent's delta
  int receive;
  float* delta[RT_BATCH_MAX_ORDER + 1];         // per ray: its transmitter's delta (order 0 given)
};
// Every order of a batch and its visibility segments in one cooperative
// launch (trace.cu); the order-0 rays must already be in rays[0].
cudaError_t launch_batch_persistent(struct ::rt_scene_s* s, const BatchLaunch& b, cudaStream_t st);
// The most CTAs the one-launch pipeline may use on this device.
int persistent_batch_ctas();

// Launches of n_tx transmitters in one kernel (device arrays: tx 3 floats
// each, off n_tx + 1 ray offsets, param the icosphere level or, for
// Fibonacci launches, fib_launch_order's w << 32 | c).
cudaError_t launch_gen_batch(int kind, const float* tx_dev, const long long* off_dev, const long long* param_dev,
                             int n_tx, long long total, float tmin, float tmax, rt_ray* rays, cudaStream_t st);
cudaError_t launch_reflect(const struct ::rt_scene_s* s, const rt_ray* rays, const rt_hit* hits,
                           long long n, const int* n_dev, rt_ray* out_rays, int* out_skip,
                           int* out_src, int* out_count, int* block_counts, long long cap,
                           cudaStream_t st);

}  // namespace rt

// Host-side scene object.
struct rt_scene_s {
  int device = 0;
  int64_t n_tri = 0;
  int64_t cap_tri = 0;          // capacity of the per-triangle buffers
  float4* tri_in = nullptr;
  int32_t* idx[2] = {nullptr, nullptr};  // idx[0]: input id of each leaf-order triangle
  float4* rec[2] = {nullptr, nullptr};   // primitive records (2 float4 each), ping-pong
  rt::Node2* node2 = nullptr;
  rt::WNode* wide = nullptr;
  rt::QNode* qwide = nullptr;   // 64-byte nodes (builds with quantize = 1)
  rt::WNode8* wide8 = nullptr;  // 8-wide nodes (builds with width = 8)
  int64_t wide8_cap = 0;
  int64_t qwide_cap = 0;
  bool q_built = false;         // the current tree has its 64-byte nodes
  int2* link2 = nullptr;        // (parent, epoch) per binary node
  int* epoch = nullptr;         // build counter on the device
  float4* tri_leaf = nullptr;
  rt::Task* qa = nullptr;       // subtree task queue
  int* qa_ready = nullptr;      // epoch stamp of each filled queue slot
  rt::TopTask* top_task = nullptr;  // [cap_t] big nodes
  int* top_done = nullptr;          // [cap_t] finished chunks of each
  unsigned* top_bins = nullptr;     // [cap_t][3 * kMaxBins * 13] merged bins
  unsigned* top_ccnt = nullptr;     // [cap_c][3 * kMaxBins] per-chunk bin counts
  unsigned* top_scnt = nullptr;     // [cap_c][3 * kMaxBins] per 32-chunk group counts
  int2* top_item = nullptr;         // [cap_c] chunk items (task slot, chunk index)
  int4* top_plan = nullptr;         // [cap_t][2] what each big node reserved for its big children
  int* top_ready = nullptr;         // [cap_c] epoch stamp of each published item
  rt::BuildGeom geom{};             // geometry the buffers were sized for
  rt::BuildCtl* ctl = nullptr;
  rt::TraceScratch scratch;     // default trace scratch
  rt::TraceScratch host_scr[2]; // scratch of the host-buffer pipeline
  int* reflect_blocks = nullptr; // per-block counts of rt_reflect
  int64_t reflect_blocks_cap = 0;
  rt_ray* stage_rays[2] = {nullptr, nullptr};
  rt_hit* stage_hits[2] = {nullptr, nullptr};
  int64_t stage_cap = 0;
  cudaStream_t host_streams[2] = {nullptr, nullptr};
  cudaEvent_t host_ev = nullptr;  // the host pipeline's wait on the caller's stream
  cudaEvent_t ev_build0 = nullptr, ev_build1 = nullptr;
  cudaEvent_t split_ev[2] = {nullptr, nullptr};  // caller's events around the split kernel
  bool built = false;
  rt_build_params params{};
  // range-limited builds: the selected triangles' ids, per-block counts, the
  // count read back by the host
  int* sel = nullptr;
  int* sel_cnt = nullptr;
  int* sel_host = nullptr;  // pinned
  int64_t n_built = 0;      // triangles in the current tree
};
