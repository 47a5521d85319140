// BVH construction on the device (Sec. II.B-C of arXiv 2208.10008).
//
// Pipeline, all asynchronous on one stream.  Every kernel after the first is
// launched with programmatic dependent launch and waits for its predecessor
// (griddepcontrol.wait) before it reads anything that kernel wrote, so the
// launches overlap their set-up with the previous kernel's tail.
//   memset        control block
//   k_prep        Eq. 3 box of every triangle -> build record; scene and
//                 centroid bounds
//   k_bin_root    30-bit Morton key of every box centre (kept in the record
//                 for the small subtrees); the root task; the root's bins
//   k_split       one persistent launch for the whole recursion of Fig. 2.
//                 Its first CTAs take the chunk items of big nodes (more than
//                 `big` triangles, cut into chunks of 256..1024 records, CTA
//                 per chunk): Eq. 2 at every bin plane from the node's merged
//                 bins, stable partition of the chunk into the other record
//                 buffer, and on the way the children's bins and per-chunk
//                 counts; the CTA finishing a node's last chunk writes the node
//                 and publishes its children's items.  Every CTA takes the
//                 subtrees (nodes of at most `big` triangles) from a second
//                 device queue, CTA per subtree, and builds each in shared
//                 memory: nodes of more than 32 triangles split by the whole
//                 CTA (the smaller child goes back to the queue), nodes of at
//                 most 32 finished by single warps in registers over the
//                 Morton order of their records.  No CTA waits for another
//                 except for work to appear (bounded waits).
//   k_post        4-wide traversal nodes (greedy by surface area), stored at the
//                 id of their binary root; triangles in leaf order
//
// Bins.  A bin holds 13 words: the record count, the union of the records'
// boxes and the bounds of their box centres, the floats as order-preserving
// unsigned codes (min slots store the complement) so that every merge is an
// atomicAdd or atomicMax and all-zero is the empty bin.  A node's bins give the
// exact boxes and centroid bounds of both children of any plane, so a child is
// binned while its parent is partitioned.
//
// Node identity: the binary node that splits its range at position s gets id
// s - 1.  Split positions of distinct internal nodes differ, so ids need no
// allocator and the tree is the same whatever order the work ran in.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int kBlock = 256;  // threads of every build CTA
constexpr int kWarps = kBlock / 32;
constexpr int kBinVals = 13;  // count, box lo xyz, box hi xyz, centre lo xyz, centre hi xyz
constexpr int kBinWords = 3 * kMaxBins * kBinVals;
constexpr int kCntStride = 3 * kMaxBins;
constexpr int kMaxRpt = 4;     // records per thread of a big node's chunk
constexpr int kBigMin = 1024;  // big nodes have more triangles than this
constexpr int kStageW = 256;   // records the global-memory warp split (oversized tasks) stages
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void set_status(BuildCtl* ctl, int code, int where) {
  if (atomicCAS(&ctl->status, 0, code) == 0) ctl->status_where = where;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Acquire load / release store / release add at GPU scope: the flag and
// counter protocol of the work queues without full memory fences.
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// AABB centre, evaluated identically wherever a bin is needed.
__device__ __forceinline__ float centre(float lo, float hi) { return __fmul_rn(__fadd_rn(lo, hi), 0.5f); }

// Bin index of centroid coordinate c for slab [cmin, cmin + K/scale).
__device__ __forceinline__ int bin_of(float c, float cmin, float scale, int K) {
  int b = (int)__fmul_rn(__fsub_rn(c, cmin), scale);
  return min(max(b, 0), K - 1);
}

__device__ __forceinline__ float bin_scale(float cmin, float cmax, int K) {
  float ext = cmax - cmin;
  return ext > 0.f ? (float)K * (1.f - 1e-6f) / ext : 0.f;
}

__device__ __forceinline__ float area(float3 lo, float3 hi) {
  float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
  return 2.f * (dx * dy + dy * dz + dz * dx);
}

__device__ __forceinline__ float sel3(float x, float y, float z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

struct CostP {
  float alpha, t_i, t_trav, sx, sy, sz;
  int dist_norm;
};

// Eq. 2 (Eq. 1 at alpha = 1): children L (nl triangles), R (nr) of node C.
// The two divisions by the node's area and squared diagonal are fast
// approximate reciprocals times products: the build's cost needs no correctly
// rounded quotient, only the same value for the same inputs.
__device__ __forceinline__ float eq2_cost(float3 llo, float3 lhi, int nl, float3 rlo, float3 rhi, int nr, float3 clo,
                                          float3 chi, const CostP& p) {
  const float sc = area(clo, chi);
  const float sah = sc > 0.f ? (area(llo, lhi) * (float)nl + area(rlo, rhi) * (float)nr) * __fdividef(1.f, sc) * p.t_i
                             : (float)(nl + nr) * p.t_i;
  const float ax = 0.5f * (llo.x + lhi.x) - p.sx, ay = 0.5f * (llo.y + lhi.y) - p.sy, az = 0.5f * (llo.z + lhi.z) - p.sz;
  const float bx = 0.5f * (rlo.x + rhi.x) - p.sx, by = 0.5f * (rlo.y + rhi.y) - p.sy, bz = 0.5f * (rlo.z + rhi.z) - p.sz;
  const float da2 = ax * ax + ay * ay + az * az, db2 = bx * bx + by * by + bz * bz;
  float d2 = 0.5f * (da2 + db2);
  if (p.dist_norm) {
    const float dx = chi.x - clo.x, dy = chi.y - clo.y, dz = chi.z - clo.z;
    const float diag2 = dx * dx + dy * dy + dz * dz;
    if (p.dist_norm == 2)  // each child's distance weighted by its triangles
      d2 = (diag2 > 0.f ? ((float)nl * da2 + (float)nr * db2) * __fdividef(1.f, diag2) : 0.f) * p.t_i;
    else
      d2 = (diag2 > 0.f ? d2 * __fdividef(1.f, diag2) : 0.f) * (float)(nl + nr) * p.t_i;
  }
  return p.alpha * sah + (1.f - p.alpha) * d2 + p.t_trav;
}

// Order-preserving unsigned code of a float: a < b <=> ucode(a) < ucode(b).
__device__ __forceinline__ unsigned ucode(float x) { return (unsigned)ford(x) ^ 0x80000000u; }
__device__ __forceinline__ float uval(unsigned u) { return iford((int)(u ^ 0x80000000u)); }

// ------------------------------------------------------------------ bins
// Union of a run of bins (or of records): count, box, centre bounds.
struct BinU {
  int n;
  float l0, l1, l2, h0, h1, h2;  // box
  float a0, a1, a2, b0, b1, b2;  // centre bounds
};

__device__ __forceinline__ BinU binu_empty() {
  return {0, FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX,
          FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};
}
__device__ __forceinline__ BinU binu_join(const BinU& x, const BinU& y) {
  return {x.n + y.n,
          fminf(x.l0, y.l0), fminf(x.l1, y.l1), fminf(x.l2, y.l2),
          fmaxf(x.h0, y.h0), fmaxf(x.h1, y.h1), fmaxf(x.h2, y.h2),
          fminf(x.a0, y.a0), fminf(x.a1, y.a1), fminf(x.a2, y.a2),
          fmaxf(x.b0, y.b0), fmaxf(x.b1, y.b1), fmaxf(x.b2, y.b2)};
}
__device__ __forceinline__ BinU binu_record(float4 lo, float4 hi) {
  const float cx = centre(lo.x, hi.x), cy = centre(lo.y, hi.y), cz = centre(lo.z, hi.z);
  return {1, lo.x, lo.y, lo.z, hi.x, hi.y, hi.z, cx, cy, cz, cx, cy, cz};
}
#define RT_BINU_SHFL(F, x, arg)                                                                               \
  BinU {                                                                                                      \
    F(kFull, (x).n, arg), F(kFull, (x).l0, arg), F(kFull, (x).l1, arg), F(kFull, (x).l2, arg),                \
        F(kFull, (x).h0, arg), F(kFull, (x).h1, arg), F(kFull, (x).h2, arg), F(kFull, (x).a0, arg),           \
        F(kFull, (x).a1, arg), F(kFull, (x).a2, arg), F(kFull, (x).b0, arg), F(kFull, (x).b1, arg),           \
        F(kFull, (x).b2, arg)                                                                                 \
  }
__device__ __forceinline__ BinU binu_xor(const BinU& x, int o) { return RT_BINU_SHFL(__shfl_xor_sync, x, o); }
#undef RT_BINU_SHFL

// Decode a 13-word bin entry.
__device__ __forceinline__ BinU binu_load(const unsigned* e) {
  const unsigned c = e[0];
  if (c == 0) return binu_empty();
  return {(int)c,          uval(~e[1]), uval(~e[2]), uval(~e[3]), uval(e[4]),  uval(e[5]), uval(e[6]),
          uval(~e[7]),     uval(~e[8]), uval(~e[9]), uval(e[10]), uval(e[11]), uval(e[12])};
}

// A record's 12 bin codes: box lo / hi and centre (twice: min and max slot).
struct RecCodes {
  unsigned v[12];
};
__device__ __forceinline__ RecCodes rec_codes(float4 lo, float4 hi, float cx, float cy, float cz) {
  RecCodes r;
  r.v[0] = ~ucode(lo.x);
  r.v[1] = ~ucode(lo.y);
  r.v[2] = ~ucode(lo.z);
  r.v[3] = ucode(hi.x);
  r.v[4] = ucode(hi.y);
  r.v[5] = ucode(hi.z);
  r.v[6] = ~ucode(cx);
  r.v[7] = ~ucode(cy);
  r.v[8] = ~ucode(cz);
  r.v[9] = ucode(cx);
  r.v[10] = ucode(cy);
  r.v[11] = ucode(cz);
  return r;
}

// Add the record of every lane with cell >= 0 to its bin on each axis: entry
// e[a] (count at bins + e[a] * kBinVals, then the 12 code maxima) and, if
// cnt is not null, cnt[e[a]].  The cell names the entries (equal cells,
// equal entries).  Lanes whose cells are equal and adjacent form a run: a
// segmented warp scan gives the run's last lane the run's count and code
// maxima, and that lane alone issues the shared-memory atomics, for all
// three axes.  Records in Morton or input order come in runs of one cell,
// so a warp costs one scan of 12 words instead of reductions per distinct
// bin and axis.  All 32 lanes of the warp must call.
__device__ __forceinline__ void bin_add_runs(int cell, const int* e, unsigned* bins, unsigned* cnt,
                                             const RecCodes& c) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  const int prev = __shfl_up_sync(kFull, cell, 1), next = __shfl_down_sync(kFull, cell, 1);
  const bool head = lane == 0 || prev != cell, tail = lane == 31 || next != cell;
  const unsigned heads = __ballot_sync(kFull, head);
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // first lane of the run
  unsigned v[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) v[q] = c.v[q];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const unsigned u = __shfl_up_sync(kFull, v[q], o);
      if (lane - o >= start) v[q] = max(v[q], u);
    }
  }
  if (tail && cell >= 0) {
    const unsigned m = (unsigned)(lane - start + 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      unsigned* b = bins + e[a] * kBinVals;
      atomicAdd(b, m);
#pragma unroll
      for (int q = 0; q < 12; ++q) atomicMax(b + 1 + q, v[q]);
      if (cnt) atomicAdd(cnt + e[a], m);
    }
  }
}

// Add one record to bin entry `e` with plain shared-memory atomics (callers
// spread the lanes over distant records, so lanes rarely share an entry).
__device__ __forceinline__ void bin_add_plain(unsigned* e, const RecCodes& c) {
  atomicAdd(e, 1u);
#pragma unroll
  for (int q = 0; q < 12; ++q) atomicMax(e + 1 + q, c.v[q]);
}

// ------------------------------------------------------------------ Eq. 2 evaluation
struct Split {
  float cost;
  int cand;  // axis * (K - 1) + plane - 1 (INT_MAX: none)
  BinU L, R;
};

__device__ __forceinline__ void split_none(Split& s) {
  s.cost = INFINITY;
  s.cand = INT_MAX;
  s.L = binu_empty();
  s.R = binu_empty();
}

// Count and box of a run of bins: the part of a bin the cost needs.
struct BinB {
  int n;
  float l0, l1, l2, h0, h1, h2;
};
__device__ __forceinline__ BinB binb_empty() { return {0, FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX}; }
__device__ __forceinline__ BinB binb_join(const BinB& x, const BinB& y) {
  return {x.n + y.n,          fminf(x.l0, y.l0), fminf(x.l1, y.l1), fminf(x.l2, y.l2),
          fmaxf(x.h0, y.h0),  fmaxf(x.h1, y.h1), fmaxf(x.h2, y.h2)};
}
__device__ __forceinline__ BinB binb_load(const unsigned* e) {
  const unsigned c = e[0];
  if (c == 0) return binb_empty();
  return {(int)c, uval(~e[1]), uval(~e[2]), uval(~e[3]), uval(e[4]), uval(e[5]), uval(e[6])};
}
#define RT_BINB_SHFL(F, x, arg)                                                                            \
  BinB {                                                                                                   \
    F(kFull, (x).n, arg), F(kFull, (x).l0, arg), F(kFull, (x).l1, arg), F(kFull, (x).l2, arg),             \
        F(kFull, (x).h0, arg), F(kFull, (x).h1, arg), F(kFull, (x).h2, arg)                                 \
  }

// Eq. 2 at the K - 1 planes of na axes (a0 .. a0 + na - 1, na * K <= 32) by
// one warp.  Lanes are cut into segments of K, lane sl of segment g holding
// bin sl of axis a0 + g (`bins0` points at the bins of axis a0, the others
// follow); segmented warp scans (log2 K steps) of the bins' counts and boxes
// give every lane the union of the bins left of plane sl and right of it,
// and lane sl evaluates Eq. 2 there.  `best` (identical in every lane) is
// replaced if a plane has a lower cost, ties going to the lower candidate
// (lowest axis, then lowest plane); the winning children's centre bounds
// are then gathered by warp reductions over the bins' codes.  The union of
// a segment is the node box.
// kVals: words per bin (13, or 7 for bins of count and box only); kCentres:
// gather the children's centre bounds (13-word bins only; otherwise the
// caller derives the children's unions itself and only best.L.n is exact).
template <int kVals, bool kCentres>
__device__ __forceinline__ void eval_seg(const unsigned* bins0, int K, int n, int a0, int na, const CostP& cp,
                                         Split& best) {
  const int lane = threadIdx.x & 31;
  const int g = lane / K, sl = lane - g * K;
  const bool in = g < na;
  const int a = a0 + (in ? g : 0);
  const unsigned* e = bins0 + ((in ? g : 0) * K + sl) * kVals;
  __syncwarp();
  const BinB x = in ? binb_load(e) : binb_empty();
  BinB pre = x, suf = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= K) break;
    const BinB u = RT_BINB_SHFL(__shfl_up_sync, pre, o), d = RT_BINB_SHFL(__shfl_down_sync, suf, o);
    if (sl >= o) pre = binb_join(pre, u);
    if (sl + o < K) suf = binb_join(suf, d);
  }
  const BinB L = RT_BINB_SHFL(__shfl_up_sync, pre, 1);  // lane sl: bins 0 .. sl-1 of its axis
  const BinB C = RT_BINB_SHFL(__shfl_sync, pre, min(g * K + K - 1, 31));
  // Eq. 2 in every lane (a plane without records on both sides costs
  // infinity), then the lowest cost by two warp reductions: costs are >= +0
  // (alpha in [0, 1], t_i > 0, t_trav >= 0), so their bit patterns order as
  // their values, and the lowest candidate among equal costs wins
  const float c = eq2_cost(make_float3(L.l0, L.l1, L.l2), make_float3(L.h0, L.h1, L.h2), L.n,
                           make_float3(suf.l0, suf.l1, suf.l2), make_float3(suf.h0, suf.h1, suf.h2), n - L.n,
                           make_float3(C.l0, C.l1, C.l2), make_float3(C.h0, C.h1, C.h2), cp);
  const bool ok = in && sl >= 1 && L.n > 0 && L.n < n && c < INFINITY;
  const unsigned key = ok ? __float_as_uint(c + 0.f) : __float_as_uint(INFINITY);
  const unsigned kmin = __reduce_min_sync(kFull, key);
  const int cand = (int)__reduce_min_sync(kFull, ok && key == kmin ? (unsigned)(a * (K - 1) + sl - 1) : 0xffffffffu);
  const float cost = __uint_as_float(kmin);
  if (cand >= 0 && (cost < best.cost || (cost == best.cost && cand < best.cand))) {
    const int ax = cand / (K - 1), gw = ax - a0, pl = cand - ax * (K - 1) + 1;  // plane pl of axis ax
    const int w = gw * K + pl;
    const BinB Lb = RT_BINB_SHFL(__shfl_sync, L, w), Rb = RT_BINB_SHFL(__shfl_sync, suf, w);
    const bool mine = in && g == gw;
    unsigned lc[6] = {0u, 0u, 0u, 0u, 0u, 0u}, rc[6] = {0u, 0u, 0u, 0u, 0u, 0u};
    if (kCentres) {
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const unsigned v = mine ? e[7 + q] : 0u;
        lc[q] = __reduce_max_sync(kFull, sl < pl ? v : 0u);
        rc[q] = __reduce_max_sync(kFull, sl >= pl ? v : 0u);
      }
    }
    best.cost = cost;
    best.cand = cand;
    best.L = {Lb.n, Lb.l0, Lb.l1, Lb.l2, Lb.h0, Lb.h1, Lb.h2,
              uval(~lc[0]), uval(~lc[1]), uval(~lc[2]), uval(lc[3]), uval(lc[4]), uval(lc[5])};
    best.R = {Rb.n, Rb.l0, Rb.l1, Rb.l2, Rb.h0, Rb.h1, Rb.h2,
              uval(~rc[0]), uval(~rc[1]), uval(~rc[2]), uval(rc[3]), uval(rc[4]), uval(rc[5])};
  }
}
#undef RT_BINB_SHFL

__device__ __forceinline__ void eval_axis(const unsigned* bins, int K, int n, int a, const CostP& cp, Split& best) {
  eval_seg<kBinVals, true>(bins + a * K * kBinVals, K, n, a, 1, cp, best);
}
__device__ __forceinline__ void eval_axes(const unsigned* bins, int K, int n, int a0, int na, const CostP& cp,
                                          Split& best) {
  eval_seg<kBinVals, true>(bins + a0 * K * kBinVals, K, n, a0, na, cp, best);
}

// ------------------------------------------------------------------ arguments
struct BuildArgs {
  const float4* tri;  // input-order triangles
  const int* sel;     // nullable: input ids of the triangles in this build (a range build)
  float4* rec[2];     // [2T] records (lo.xyz, id) (hi.xyz, morton); a node's range lives
                      // in one buffer, its children go to the other
  Node2* node2;
  int2* link2;
  BuildCtl* ctl;
  Task* qa;  // subtree queue
  int* qa_ready;
  TopTask* ttask;  // big nodes
  int* tdone;
  unsigned* tbins;
  unsigned* tccnt;
  unsigned* tscnt;
  int2* titem;  // chunk items of big nodes
  int4* tplan;  // [cap_t][2]: what a big node reserved for each big child (task slots, count slots,
                // chunk items, count slots to clear), written by its chunk 0
  int* tready;
  WNode* wide;
  QNode* qwide;  // nullable: also write the 64-byte nodes
  WNode8* wide8; // nullable: write 8-wide traversal nodes (instead of the 4-wide ones)
  float4* tri_leaf;
  int32_t* order;
  int* epoch_dev;
  int n, K, max_leaf;  // n: records in this build
  int n_all;           // triangles in the scene (input ids are below it)
  int big, chunk, rpt, cap_t, cap_c, qa_cap, top_ctas;
  int spin_limit;                    // polls without progress before a wait gives up
  int phantom_tasks, phantom_items;  // test hooks: pending work that never comes
  CostP cp;
};

__device__ __forceinline__ unsigned* tbins_at(const BuildArgs& A, int slot) {
  return A.tbins + (size_t)slot * kBinWords;
}
__device__ __forceinline__ unsigned* tccnt_at(const BuildArgs& A, int c) { return A.tccnt + (size_t)c * kCntStride; }
__device__ __forceinline__ unsigned* tscnt_at(const BuildArgs& A, int c) { return A.tscnt + (size_t)c * kCntStride; }

__device__ __forceinline__ TopTask load_top_cg(const TopTask* p) {
  const int4* q = reinterpret_cast<const int4*>(p);
  const int4 a = __ldcg(q), b = __ldcg(q + 1), c = __ldcg(q + 2), d = __ldcg(q + 3);
  TopTask t;
  t.begin = a.x;
  t.count = a.y;
  t.parent = a.z;
  t.side = a.w;
  t.clo[0] = __int_as_float(b.x);
  t.clo[1] = __int_as_float(b.y);
  t.clo[2] = __int_as_float(b.z);
  t.depth = b.w;
  t.chi[0] = __int_as_float(c.x);
  t.chi[1] = __int_as_float(c.y);
  t.chi[2] = __int_as_float(c.z);
  t.nchunk = c.w;
  t.chunk_first = d.x;
  t.child_slot = d.y;
  t.chunk_res = d.z;
  t.parity = d.w;
  return t;
}

// Hand a task to the subtree queue (one thread).  The slot's ready word
// takes this build's epoch, so stale slots from older builds never match.
__device__ void push_task(const BuildArgs& A, const Task& t, int epoch) {
  const int s = atomicAdd(&A.ctl->qa_tail, 1);
  if (s >= A.qa_cap) {
    set_status(A.ctl, kStQueueOverflow, 1);
    return;
  }
  atomicAdd(&A.ctl->qa_pending, 1);
  A.qa[s] = t;
  st_release(&A.qa_ready[s], epoch);
}

// Hand up to 3 tasks to the subtree queue at once (one thread): one slot
// reservation, one fence.
__device__ void push_tasks(const BuildArgs& A, const Task* t, int k, int epoch) {
  if (k <= 0) return;
  const int s = atomicAdd(&A.ctl->qa_tail, k);
  if (s + k > A.qa_cap) {
    set_status(A.ctl, kStQueueOverflow, 3);
    return;
  }
  atomicAdd(&A.ctl->qa_pending, k);
  for (int i = 0; i < k; ++i) A.qa[s + i] = t[i];
  for (int i = 0; i < k; ++i) st_release(&A.qa_ready[s + i], epoch);
}

__device__ __forceinline__ Task make_task(int begin, int count, int parent, int side, int depth, const BinU& u,
                                          int parity) {
  Task t;
  t.begin = begin;
  t.count = count;
  t.parent = parent;
  t.side = side;
  t.clo[0] = u.a0;
  t.clo[1] = u.a1;
  t.clo[2] = u.a2;
  t.chi[0] = u.b0;
  t.chi[1] = u.b1;
  t.chi[2] = u.b2;
  t.depth = depth;
  t.pad = parity;
  return t;
}

// Reserve `amt` consecutive items of a counter bounded by `cap`: one atomic
// add; -1 if they do not fit (the items past cap are then never used).
__device__ __forceinline__ int reserve(int* ctr, int amt, int cap) {
  const int old = atomicAdd(ctr, amt);
  return old + amt <= cap ? old : -1;
}

// Write binary node `id` (both children's boxes, refs, counts) and link it
// to its parent.  One thread.
__device__ __forceinline__ void write_node(const BuildArgs& A, int id, int parent, int side, const BinU& L, int refl,
                                           int nl, const BinU& R, int refr, int nr, int epoch) {
  Node2 nd;
  nd.a_lo = make_float4(L.l0, L.l1, L.l2, __int_as_float(refl));
  nd.a_hi = make_float4(L.h0, L.h1, L.h2, __int_as_float(nl));
  nd.b_lo = make_float4(R.l0, R.l1, R.l2, __int_as_float(refr));
  nd.b_hi = make_float4(R.h0, R.h1, R.h2, __int_as_float(nr));
  A.node2[id] = nd;
  if (parent < 0)
    A.ctl->root_ref = id;
  else if (parent < A.n - 1)
    *(side == 0 ? &A.node2[parent].a_lo.w : &A.node2[parent].b_lo.w) = __int_as_float(id);
  else
    set_status(A.ctl, kStBadLink, 3);
  A.link2[id] = make_int2(parent, epoch);
}

// ------------------------------------------------------------------ range selection
// A build with a ray action range keeps the triangles whose box lies within
// the range of the source (Sec. II.B): no point of a path of total length
// <= range is farther from the source, at any reflection order.  The
// selection keeps input order (block counts, one scan, ordered writes), so
// the build is the same every time.  The range is widened by 1e-5 of itself
// so that rounding never drops a reachable triangle.
__device__ __forceinline__ bool tri_in_range(const float4* __restrict__ tri, int i, float3 s, float r2) {
  const float4 a = __ldg(tri + 3 * (size_t)i), b = __ldg(tri + 3 * (size_t)i + 1), c = __ldg(tri + 3 * (size_t)i + 2);
  const float dx = fmaxf(fmaxf(fminf(a.x, fminf(b.x, c.x)) - s.x, s.x - fmaxf(a.x, fmaxf(b.x, c.x))), 0.f);
  const float dy = fmaxf(fmaxf(fminf(a.y, fminf(b.y, c.y)) - s.y, s.y - fmaxf(a.y, fmaxf(b.y, c.y))), 0.f);
  const float dz = fmaxf(fmaxf(fminf(a.z, fminf(b.z, c.z)) - s.z, s.z - fmaxf(a.z, fmaxf(b.z, c.z))), 0.f);
  return dx * dx + dy * dy + dz * dz <= r2;
}

__global__ void __launch_bounds__(kBlock) k_sel_count(const float4* __restrict__ tri, int n, float3 s, float r2,
                                                      int* __restrict__ cnt) {
  const int i = blockIdx.x * kBlock + threadIdx.x;
  const int c = __syncthreads_count(i < n && tri_in_range(tri, i, s, r2));
  if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

// Exclusive scan of cnt[0 .. nb) in place by one CTA; the total goes to cnt[nb].
__global__ void __launch_bounds__(1024) k_sel_scan(int* __restrict__ cnt, int nb) {
  __shared__ int part[1024];
  const int t = threadIdx.x, per = (nb + 1023) / 1024, b0 = min(t * per, nb), b1 = min(b0 + per, nb);
  int sum = 0;
  for (int b = b0; b < b1; ++b) sum += cnt[b];
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - sum;
  for (int b = b0; b < b1; ++b) {
    const int v = cnt[b];
    cnt[b] = run;
    run += v;
  }
  if (t == 1023) cnt[nb] = part[1023];
}

__global__ void __launch_bounds__(kBlock) k_sel_write(const float4* __restrict__ tri, int n, float3 s, float r2,
                                                      const int* __restrict__ off, int* __restrict__ sel) {
  __shared__ int wc[kWarps];
  const int i = blockIdx.x * kBlock + threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool f = i < n && tri_in_range(tri, i, s, r2);
  const unsigned bal = __ballot_sync(kFull, f);
  if (lane == 0) wc[warp] = __popc(bal);
  __syncthreads();
  int base = off[blockIdx.x];
  for (int w = 0; w < warp; ++w) base += wc[w];
  if (f) sel[base + __popc(bal & ((1u << lane) - 1u))] = i;
}

// ------------------------------------------------------------------ prep
__global__ void __launch_bounds__(kBlock) k_prep(BuildArgs A) {
  pdl_wait();
  pdl_launch();
  __shared__ float red[kWarps][12];
  const int n = A.n;
  const int gt = blockIdx.x * kBlock + threadIdx.x, gs = gridDim.x * kBlock;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (gt == 0) {
    const int e = *A.epoch_dev + 1;
    *A.epoch_dev = e;
    A.ctl->epoch = e;
  }
  // the root's bins and 32-chunk group counts start empty
  const int nch = (n + A.chunk - 1) / A.chunk;
  for (int k = gt; k < kBinWords; k += gs) A.tbins[k] = 0u;
  for (int k = gt; k < (nch / 32 + 1) * kCntStride; k += gs) A.tscnt[k] = 0u;
  float v[12];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    v[k] = FLT_MAX;       // box lo
    v[3 + k] = -FLT_MAX;  // box hi
    v[6 + k] = FLT_MAX;   // centre lo
    v[9 + k] = -FLT_MAX;  // centre hi
  }
  for (int i = gt; i < n; i += gs) {
    const int t = A.sel ? __ldg(A.sel + i) : i;
    const float4 a = A.tri[3 * (size_t)t], b = A.tri[3 * (size_t)t + 1], c = A.tri[3 * (size_t)t + 2];
    const float lx = fminf(a.x, fminf(b.x, c.x)), ly = fminf(a.y, fminf(b.y, c.y)), lz = fminf(a.z, fminf(b.z, c.z));
    const float hx = fmaxf(a.x, fmaxf(b.x, c.x)), hy = fmaxf(a.y, fmaxf(b.y, c.y)), hz = fmaxf(a.z, fmaxf(b.z, c.z));
    A.rec[0][2 * (size_t)i] = make_float4(lx, ly, lz, __int_as_float(t));
    A.rec[0][2 * (size_t)i + 1] = make_float4(hx, hy, hz, 0.f);
    const float cx = centre(lx, hx), cy = centre(ly, hy), cz = centre(lz, hz);
    v[0] = fminf(v[0], lx);
    v[1] = fminf(v[1], ly);
    v[2] = fminf(v[2], lz);
    v[3] = fmaxf(v[3], hx);
    v[4] = fmaxf(v[4], hy);
    v[5] = fmaxf(v[5], hz);
    v[6] = fminf(v[6], cx);
    v[7] = fminf(v[7], cy);
    v[8] = fminf(v[8], cz);
    v[9] = fmaxf(v[9], cx);
    v[10] = fmaxf(v[10], cy);
    v[11] = fmaxf(v[11], cz);
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const bool mn = k < 3 || (k >= 6 && k < 9);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float y = __shfl_xor_sync(kFull, v[k], o);
      v[k] = mn ? fminf(v[k], y) : fmaxf(v[k], y);
    }
    if (lane == 0) red[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    const int k = threadIdx.x;
    const bool mn = k < 3 || (k >= 6 && k < 9);
    float x = red[0][k];
    for (int w = 1; w < kWarps; ++w) x = mn ? fminf(x, red[w][k]) : fmaxf(x, red[w][k]);
    if (n > 0) atomicMax(&A.ctl->sb[k], mn ? ~ucode(x) : ucode(x));
  }
}

// Spread the low 10 bits of v to every third bit.
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// ------------------------------------------------------------------ root
// Morton keys of all records; the root task (a top task, a subtree task, a
// leaf or nothing); the root's bins and per-chunk counts when it is a top task.
__global__ void __launch_bounds__(kBlock) k_bin_root(BuildArgs A) {
  pdl_wait();
  pdl_launch();
  __shared__ unsigned sbins[kBinWords];
  __shared__ unsigned scnt[kCntStride];
  const int n = A.n, K = A.K, K3 = 3 * K, CH = A.chunk;
  const int nch = (n + CH - 1) / CH;
  const bool top = n > A.big;
  const int gt = blockIdx.x * kBlock + threadIdx.x, gs = gridDim.x * kBlock;
  float cl[3], chh[3], msc[3], scl[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cl[a] = uval(~__ldcg(&A.ctl->sb[6 + a]));
    chh[a] = uval(__ldcg(&A.ctl->sb[9 + a]));
    const float ext = chh[a] - cl[a];
    msc[a] = ext > 0.f ? 1023.99f / ext : 0.f;
    scl[a] = bin_scale(cl[a], chh[a], K);
  }
  if (gt == 0) {
    const int epoch = __ldcg(&A.ctl->epoch);
    BinU cu = binu_empty();
    cu.a0 = cl[0];
    cu.a1 = cl[1];
    cu.a2 = cl[2];
    cu.b0 = chh[0];
    cu.b1 = chh[1];
    cu.b2 = chh[2];
    if (n == 0) {
      A.ctl->root_ref = INT_MIN;
    } else if (n <= A.max_leaf) {
      A.ctl->root_ref = leaf_ref(0, n);
      A.ctl->n_leaves = 1;
      A.ctl->depth2 = 1;
      A.ctl->max_leaf_size = n;
    } else if (!top) {
      push_task(A, make_task(0, n, -1, 0, 1, cu, 0), epoch);
    } else {
      TopTask R;
      R.begin = 0;
      R.count = n;
      R.parent = -1;
      R.side = 0;
      for (int a = 0; a < 3; ++a) {
        R.clo[a] = cl[a];
        R.chi[a] = chh[a];
      }
      R.depth = 1;
      R.nchunk = nch;
      R.chunk_first = 0;   // count slots 0 .. nch-1: the root's chunks (written below)
      R.child_slot = 1;    // task slots 1, 2
      R.chunk_res = nch;   // count slots nch .. 2 nch + 1
      R.parity = 0;
      A.ttask[0] = R;
      A.ctl->t_slot_next = 3;
      A.ctl->t_cnt_next = 2 * nch + 2;
      A.ctl->ti_tail = nch;
      A.ctl->ti_pending = nch;
    }
    if (A.phantom_tasks) atomicAdd(&A.ctl->qa_pending, A.phantom_tasks);
    if (A.phantom_items) atomicAdd(&A.ctl->ti_pending, A.phantom_items);
  }
  if (top) {
    // the root's children start empty; the root's chunks become items
    const int epoch = __ldcg(&A.ctl->epoch);
    for (int k = gt; k < 2 * kBinWords; k += gs) tbins_at(A, 1)[k] = 0u;
    for (int k = gt; k < (nch + 2) * kCntStride; k += gs) {
      tccnt_at(A, nch)[k] = 0u;
      tscnt_at(A, nch)[k] = 0u;
    }
    if (gt < 3) A.tdone[gt] = 0;
    for (int c = gt; c < nch; c += gs) {
      A.titem[c] = make_int2(0, c);
      A.tready[c] = epoch;
    }
  }
  float4* rec = A.rec[0];
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    if (top) {
      for (int w = threadIdx.x; w < K3 * kBinVals; w += kBlock) sbins[w] = 0u;
      for (int w = threadIdx.x; w < K3; w += kBlock) scnt[w] = 0u;
      __syncthreads();
    }
    for (int r = 0; r < A.rpt; ++r) {
      const int k = c * CH + r * kBlock + threadIdx.x;
      const bool valid = k < n;
      float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
      float cx = 0.f, cy = 0.f, cz = 0.f;
      if (valid) {
        lo = __ldcg(rec + 2 * (size_t)k);
        hi = __ldcg(rec + 2 * (size_t)k + 1);
        cx = centre(lo.x, hi.x);
        cy = centre(lo.y, hi.y);
        cz = centre(lo.z, hi.z);
        uint32_t q[3];
        const float cc[3] = {cx, cy, cz};
#pragma unroll
        for (int a = 0; a < 3; ++a) q[a] = (uint32_t)min(max((int)((cc[a] - cl[a]) * msc[a]), 0), 1023);
        const uint32_t key = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
        hi.w = __uint_as_float(key);
        rec[2 * (size_t)k + 1] = hi;
      }
      if (top) {
        const float cc[3] = {cx, cy, cz};
        const RecCodes rc = rec_codes(lo, hi, cx, cy, cz);
        int e[3], cell = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int b = bin_of(cc[a], cl[a], scl[a], K);
          e[a] = a * K + b;
          cell = cell * kMaxBins + b;
        }
        bin_add_runs(valid ? cell : -1, e, sbins, scnt, rc);
      }
    }
    if (top) {
      __syncthreads();
      unsigned* gc = tccnt_at(A, c);
      unsigned* gg = tscnt_at(A, c >> 5);
      for (int w = threadIdx.x; w < K3; w += kBlock) {
        const unsigned v = scnt[w];
        gc[w] = v;
        if (v) atomicAdd(gg + w, v);
      }
      unsigned* gb = tbins_at(A, 0);
      for (int w = threadIdx.x; w < K3 * kBinVals; w += kBlock) {
        const unsigned v = sbins[w];
        if (v) {
          if (w % kBinVals == 0)
            atomicAdd(gb + w, v);
          else
            atomicMax(gb + w, v);
        }
      }
      __syncthreads();
    }
  }
}

// Tree facts gathered by a warp, added to the control block when it exits.
struct WarpStats {
  int n_int, n_leaf, big, deep;
};

// Account a written binary node (one thread per node).
__device__ __forceinline__ void note_node(WarpStats& ws, int nl, int nr, bool leafl, bool leafr, int depth) {
  ++ws.n_int;
  ws.n_leaf += (int)leafl + (int)leafr;
  if (leafl) ws.big = max(ws.big, nl);
  if (leafr) ws.big = max(ws.big, nr);
  ws.deep = max(ws.deep, (leafl || leafr) ? depth + 1 : depth);
}

// ------------------------------------------------------------------ big nodes
struct TopSmem {
  unsigned pbins[kBinWords];
  unsigned cbins[2][kBinWords];
  unsigned ccnt[2][2][kCntStride];
  Split ax[3];
  int wl[kWarps];
  int red[kWarps];
  int2 item;
  int last;
  int created[2], ibase[2];
  int4 plan[2];
  Task ptask[2];  // subtree-sized children the emit hands to the subtree queue
  int np;
};

__device__ __forceinline__ int block_sum(int v, int* red) {
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int t = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) t += red[w];
  __syncthreads();
  return t;
}

// One thread takes the next chunk item and waits for it to be published
// (no warp-synchronous operation in this loop; the other threads wait at a
// barrier).  Returns (-1, 0) when no big node is left (or the build failed).
// The wait is bounded: spin_limit polls without new items set a timeout
// status.
__device__ int2 claim_item(const BuildArgs& A, int epoch) {
  const int s = atomicAdd(&A.ctl->ti_head, 1);
  int seen = -1;
  for (int it = 0;; ++it) {
    if (s < A.cap_c && ld_acquire(&A.tready[s]) == epoch) {
      return __ldcg(A.titem + s);
    }
    if ((it & 3) == 0) {
      if (ld_volatile(&A.ctl->ti_pending) == 0 || ld_volatile(&A.ctl->status) != 0) break;
      const int tail = ld_volatile(&A.ctl->ti_tail);
      if (tail != seen) {  // new items appeared: restart the no-progress budget
        seen = tail;
        it = 0;
      }
    }
    if (it > A.spin_limit) {
      set_status(A.ctl, kStQueueTimeout, 2);
      break;
    }
    __nanosleep(128);
  }
  return make_int2(-1, 0);
}

__device__ void top_emit(const BuildArgs& A, TopSmem& S, const TopTask& T, int slot, int epoch, int nl, int nr,
                         const BinU& cu0, const BinU& cu1, bool top0, bool top1, int nch0, int nch1, int cfirst0,
                         int cfirst1, WarpStats& ts);

// Chunk 0 of a big node, as soon as its split is known: reserve what the
// node's big children will need (two task slots and the count slots for
// their own children, their chunk items) and clear what their chunks will
// fill, so that the CTA finishing the node's last chunk only writes and
// publishes.  The clearing is ordered before that CTA's emit by chunk 0's
// release of its done count.
__device__ void top_plan(const BuildArgs& A, TopSmem& S, int slot, bool top0, bool top1, int nch0, int nch1) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    int cs[2] = {-1, -1}, cr[2] = {-1, -1}, ib[2] = {-1, -1};
    // every reservation is issued before any result is used: one round trip
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (!(s ? top1 : top0)) continue;
      const int ncs = s ? nch1 : nch0;
      cs[s] = reserve(&A.ctl->t_slot_next, 2, A.cap_t);
      cr[s] = reserve(&A.ctl->t_cnt_next, ncs + 2, A.cap_c);
      ib[s] = reserve(&A.ctl->ti_tail, ncs, A.cap_c);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int ncs = s ? nch1 : nch0;
      const int4 pl = (cs[s] >= 0 && cr[s] >= 0 && ib[s] >= 0) ? make_int4(cs[s], cr[s], ib[s], ncs + 2)
                                                             : make_int4(-1, -1, -1, 0);
      S.plan[s] = pl;
      A.tplan[2 * slot + s] = pl;
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int4 pl = S.plan[s];
    if (pl.x < 0) continue;
    unsigned* zb = tbins_at(A, pl.x);
    for (int w = tid; w < 2 * kBinWords; w += kBlock) zb[w] = 0u;
    if (tid < 2) A.tdone[pl.x + tid] = 0;
    unsigned* zc = tccnt_at(A, pl.y);
    unsigned* zs = tscnt_at(A, pl.y);
    for (int w = tid; w < pl.w * kCntStride; w += kBlock) {
      zc[w] = 0u;
      zs[w] = 0u;
    }
  }
}

// Chunk j of big node T (one CTA): Eq. 2 at every bin plane from the node's
// merged bins (every chunk of the node picks the same plane), stable
// partition of the chunk into the other record buffer, and on the way the
// bins and per-chunk counts of the children that are big nodes too.  The CTA
// that finishes the node's last chunk writes the node and creates its
// children: big ones get their chunk items, the others go to the subtree
// queue.  No CTA ever waits for another.
__device__ void top_chunk(const BuildArgs& A, TopSmem& S, const TopTask& T, int slot, int j, int epoch,
                          WarpStats& ts) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = A.K, K3 = 3 * K, CH = A.chunk;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int n = T.count;
  const int par = T.parity & 1;
  const float4* src = A.rec[par];
  float4* dst = A.rec[par ^ 1];
  const int r0 = j * CH;
  const int rn = min(CH, n - r0);
  // the chunk's records, in flight while the split is chosen
  float4 lo[kMaxRpt], hi[kMaxRpt];
#pragma unroll
  for (int r = 0; r < kMaxRpt; ++r) {
    const int k = r * kBlock + tid;
    lo[r] = hi[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < A.rpt && k < rn) {
      const float4* p = src + 2 * ((size_t)T.begin + r0 + k);
      lo[r] = __ldcg(p);
      hi[r] = __ldcg(p + 1);
    }
  }
  {
    for (int w = tid; w < 2 * kBinWords; w += kBlock) (&S.cbins[0][0])[w] = 0u;
    for (int w = tid; w < 4 * kCntStride; w += kBlock) (&S.ccnt[0][0][0])[w] = 0u;
  }
  float cmin[3], scl[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cmin[a] = T.clo[a];
    scl[a] = bin_scale(T.clo[a], T.chi[a], K);
  }
  __syncthreads();
  // Eq. 2 at every plane.  Up to 10 bins warp 0 evaluates all three axes in
  // one pass; otherwise warp a evaluates axis a (a < 3).  The others wait at
  // the barrier and read the choice from shared memory.  An axis without
  // extent has all records in bin 0 and yields no candidate.
  Split best;
  if (warp < (3 * K <= 32 ? 1 : 3)) {
    Split sp;
    split_none(sp);
    if (3 * K <= 32)
      eval_axes(S.pbins, K, n, 0, 3, A.cp, sp);
    else
      eval_axis(S.pbins, K, n, warp, A.cp, sp);
    if (lane == 0) S.ax[warp] = sp;
  }
  __syncthreads();
  if (3 * K <= 32) {
    best = S.ax[0];
  } else {
    best = S.ax[0];
#pragma unroll
    for (int a = 1; a < 3; ++a) {
      const float ca = S.ax[a].cost;
      const int ka = S.ax[a].cand;
      if (ka != INT_MAX && (ca < best.cost || (ca == best.cost && ka < best.cand))) best = S.ax[a];
    }
  }
  int axis, plane, nl;
  BinU cu0, cu1;
  if (best.cand != INT_MAX) {
    axis = best.cand / (K - 1);
    plane = 1 + best.cand % (K - 1);
    nl = best.L.n;
    cu0 = best.L;
    cu1 = best.R;
  } else {  // no usable plane: split the range in the middle, children take the node's bounds
    axis = -1;
    plane = 0;
    nl = n / 2;
    BinU node = binu_empty();
    for (int b = 0; b < K; ++b) node = binu_join(node, binu_load(S.pbins + b * kBinVals));
    node.a0 = T.clo[0];
    node.a1 = T.clo[1];
    node.a2 = T.clo[2];
    node.b0 = T.chi[0];
    node.b1 = T.chi[1];
    node.b2 = T.chi[2];
    cu0 = node;
    cu1 = node;
  }
  const int nr = n - nl;
  cu0.n = nl;
  cu1.n = nr;
  const bool top0 = nl > A.big, top1 = nr > A.big;
  const int nch0 = (nl + CH - 1) / CH, nch1 = (nr + CH - 1) / CH;
  const int cfirst0 = T.chunk_res, cfirst1 = T.chunk_res + nch0;
  if (j == 0) top_plan(A, S, slot, top0, top1, nch0, nch1);
  const float cmin0[3] = {cu0.a0, cu0.a1, cu0.a2}, cmin1[3] = {cu1.a0, cu1.a1, cu1.a2};
  const float scl0[3] = {bin_scale(cu0.a0, cu0.b0, K), bin_scale(cu0.a1, cu0.b1, K), bin_scale(cu0.a2, cu0.b2, K)};
  const float scl1[3] = {bin_scale(cu1.a0, cu1.b0, K), bin_scale(cu1.a1, cu1.b1, K), bin_scale(cu1.a2, cu1.b2, K)};
  // records of the node's earlier chunks that go left: 32-chunk group
  // totals, then the chunks of this chunk's own group
  int lbase;
  if (axis >= 0) {
    const int g = j >> 5;
    const int ng = g * plane, nc = (j - 32 * g) * plane;
    int part = 0;
    for (int it = tid; it < ng + nc; it += kBlock) {
      if (it < ng) {
        const int q = it / plane, b = it - q * plane;
        part += (int)__ldcg(tscnt_at(A, T.chunk_first + q) + axis * K + b);
      } else {
        const int i2 = it - ng, q = i2 / plane, b = i2 - q * plane;
        part += (int)__ldcg(tccnt_at(A, T.chunk_first + 32 * g + q) + axis * K + b);
      }
    }
    lbase = block_sum(part, S.red);
  } else {
    lbase = min(r0, nl);
  }
  const int rbase = r0 - lbase;
  const int dfirst0 = lbase / CH, dfirst1 = rbase / CH;
  // stable partition of the chunk; the records of children that are big
  // nodes too are binned for them on the way
  int lrun = 0, rrun = 0;
#pragma unroll
  for (int r = 0; r < kMaxRpt; ++r) {
    if (r >= A.rpt || r * kBlock >= rn) break;
    const int k = r * kBlock + tid;
    const bool valid = k < rn;
    bool left = false;
    if (valid) {
      if (axis >= 0) {
        const float cc = axis == 0 ? centre(lo[r].x, hi[r].x)
                                   : (axis == 1 ? centre(lo[r].y, hi[r].y) : centre(lo[r].z, hi[r].z));
        left = bin_of(cc, sel3(cmin[0], cmin[1], cmin[2], axis), sel3(scl[0], scl[1], scl[2], axis), K) < plane;
      } else {
        left = r0 + k < nl;
      }
    }
    __syncwarp();
    const unsigned bal = __ballot_sync(kFull, left);
    if (lane == 0) S.wl[warp] = __popc(bal);
    __syncthreads();
    int woff = 0, rtot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const int v = S.wl[w];
      woff += w < warp ? v : 0;
      rtot += v;
    }
    const int lbefore = woff + __popc(bal & lt_mask);
    const int dest = left ? lbase + lrun + lbefore : rbase + rrun + tid - lbefore;
    const int s = left ? 0 : 1;
    if (valid) {
      if (dest < (s ? nr : nl)) {
        const size_t gp = (size_t)T.begin + (s ? nl : 0) + dest;
        dst[2 * gp] = lo[r];
        dst[2 * gp + 1] = hi[r];
      } else {
        set_status(A.ctl, kStBadSplit, 3);
      }
    }
    if (top0 || top1) {
      const bool act = valid && (s ? top1 : top0);
      const int jj = dest / CH - (s ? dfirst1 : dfirst0);
      const float cx = centre(lo[r].x, hi[r].x), cy = centre(lo[r].y, hi[r].y), cz = centre(lo[r].z, hi[r].z);
      const float cc[3] = {cx, cy, cz};
      const RecCodes rc = rec_codes(lo[r], hi[r], cx, cy, cz);
      int e[3], cell = s * 2 + (jj & 1);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int b = s ? bin_of(cc[a], cmin1[a], scl1[a], K) : bin_of(cc[a], cmin0[a], scl0[a], K);
        e[a] = a * K + b;
        cell = cell * kMaxBins + b;
      }
      bin_add_runs(act ? cell : -1, e, &S.cbins[s][0], &S.ccnt[s][jj & 1][0], rc);
    }
    lrun += rtot;
    rrun += min(kBlock, rn - r * kBlock) - rtot;
    __syncthreads();
  }
  // the children's bins and chunk counts
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if (!(s ? top1 : top0)) continue;
    unsigned* gb = tbins_at(A, T.child_slot + s);
    for (int w = tid; w < K3 * kBinVals; w += kBlock) {
      const unsigned v = S.cbins[s][w];
      if (v) {
        if (w % kBinVals == 0)
          atomicAdd(gb + w, v);
        else
          atomicMax(gb + w, v);
      }
    }
    const int cf = s ? cfirst1 : cfirst0, df = s ? dfirst1 : dfirst0, ncs = s ? nch1 : nch0;
    for (int q = tid; q < 2 * K3; q += kBlock) {
      const int jj = q / K3, e = q - jj * K3;
      const unsigned v = S.ccnt[s][jj][e];
      const int chunk = df + jj;
      if (v && chunk < ncs) {
        atomicAdd(tccnt_at(A, cf + chunk) + e, v);
        atomicAdd(tscnt_at(A, cf + (chunk >> 5)) + e, v);
      }
    }
  }
  // the last chunk of the node to finish writes it and creates its children:
  // the count is an acquire-release add (this CTA's writes, ordered before
  // thread 0 by the barrier, are released with it; the last chunk's thread 0
  // acquires every other chunk's, among them chunk 0's plan)
  __syncthreads();
  if (tid == 0) S.last = atom_add_acq_rel(&A.tdone[slot], 1) == T.nchunk - 1;
  __syncthreads();
  if (S.last) top_emit(A, S, T, slot, epoch, nl, nr, cu0, cu1, top0, top1, nch0, nch1, cfirst0, cfirst1, ts);
}

// Write the node split by the chunks just finished and create its children
// (the CTA that finished the node's last chunk), with what chunk 0 reserved
// for them; tree facts go to the CTA's own tally (thread 0).
__device__ void top_emit(const BuildArgs& A, TopSmem& S, const TopTask& T, int slot, int epoch, int nl, int nr,
                         const BinU& cu0, const BinU& cu1, bool top0, bool top1, int nch0, int nch1, int cfirst0,
                         int cfirst1, WarpStats& ts) {
  const int tid = threadIdx.x;
  const int par = T.parity & 1;
  if (tid == 0) {
    S.np = 0;
    const int id = T.begin + nl - 1;
    const int refl = nl <= A.max_leaf ? leaf_ref(T.begin, nl) : INT_MAX;
    const int refr = nr <= A.max_leaf ? leaf_ref(T.begin + nl, nr) : INT_MAX;
    write_node(A, id, T.parent, T.side, cu0, refl, nl, cu1, refr, nr, epoch);
    note_node(ts, nl, nr, refl != INT_MAX, refr != INT_MAX, T.depth);
    for (int s = 0; s < 2; ++s) {
      const int cn = s ? nr : nl, cb = T.begin + (s ? nl : 0);
      const BinU& cu = s ? cu1 : cu0;
      S.created[s] = 0;
      if (cn <= A.max_leaf) {
        if (par == 0) S.ptask[S.np++] = make_task(cb, cn, id, s, T.depth + 1, cu, 1);  // copy to buffer 0
        continue;
      }
      if (s ? top1 : top0) {
        const int4 pl = __ldcg(A.tplan + 2 * slot + s);
        if (pl.x >= 0) {
          TopTask X;
          X.begin = cb;
          X.count = cn;
          X.parent = id;
          X.side = s;
          X.clo[0] = cu.a0;
          X.clo[1] = cu.a1;
          X.clo[2] = cu.a2;
          X.chi[0] = cu.b0;
          X.chi[1] = cu.b1;
          X.chi[2] = cu.b2;
          X.depth = T.depth + 1;
          X.nchunk = s ? nch1 : nch0;
          X.chunk_first = s ? cfirst1 : cfirst0;
          X.child_slot = pl.x;
          X.chunk_res = pl.y;
          X.parity = par ^ 1;
          A.ttask[T.child_slot + s] = X;
          S.created[s] = 1;
          S.ibase[s] = pl.z;
          continue;
        }
      }
      S.ptask[S.np++] = make_task(cb, cn, id, s, T.depth + 1, cu, par ^ 1);  // pools full: a warp takes it
    }
    if (S.created[0] || S.created[1])
      atomicAdd(&A.ctl->ti_pending, (S.created[0] ? nch0 : 0) + (S.created[1] ? nch1 : 0));
  }
  __syncthreads();
  // publish the children's chunk items: each release store also publishes
  // what every thread wrote before the barrier (the tasks, the pending
  // count); meanwhile a thread of warp 1 hands the subtree-sized children to
  // the subtree queue (one reservation, release stores), so that neither
  // publication waits for the other's fence
  if (tid == 32 && S.np > 0) push_tasks(A, S.ptask, S.np, epoch);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if (!S.created[s]) continue;
    const int ncs = s ? nch1 : nch0;
    for (int q = tid; q < ncs; q += kBlock) {
      A.titem[S.ibase[s] + q] = make_int2(T.child_slot + s, q);
      st_release(&A.tready[S.ibase[s] + q], epoch);
    }
  }
}

// Chunk j of big node `slot`, after checking the node's fields.
__device__ void top_item(const BuildArgs& A, TopSmem& S, int slot, int j, int epoch, WarpStats& ts) {
  const int tid = threadIdx.x;
  TopTask T;
  bool ok = slot >= 0 && slot < A.cap_t;
  // the node's merged bins depend on the slot only: their loads go out with
  // the task's, into shared memory once both have arrived
  constexpr int kPer = (kBinWords + kBlock - 1) / kBlock;
  const int nw = 3 * A.K * kBinVals;
  unsigned bv[kPer];
  if (ok) {
    const unsigned* gb = tbins_at(A, slot);
#pragma unroll
    for (int q = 0; q < kPer; ++q) bv[q] = tid + q * kBlock < nw ? __ldcg(gb + tid + q * kBlock) : 0u;
    T = load_top_cg(A.ttask + slot);
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      if (tid + q * kBlock < nw) S.pbins[tid + q * kBlock] = bv[q];
  }
  const int n = ok ? T.count : 0;
  ok = ok && T.begin >= 0 && n > A.big && T.begin <= A.n - n && j >= 0 && j < T.nchunk && T.chunk_first >= 0 &&
       T.chunk_first + T.nchunk <= A.cap_c && T.child_slot >= 0 && T.child_slot + 2 <= A.cap_t &&
       T.chunk_res >= 0 && T.chunk_res + T.nchunk + 2 <= A.cap_c;
  if (!ok) {
    if (tid == 0) set_status(A.ctl, kStBadSplit, 4);
  } else {
    top_chunk(A, S, T, slot, j, epoch, ts);
  }
}

__device__ void top_loop(const BuildArgs& A, TopSmem& S, int epoch) {
  WarpStats ts{0, 0, 0, 0};  // thread 0's tally of the nodes this CTA wrote
  for (;;) {
    if (threadIdx.x == 0) S.item = claim_item(A, epoch);
    __syncthreads();
    const int2 it = S.item;
    __syncthreads();
    if (it.x < 0) break;
    top_item(A, S, it.x, it.y, epoch, ts);
    __syncthreads();
    // release: the subtree tasks this item pushed are counted before the
    // item stops counting (the warps' exit test reads ti_pending first)
    if (threadIdx.x == 0) red_release_add(&A.ctl->ti_pending, -1);
  }
  if (threadIdx.x == 0) {
    if (ts.n_int) atomicAdd(&A.ctl->n_internal, ts.n_int);
    if (ts.n_leaf) atomicAdd(&A.ctl->n_leaves, ts.n_leaf);
    if (ts.big) atomicMax(&A.ctl->max_leaf_size, ts.big);
    if (ts.deep) atomicMax(&A.ctl->depth2, ts.deep);
  }
}

// ------------------------------------------------------------------ small subtrees
// A node of at most 32 triangles is finished by one warp in registers: lane
// j holds record j of the node's range in Morton order.  Every split of the
// subtree is the minimum of Eq. 2 over all splits of that order, evaluated
// from warp scans of the records' boxes; ranges never move, so there is no
// partition step, and all nodes of one level of the subtree are split
// together (scans that stop at each node's bounds).
struct Box6 {
  float l0, l1, l2, h0, h1, h2;
};
__device__ __forceinline__ Box6 box_empty() { return {FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX}; }
__device__ __forceinline__ Box6 box_join(const Box6& a, const Box6& b) {
  return {fminf(a.l0, b.l0), fminf(a.l1, b.l1), fminf(a.l2, b.l2),
          fmaxf(a.h0, b.h0), fmaxf(a.h1, b.h1), fmaxf(a.h2, b.h2)};
}
__device__ __forceinline__ Box6 box_shfl_up(const Box6& a, int o) {
  return {__shfl_up_sync(kFull, a.l0, o), __shfl_up_sync(kFull, a.l1, o), __shfl_up_sync(kFull, a.l2, o),
          __shfl_up_sync(kFull, a.h0, o), __shfl_up_sync(kFull, a.h1, o), __shfl_up_sync(kFull, a.h2, o)};
}
__device__ __forceinline__ Box6 box_shfl_down(const Box6& a, int o) {
  return {__shfl_down_sync(kFull, a.l0, o), __shfl_down_sync(kFull, a.l1, o), __shfl_down_sync(kFull, a.l2, o),
          __shfl_down_sync(kFull, a.h0, o), __shfl_down_sync(kFull, a.h1, o), __shfl_down_sync(kFull, a.h2, o)};
}
__device__ __forceinline__ Box6 box_shfl(const Box6& a, int src) {
  return {__shfl_sync(kFull, a.l0, src), __shfl_sync(kFull, a.l1, src), __shfl_sync(kFull, a.l2, src),
          __shfl_sync(kFull, a.h0, src), __shfl_sync(kFull, a.h1, src), __shfl_sync(kFull, a.h2, src)};
}


__device__ void micro_build(const BuildArgs& A, float4 rlo, float4 rhi, int n, int gbase, int parent, int side,
                            int depth, int epoch, WarpStats& ws) {
  const int lane = threadIdx.x & 31;
  // every lane follows the node its record belongs to: range [b, e), its
  // parent, side and depth; lanes past n sit in empty ranges of their own
  const bool valid = lane < n;
  int b = valid ? 0 : lane, e = valid ? n : lane + 1;
  int par = parent, sd = side, dep = depth;
  const Box6 x = valid ? Box6{rlo.x, rlo.y, rlo.z, rhi.x, rhi.y, rhi.z} : box_empty();
  int n_int = 0, n_leaf = 0, big = 0, deep = 0;  // per node, counted by its first lane
  for (int level = 0; level < 32; ++level) {
    const bool active = valid && e - b > A.max_leaf;
    if (!__any_sync(kFull, active)) break;
    // unions of the records from the start of the lane's node up to the lane
    // (ip) and from the lane to the node's end (is): scans that stop at the
    // node's bounds, all nodes of the level at once
    Box6 ip = x, is = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Box6 u = box_shfl_up(ip, o), d = box_shfl_down(is, o);
      if (lane - o >= b) ip = box_join(ip, u);
      if (lane + o < e) is = box_join(is, d);
    }
    const Box6 sufn = box_shfl_down(is, 1);    // records after the lane, within the node
    const Box6 node = box_shfl(ip, e - 1);     // the whole node
    const float3 clo = make_float3(node.l0, node.l1, node.l2), chi = make_float3(node.h0, node.h1, node.h2);
    // candidate: the lane is the last left record
    float cost = INFINITY;
    int cq = 1 << 20;
    if (active && lane + 1 < e) {
      const float c = eq2_cost(make_float3(ip.l0, ip.l1, ip.l2), make_float3(ip.h0, ip.h1, ip.h2), lane - b + 1,
                               make_float3(sufn.l0, sufn.l1, sufn.l2), make_float3(sufn.h0, sufn.h1, sufn.h2),
                               e - lane - 1, clo, chi, A.cp);
      if (c < INFINITY) {
        cost = c;
        cq = lane;
      }
    }
    // lowest cost of the node (ties: lowest position), found at its last lane
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float oc = __shfl_up_sync(kFull, cost, o);
      const int oq = __shfl_up_sync(kFull, cq, o);
      if (lane - o >= b && (oc < cost || (oc == cost && oq < cq))) {
        cost = oc;
        cq = oq;
      }
    }
    const int wq = __shfl_sync(kFull, cq, e - 1);
    const int q = !active ? lane : (wq < (1 << 20) ? wq : (b + e) / 2 - 1);  // no finite cost: middle
    const int j = q + 1;                                                       // first record of the right child
    const Box6 L = box_shfl(ip, q);
    const Box6 R = box_shfl(is, min(j, 31));
    if (active) {
      const int id = gbase + q;
      const int nl = j - b, nr = e - j;
      const int rl = nl <= A.max_leaf ? leaf_ref(gbase + b, nl) : INT_MAX;
      const int rr = nr <= A.max_leaf ? leaf_ref(gbase + j, nr) : INT_MAX;
      if (lane == b) {
        Node2 nd;
        nd.a_lo = make_float4(L.l0, L.l1, L.l2, __int_as_float(rl));
        nd.a_hi = make_float4(L.h0, L.h1, L.h2, __int_as_float(nl));
        nd.b_lo = make_float4(R.l0, R.l1, R.l2, __int_as_float(rr));
        nd.b_hi = make_float4(R.h0, R.h1, R.h2, __int_as_float(nr));
        A.node2[id] = nd;
        if (par < 0)
          A.ctl->root_ref = id;
        else if (par < A.n - 1)
          *(sd == 0 ? &A.node2[par].a_lo.w : &A.node2[par].b_lo.w) = __int_as_float(id);
        else
          set_status(A.ctl, kStBadLink, 4);
        A.link2[id] = make_int2(par, epoch);
        ++n_int;
        deep = max(deep, dep);
        if (rl != INT_MAX) {
          ++n_leaf;
          big = max(big, nl);
          deep = max(deep, dep + 1);
        }
        if (rr != INT_MAX) {
          ++n_leaf;
          big = max(big, nr);
          deep = max(deep, dep + 1);
        }
      }
      // follow the child holding this lane's record
      if (lane < j) {
        e = j;
        sd = 0;
      } else {
        b = j;
        sd = 1;
      }
      par = id;
      ++dep;
    }
  }
  ws.n_int += __reduce_add_sync(kFull, n_int);
  ws.n_leaf += __reduce_add_sync(kFull, n_leaf);
  ws.big = max(ws.big, (int)__reduce_max_sync(kFull, (unsigned)big));
  ws.deep = max(ws.deep, (int)__reduce_max_sync(kFull, (unsigned)deep));
}

// A node of at most 32 records, record `lane` in registers (lo, hi): order
// them by (Morton key, id) with a warp bitonic sort, write them to buffer 0
// at gbegin in that order (the final order of their leaves) and build the
// subtree.
__device__ void micro_sort_build(const BuildArgs& A, float4 lo, float4 hi, int gbegin, int n, int parent, int side,
                                 int depth, int epoch, WarpStats& ws) {
  const int lane = threadIdx.x & 31;
  unsigned long long key =
      lane < n ? ((unsigned long long)__float_as_uint(hi.w) << 32) | (unsigned)__float_as_int(lo.w) : ~0ull;
  int src = lane;
  __syncwarp();
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(kFull, key, jj);
      const int os = __shfl_xor_sync(kFull, src, jj);
      const bool up = (lane & k) == 0;
      const bool lower = (lane & jj) == 0;
      const bool take = (lower == up) ? (ok < key) : (ok > key);
      if (take) {
        key = ok;
        src = os;
      }
    }
  }
  const float4 slo = make_float4(__shfl_sync(kFull, lo.x, src), __shfl_sync(kFull, lo.y, src),
                                 __shfl_sync(kFull, lo.z, src), __shfl_sync(kFull, lo.w, src));
  const float4 shi = make_float4(__shfl_sync(kFull, hi.x, src), __shfl_sync(kFull, hi.y, src),
                                 __shfl_sync(kFull, hi.z, src), __shfl_sync(kFull, hi.w, src));
  if (lane < n) {
    float4* p = A.rec[0] + 2 * ((size_t)gbegin + lane);
    p[0] = slo;
    p[1] = shi;
  }
  if (__any_sync(kFull, n > A.max_leaf)) micro_build(A, slo, shi, n, gbegin, parent, side, depth, epoch, ws);
}

// micro_sort_build of a node whose records sit in global buffer `parity`.
__device__ void micro_task(const BuildArgs& A, int begin, int n, int parity, int parent, int side, int depth,
                           int epoch, WarpStats& ws) {
  const int lane = threadIdx.x & 31;
  float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
  if (lane < n) {
    const float4* p = A.rec[parity] + 2 * ((size_t)begin + lane);
    lo = __ldcg(p);
    hi = __ldcg(p + 1);
  }
  micro_sort_build(A, lo, hi, begin, n, parent, side, depth, epoch, ws);
}

// ------------------------------------------------------------------ subtree queue
// Claiming subtree tasks, and the split of tasks too large for a CTA's
// shared memory (more than kSubMax records: a big node whose pools were
// full, or any task when big = T / 4096 > 1024), done in global memory by
// one warp until the part it keeps fits.
struct MidWarp {
  unsigned bins[kBinWords];
  float4 stage[2 * kStageW];
};
// One thread takes the next queue slot and waits for it to be filled (the
// other threads of the CTA wait at a barrier; nothing warp-synchronous runs
// in this loop).  Returns false when the queue is drained (no big node and
// no task pending) or the build failed.  The wait is bounded: spin_limit
// polls without progress set a timeout status.
__device__ bool claim_task(const BuildArgs& A, int epoch, Task& t) {
  const int s = atomicAdd(&A.ctl->qa_head, 1);
  int seen = -1;
  for (int it = 0;; ++it) {
    if (s < A.qa_cap && ld_acquire(&A.qa_ready[s]) == epoch) {
      const int4* q = reinterpret_cast<const int4*>(A.qa + s);
      const int4 a = __ldcg(q), b = __ldcg(q + 1), c = __ldcg(q + 2);
      t.begin = a.x;
      t.count = a.y;
      t.parent = a.z;
      t.side = a.w;
      t.clo[0] = __int_as_float(b.x);
      t.clo[1] = __int_as_float(b.y);
      t.clo[2] = __int_as_float(b.z);
      t.depth = b.w;
      t.chi[0] = __int_as_float(c.x);
      t.chi[1] = __int_as_float(c.y);
      t.chi[2] = __int_as_float(c.z);
      t.pad = c.w;
      return true;
    }
    if ((it & 3) == 0) {
      // done when no big node is left and then no subtree task either
      if (ld_acquire(&A.ctl->ti_pending) == 0 && ld_volatile(&A.ctl->qa_pending) == 0) return false;
      if (ld_volatile(&A.ctl->status) != 0) return false;
      const int prog = ld_volatile(&A.ctl->qa_tail) + ld_volatile(&A.ctl->ti_head);
      if (prog != seen) {  // work moved: restart the no-progress budget
        seen = prog;
        it = 0;
      }
    }
    if (it > A.spin_limit) {
      set_status(A.ctl, kStQueueTimeout, 1);
      return false;
    }
    __nanosleep(200);
  }
}

// Split one node of more than 32 triangles with one warp (bin, Eq. 2, stable
// partition), write it, and route its children: the larger internal child
// becomes *cont, the other is queued, small ones are finished here.
__device__ void mid_split(const BuildArgs& A, MidWarp& W, const Task& t, int epoch, WarpStats& ws, Task& cont,
                          bool& have_cont) {
  const int lane = threadIdx.x & 31;
  const int K = A.K, K3 = 3 * K, n = t.count, par = t.pad & 1;
  const float4* src = A.rec[par] + 2 * (size_t)t.begin;
  float4* dst = A.rec[par ^ 1] + 2 * (size_t)t.begin;
  const bool staged = n <= kStageW;
  float cmin[3], scl[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cmin[a] = t.clo[a];
    scl[a] = bin_scale(t.clo[a], t.chi[a], K);
  }
  for (int w = lane; w < K3 * kBinVals; w += 32) W.bins[w] = 0u;
  if (staged) {  // two records per lane in flight
    for (int k0 = lane; k0 < n; k0 += 64) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (k0 + 32 * u < n) {
          v[2 * u] = __ldcg(src + 2 * (k0 + 32 * u));
          v[2 * u + 1] = __ldcg(src + 2 * (k0 + 32 * u) + 1);
        }
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (k0 + 32 * u < n) {
          W.stage[2 * (k0 + 32 * u)] = v[2 * u];
          W.stage[2 * (k0 + 32 * u) + 1] = v[2 * u + 1];
        }
    }
  }
  __syncwarp();
  // lane l bins records l*c .. l*c + c - 1: lanes work on distant records,
  // which seldom share a bin, so plain atomics rarely collide
  {
    const int c = (n + 31) / 32;
    for (int i = 0; i < c; ++i) {
      const int k = lane * c + i;
      if (k < n) {
        const float4 lo = staged ? W.stage[2 * k] : __ldcg(src + 2 * k);
        const float4 hi = staged ? W.stage[2 * k + 1] : __ldcg(src + 2 * k + 1);
        const float cx = centre(lo.x, hi.x), cy = centre(lo.y, hi.y), cz = centre(lo.z, hi.z);
        const RecCodes rc = rec_codes(lo, hi, cx, cy, cz);
        bin_add_plain(W.bins + (0 * K + bin_of(cx, cmin[0], scl[0], K)) * kBinVals, rc);
        bin_add_plain(W.bins + (1 * K + bin_of(cy, cmin[1], scl[1], K)) * kBinVals, rc);
        bin_add_plain(W.bins + (2 * K + bin_of(cz, cmin[2], scl[2], K)) * kBinVals, rc);
      }
    }
  }
  __syncwarp();
  Split best;
  split_none(best);
  if (3 * K <= 32) {  // all three axes in one pass
    eval_axes(W.bins, K, n, 0, 3, A.cp, best);
  } else if (2 * K <= 32) {  // x and y in one pass, then z
    eval_axes(W.bins, K, n, 0, 2, A.cp, best);
    if (__any_sync(kFull, scl[2] > 0.f)) eval_axis(W.bins, K, n, 2, A.cp, best);
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (__any_sync(kFull, scl[a] > 0.f)) eval_axis(W.bins, K, n, a, A.cp, best);
  }
  int axis, plane, nl;
  if (best.cand != INT_MAX) {
    axis = best.cand / (K - 1);
    plane = 1 + best.cand % (K - 1);
    nl = best.L.n;
  } else {
    axis = -1;
    plane = 0;
    nl = n / 2;
  }
  const float acmin = sel3(cmin[0], cmin[1], cmin[2], axis < 0 ? 0 : axis);
  const float ascl = sel3(scl[0], scl[1], scl[2], axis < 0 ? 0 : axis);
  // stable partition into the other buffer (child bounds by reduction when
  // no plane was usable)
  int lrun = 0, rrun = 0;
  BinU accL = binu_empty(), accR = binu_empty();
  for (int g = 0; __any_sync(kFull, g < n); g += 32) {
    const int k = g + lane;
    const bool valid = k < n;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    if (valid) {
      if (staged) {
        lo = W.stage[2 * k];
        hi = W.stage[2 * k + 1];
      } else {
        lo = __ldcg(src + 2 * k);
        hi = __ldcg(src + 2 * k + 1);
      }
    }
    bool left = false;
    if (valid) {
      if (axis >= 0) {
        const float cc = axis == 0 ? centre(lo.x, hi.x) : (axis == 1 ? centre(lo.y, hi.y) : centre(lo.z, hi.z));
        left = bin_of(cc, acmin, ascl, K) < plane;
      } else {
        left = k < nl;
      }
    }
    __syncwarp();
    const unsigned bal = __ballot_sync(kFull, left);
    const int rank = __popc(bal & ((1u << lane) - 1u));
    const int dest = left ? lrun + rank : nl + rrun + (lane - rank);
    if (valid && dest < n) {
      dst[2 * dest] = lo;
      dst[2 * dest + 1] = hi;
      if (axis < 0) {
        if (left)
          accL = binu_join(accL, binu_record(lo, hi));
        else
          accR = binu_join(accR, binu_record(lo, hi));
      }
    }
    const int tot = __popc(bal);
    lrun += tot;
    rrun += min(32, n - g) - tot;
  }
  BinU L = best.L, R = best.R;
  if (__any_sync(kFull, axis < 0)) {
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      accL = binu_join(accL, binu_xor(accL, o));
      accR = binu_join(accR, binu_xor(accR, o));
    }
    L = accL;
    R = accR;
  }
  if (lane == 0 && lrun != nl) set_status(A.ctl, kStBadSplit, 2);
  __syncwarp();
  const int nr = n - nl;
  // leaves keep their records in buffer 0
  if (par == 0) {
    if (nl <= A.max_leaf)
      for (int k = lane; k < 2 * nl; k += 32) A.rec[0][2 * (size_t)t.begin + k] = __ldcg(dst + k);
    if (nr <= A.max_leaf)
      for (int k = lane; k < 2 * nr; k += 32) A.rec[0][2 * ((size_t)t.begin + nl) + k] = __ldcg(dst + 2 * nl + k);
  }
  const int id = t.begin + nl - 1;
  const int refl = nl <= A.max_leaf ? leaf_ref(t.begin, nl) : INT_MAX;
  const int refr = nr <= A.max_leaf ? leaf_ref(t.begin + nl, nr) : INT_MAX;
  if (lane == 0) write_node(A, id, t.parent, t.side, L, refl, nl, R, refr, nr, epoch);
  ++ws.n_int;
  const int leaves = (refl != INT_MAX) + (refr != INT_MAX);
  ws.n_leaf += leaves;
  if (refl != INT_MAX) ws.big = max(ws.big, nl);
  if (refr != INT_MAX) ws.big = max(ws.big, nr);
  ws.deep = max(ws.deep, leaves ? t.depth + 1 : t.depth);
  // children: the larger one of more than 32 stays with this warp
  L.n = nl;
  R.n = nr;
  const bool bigl = nl > kMicro, bigr = nr > kMicro;
  const int keep = (bigl && bigr) ? (nl >= nr ? 0 : 1) : (bigl ? 0 : (bigr ? 1 : -1));
  if (keep >= 0) {
    cont = keep == 0 ? make_task(t.begin, nl, id, 0, t.depth + 1, L, par ^ 1)
                     : make_task(t.begin + nl, nr, id, 1, t.depth + 1, R, par ^ 1);
    have_cont = true;
  }
  if (lane == 0) {
    Task out[3];
    int k = 0;
    if (bigl && bigr)  // the other big child
      out[k++] = keep == 0 ? make_task(t.begin + nl, nr, id, 1, t.depth + 1, R, par ^ 1)
                           : make_task(t.begin, nl, id, 0, t.depth + 1, L, par ^ 1);
    // small subtrees go to idle warps while this one goes on down the tree
    if (keep >= 0) {
      if (nl > A.max_leaf && !bigl) out[k++] = make_task(t.begin, nl, id, 0, t.depth + 1, L, par ^ 1);
      if (nr > A.max_leaf && !bigr) out[k++] = make_task(t.begin + nl, nr, id, 1, t.depth + 1, R, par ^ 1);
    }
    push_tasks(A, out, k, epoch);
  }
  __syncwarp();
  if (keep < 0) {
    if (nl > A.max_leaf) micro_task(A, t.begin, nl, par ^ 1, id, 0, t.depth + 1, epoch, ws);
    if (nr > A.max_leaf) micro_task(A, t.begin + nl, nr, par ^ 1, id, 1, t.depth + 1, epoch, ws);
  }
}

// ------------------------------------------------------------------ subtrees in shared memory
// A CTA takes a task of at most kSubMax records, loads its records into
// shared memory once and builds the subtree there.  Every node of more than
// 32 records is split by the whole CTA; the larger child stays with the CTA
// and the smaller one, if it has more than 32 records, goes back to the
// device queue (records to buffer 1) for an idle CTA, so a subtree spreads
// over the SMs as it branches.  Nodes of at most 32 records are collected
// and finished at the end by the warps in parallel, in registers.  Records
// leave shared memory only as leaves, in their final order, into buffer 0.
constexpr int kSubMax = 1024;            // records of a subtree built in shared memory
constexpr int kMicroList = kSubMax / 2;  // nodes of at most 32 records (>= 2 each, disjoint)
constexpr int kBoxVals = 7;              // a subtree bin: count, box lo (complemented codes), box hi
constexpr int kCtaBinWords = 3 * kMaxBins * kBoxVals + 4 * kBinVals;  // bins, then two sets of children's unions
static_assert(kSubMax <= kBlock * 4, "a CTA partition keeps at most 4 records per thread");
static_assert(kSubMax <= 1024 && kMicro < 64, "packed small-node fields");

// A node of the subtree: local range [b, b + n) of shared buffer `par`,
// parent id, side, depth, centroid bounds.
struct SubNode {
  int b, n, parent, side, depth, par;
  float clo[3], chi[3];
};

struct SubSmem {
  float4 rec[2][2 * kSubMax];
  unsigned bins[kCtaBinWords];
  int2 ml[kMicroList];  // nodes of at most 32: (parent, b | n << 10 | side << 16 | par << 17 | depth << 18)
  Task task;
  int red[kWarps];
  int2 pick;  // the split Eq. 2 chose: candidate, records on the left
  int mord[32];  // the order in which the warps take the small nodes (largest first)
  float4 pbox[3];  // and the boxes of its children (left lo, hi; right lo, hi)
  int nm, mnext, got;
};
static_assert(sizeof(MidWarp) <= sizeof(float4) * 2 * 2 * kSubMax, "a warp's global-memory split state fits");

__device__ __forceinline__ SubNode sub_node(int b, int n, int parent, int side, int depth, int par, const BinU& u) {
  SubNode x;
  x.b = b;
  x.n = n;
  x.parent = parent;
  x.side = side;
  x.depth = depth;
  x.par = par;
  x.clo[0] = u.a0;
  x.clo[1] = u.a1;
  x.clo[2] = u.a2;
  x.chi[0] = u.b0;
  x.chi[1] = u.b1;
  x.chi[2] = u.b2;
  return x;
}

// Packed node of at most 32 records; depth is relative to the task (a
// subtree of kSubMax records is less than kSubMax deep).
__device__ __forceinline__ int2 micro_pack(int b, int n, int parent, int side, int depth, int par) {
  return make_int2(parent, b | (n << 10) | (side << 16) | (par << 17) | (depth << 18));
}

// Bin the run of records [k0, k1) of src on all three axes (count and box
// per bin).  Consecutive records of the Morton order mostly share a bin, so
// the run is accumulated in registers and each stretch of equal bins costs
// one flush of shared-memory atomics.
__device__ __forceinline__ void flush_box(unsigned* e, const unsigned* acc) {
  atomicAdd(e, acc[0]);
#pragma unroll
  for (int q = 1; q < kBoxVals; ++q) atomicMax(e + q, acc[q]);
}
__device__ __forceinline__ void bin_run(unsigned* bins, const float4* src, int k0, int k1, int K, const float* cmin,
                                        const float* scl) {
  int key[3] = {-1, -1, -1};
  unsigned acc[3][kBoxVals];
  for (int k = k0; k < k1; ++k) {
    const float4 lo = src[2 * k], hi = src[2 * k + 1];
    const unsigned c6[6] = {~ucode(lo.x), ~ucode(lo.y), ~ucode(lo.z), ucode(hi.x), ucode(hi.y), ucode(hi.z)};
    const float cc[3] = {centre(lo.x, hi.x), centre(lo.y, hi.y), centre(lo.z, hi.z)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int kk = bin_of(cc[a], cmin[a], scl[a], K);
      if (kk != key[a]) {
        if (key[a] >= 0) flush_box(bins + (a * K + key[a]) * kBoxVals, acc[a]);
        key[a] = kk;
        acc[a][0] = 1u;
#pragma unroll
        for (int q = 0; q < 6; ++q) acc[a][1 + q] = c6[q];
      } else {
        acc[a][0] += 1u;
#pragma unroll
        for (int q = 0; q < 6; ++q) acc[a][1 + q] = max(acc[a][1 + q], c6[q]);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (key[a] >= 0) flush_box(bins + (a * K + key[a]) * kBoxVals, acc[a]);
}

// Eq. 2 over the 7-word bins of all three axes (as many axes per warp pass
// as 32 lanes hold).  Only best.cand and best.L.n are used afterwards.
__device__ __forceinline__ void eval_box(const unsigned* bins, int K, int n, const float* scl, const CostP& cp,
                                         Split& best) {
  for (int g = 0; g < 3;) {
    const int m = min(3 - g, 32 / K);
    if (m >= 2 || __any_sync(kFull, scl[g] > 0.f))
      eval_seg<kBoxVals, false>(bins + g * K * kBoxVals, K, n, g, m, cp, best);
    g += m;
  }
}

// A child's union (count, box, centre bounds) accumulated over records: 13
// words in bin order (count, then the codes of a record).
__device__ __forceinline__ void acc13_add(unsigned* v, const RecCodes& c) {
  v[0] += 1u;
#pragma unroll
  for (int q = 0; q < 12; ++q) v[1 + q] = max(v[1 + q], c.v[q]);
}
__device__ __forceinline__ void acc13_warp(unsigned* v) {
  v[0] = __reduce_add_sync(kFull, v[0]);
#pragma unroll
  for (int q = 1; q < kBinVals; ++q) v[q] = __reduce_max_sync(kFull, v[q]);
}

// Copy a leaf's records from shared memory to buffer 0 (its final place).
__device__ __forceinline__ void leaf_out(const BuildArgs& A, const float4* src, int gpos, int n, int t0, int nt) {
  for (int k = t0; k < 2 * n; k += nt) A.rec[0][2 * (size_t)gpos + k] = src[k];
}


// Split node X of the subtree with the whole CTA (split `it` of the task's
// chain): bins (count and box) in one shared array, each thread binning a
// run of records (thread (w, l) takes run l * 8 + w, so the lanes of a warp
// work far apart); Eq. 2 evaluated by warp 0, its choice read by all from
// shared memory (one warp's shuffles instead of eight); stable partition by
// a block scan, which also gathers both children's unions (into one of two
// sets, alternating with `it`) and clears the bins and the other set for
// the next split.  Thread 0 writes the node and routes the other children:
// the smaller one of more than 32 records goes to the device queue, those
// of at most 32 to the small-node list.  If the larger child has more than
// 32 records, every thread makes it X (true) and goes on without a barrier.
__device__ bool cta_split(const BuildArgs& A, SubSmem& S, SubNode& X, int it, int gbegin, int tdepth, int epoch,
                          WarpStats& ws) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = A.K, n = X.n, p = X.par;
  const int nbw = 3 * K * kBoxVals;
  unsigned* cb = S.bins;  // zero on entry
  unsigned* cu = cb + nbw + (it & 1) * 2 * kBinVals;  // the children's unions, 2 x 13 words (zero on entry)
  unsigned* cu_next = cb + nbw + ((it + 1) & 1) * 2 * kBinVals;
  const float4* src = S.rec[p] + 2 * X.b;
  float4* dst = S.rec[p ^ 1] + 2 * X.b;
  float cmin[3], scl[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cmin[a] = X.clo[a];
    scl[a] = bin_scale(X.clo[a], X.chi[a], K);
  }
  // thread t owns records [t c, t c + c), c <= 4, for the partition; runs
  // for the bins use the spread order
  const int c = (n + kBlock - 1) / kBlock;
  {
    const int r = lane * kWarps + warp, k0 = min(r * c, n), k1 = min(k0 + c, n);
    bin_run(cb, src, k0, k1, K, cmin, scl);
  }
  __syncthreads();
  if (warp == 0) {  // one warp evaluates Eq. 2 (the others wait at the barrier)
    Split best;
    split_none(best);
    eval_box(cb, K, n, scl, A.cp, best);
    if (lane == 0) {
      S.pick = make_int2(best.cand, best.L.n);
      // both children's boxes: the unions of the bins' boxes on each side
      S.pbox[0] = make_float4(best.L.l0, best.L.l1, best.L.l2, best.L.h0);
      S.pbox[1] = make_float4(best.L.h1, best.L.h2, best.R.l0, best.R.l1);
      S.pbox[2] = make_float4(best.R.l2, best.R.h0, best.R.h1, best.R.h2);
    }
  }
  __syncthreads();
  const int2 pick = S.pick;
  int axis, plane, nl;
  if (pick.x != INT_MAX) {
    axis = pick.x / (K - 1);
    plane = 1 + pick.x % (K - 1);
    nl = pick.y;
  } else {
    axis = -1;
    plane = 0;
    nl = n / 2;
  }
  const float acmin = sel3(cmin[0], cmin[1], cmin[2], axis < 0 ? 0 : axis);
  const float ascl = sel3(scl[0], scl[1], scl[2], axis < 0 ? 0 : axis);
  const int k0 = min(tid * c, n);
  float4 rl[4], rh[4];
  unsigned fl = 0;
  int cnt = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = k0 + i;
    if (i < c && k < n) {
      rl[i] = src[2 * k];
      rh[i] = src[2 * k + 1];
      bool left;
      if (axis >= 0) {
        const float cc = axis == 0 ? centre(rl[i].x, rh[i].x)
                                   : (axis == 1 ? centre(rl[i].y, rh[i].y) : centre(rl[i].z, rh[i].z));
        left = bin_of(cc, acmin, ascl, K) < plane;
      } else {
        left = k < nl;
      }
      fl |= (unsigned)left << i;
      cnt += left;
    }
  }
  int inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) S.red[warp] = inc;
  __syncthreads();
  int before = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const int v = S.red[w];
    before += w < warp ? v : 0;
    total += v;
  }
  int lb = before + inc - cnt, rb = k0 - lb;
  // the bins are done with (Eq. 2 read them before the barriers above):
  // clear them, and the other unions, for the next split
  for (int w = tid; w < nbw; w += kBlock) cb[w] = 0u;
  if (tid < 2 * kBinVals) cu_next[tid] = 0u;
  // the larger child of more than 32 records stays; the other one of more
  // than 32 goes to the device queue, where an idle CTA takes it, so the
  // subtree spreads over the SMs as it branches: its records go straight to
  // buffer 1 here instead of to shared memory
  const int nr = n - nl;
  const int keep = nl >= nr ? 0 : 1;
  const int ex = (keep == 0 ? nr : nl) > kMicro ? 1 - keep : -1;
  float4* gx = A.rec[1] + 2 * ((size_t)gbegin + X.b);
  unsigned ua[kBinVals], ub[kBinVals];
#pragma unroll
  for (int q = 0; q < kBinVals; ++q) ua[q] = ub[q] = 0u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = k0 + i;
    if (i < c && k < n) {
      const bool left = (fl >> i) & 1u;
      const int d = left ? lb++ : nl + rb++;
      if (d < n) {
        if ((left ? 0 : 1) == ex) {
          __stcg(gx + 2 * d, rl[i]);
          __stcg(gx + 2 * d + 1, rh[i]);
        } else {
          dst[2 * d] = rl[i];
          dst[2 * d + 1] = rh[i];
        }
      }
      const RecCodes rc =
          rec_codes(rl[i], rh[i], centre(rl[i].x, rh[i].x), centre(rl[i].y, rh[i].y), centre(rl[i].z, rh[i].z));
      if (left)
        acc13_add(ua, rc);
      else
        acc13_add(ub, rc);
    }
  }
  // the children's unions: with a plane, count and box are known (Eq. 2's
  // scans) and only the centre bounds (words 7..12) are gathered; without
  // one, all 13 words
  if (axis >= 0) {
#pragma unroll
    for (int q = 7; q < kBinVals; ++q) {
      ua[q] = __reduce_max_sync(kFull, ua[q]);
      ub[q] = __reduce_max_sync(kFull, ub[q]);
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 7; q < kBinVals; ++q) {
        atomicMax(cu + q, ua[q]);
        atomicMax(cu + kBinVals + q, ub[q]);
      }
    }
  } else {
    acc13_warp(ua);
    acc13_warp(ub);
    if (lane == 0) {
      atomicAdd(cu, ua[0]);
      atomicAdd(cu + kBinVals, ub[0]);
#pragma unroll
      for (int q = 1; q < kBinVals; ++q) {
        atomicMax(cu + q, ua[q]);
        atomicMax(cu + kBinVals + q, ub[q]);
      }
    }
  }
  __syncthreads();
  BinU L, R;
  if (axis >= 0) {
    const float4 b0 = S.pbox[0], b1 = S.pbox[1], b2 = S.pbox[2];
    L = {nl, b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, uval(~cu[7]), uval(~cu[8]), uval(~cu[9]), uval(cu[10]),
         uval(cu[11]), uval(cu[12])};
    R = {n - nl, b1.z, b1.w, b2.x, b2.y, b2.z, b2.w, uval(~cu[kBinVals + 7]), uval(~cu[kBinVals + 8]),
         uval(~cu[kBinVals + 9]), uval(cu[kBinVals + 10]), uval(cu[kBinVals + 11]), uval(cu[kBinVals + 12])};
  } else {
    L = binu_load(cu);
    R = binu_load(cu + kBinVals);
  }
  const bool leafl = nl <= A.max_leaf, leafr = nr <= A.max_leaf;
  if (leafl) leaf_out(A, dst, gbegin + X.b, nl, tid, kBlock);
  if (leafr) leaf_out(A, dst + 2 * nl, gbegin + X.b + nl, nr, tid, kBlock);
  const int id = gbegin + X.b + nl - 1;
  if (tid == 0) {
    if (total != nl) set_status(A.ctl, kStBadSplit, 6);
    write_node(A, id, X.parent, X.side, L, leafl ? leaf_ref(gbegin + X.b, nl) : INT_MAX, nl, R,
               leafr ? leaf_ref(gbegin + X.b + nl, nr) : INT_MAX, nr, epoch);
    note_node(ws, nl, nr, leafl, leafr, X.depth);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int cn = s ? nr : nl, b = X.b + (s ? nl : 0);
      if (cn <= A.max_leaf) continue;
      if (s == ex) {
        // the records written to buffer 1 by every thread are ordered before
        // this thread by the barrier; push_task's release store publishes them
        push_task(A, make_task(gbegin + b, cn, id, s, X.depth + 1, s ? R : L, 1), epoch);
      } else if (cn <= kMicro) {
        if (S.nm < kMicroList)
          S.ml[S.nm++] = micro_pack(b, cn, id, s, X.depth + 1 - tdepth, p ^ 1);
        else
          set_status(A.ctl, kStQueueOverflow, 4);
      }
    }
  }
  // every thread takes the kept child from the unions it read (no barrier:
  // thread 0's node write and release fence overlap the next split's
  // binning, which reads only the kept child's records)
  if ((keep ? nr : nl) <= kMicro) return false;
  X = sub_node(X.b + (keep ? nl : 0), keep ? nr : nl, id, keep, X.depth + 1, p ^ 1, keep ? R : L);
  return true;
}

// The warps finish the collected nodes of at most 32 records, one node per
// warp at a time (no node is added any more).
__device__ void micro_phase(const BuildArgs& A, SubSmem& S, int gbegin, int tdepth, int epoch, WarpStats& ws) {
  const int lane = threadIdx.x & 31;
  const int nm = S.nm;
  // more nodes than warps (up to 32): warp 0 orders them largest first, so
  // that the last round of builds holds the quickest ones
  const bool order = nm > kWarps && nm <= 32;
  if (order) {
    if (threadIdx.x < 32) {
      unsigned key = lane < nm ? ((unsigned)(63 - ((S.ml[lane].y >> 10) & 63)) << 8) | (unsigned)lane : 0xffffffffu;
#pragma unroll
      for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
          const unsigned ok = __shfl_xor_sync(kFull, key, jj);
          const bool up = (lane & k) == 0, lower = (lane & jj) == 0;
          if ((lower == up) ? (ok < key) : (ok > key)) key = ok;
        }
      }
      S.mord[lane] = (int)(key & 255u);
    }
    __syncthreads();
  }
  for (;;) {
    int i = 0;
    if (lane == 0) i = atomicAdd(&S.mnext, 1);
    i = __shfl_sync(kFull, i, 0);
    if (i >= nm) break;
    const int2 m = S.ml[order ? S.mord[i] : i];
    const int f = m.y;
    const int b = f & 1023, n = (f >> 10) & 63, side = (f >> 16) & 1, par = (f >> 17) & 1, dep = f >> 18;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    if (lane < n) {
      lo = S.rec[par][2 * (b + lane)];
      hi = S.rec[par][2 * (b + lane) + 1];
    }
    micro_sort_build(A, lo, hi, gbegin + b, n, m.x, side, tdepth + dep, epoch, ws);
  }
}

// Build the subtree of task t (max_leaf < t.count <= kSubMax) in shared
// memory with the whole CTA.
__device__ void sub_tree(const BuildArgs& A, SubSmem& S, const Task& t, int epoch, WarpStats& ws) {
  const int tid = threadIdx.x;
  const int n = t.count;
  const float4* g = A.rec[t.pad & 1] + 2 * (size_t)t.begin;
  for (int k = tid; k < 2 * n; k += kBlock) S.rec[0][k] = __ldcg(g + k);
  // the first split's bins and unions start at zero
  for (int w = tid; w < kCtaBinWords; w += kBlock) S.bins[w] = 0u;
  if (tid == 0) {
    S.nm = 0;
    S.mnext = 0;
    if (n <= kMicro) S.ml[S.nm++] = micro_pack(0, n, t.parent, t.side, 0, 0);
  }
  __syncthreads();
  if (n > kMicro) {  // the chain of larger children, split by the whole CTA
    SubNode X;
    X.b = 0;
    X.n = n;
    X.parent = t.parent;
    X.side = t.side;
    X.depth = t.depth;
    X.par = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      X.clo[a] = t.clo[a];
      X.chi[a] = t.chi[a];
    }
    for (int it = 0; cta_split(A, S, X, it, t.begin, t.depth, epoch, ws); ++it) {
    }
    __syncthreads();  // thread 0's last additions to the small-node list
  }
  micro_phase(A, S, t.begin, t.depth, epoch, ws);
  __syncthreads();
}

// The subtree role of every CTA: take a task from the queue, build its
// subtree (tasks of more than kSubMax records are first split in global
// memory by one warp, down to a part that fits), repeat until the queue is
// drained.
__device__ void sub_loop(const BuildArgs& A, SubSmem& S, int epoch) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  WarpStats ws{0, 0, 0, 0};
  for (;;) {
    if (tid == 0) S.got = claim_task(A, epoch, S.task);
    __syncthreads();
    const bool got = S.got;
    Task t = S.task;
    __syncthreads();
    if (!got) break;
    const int par = t.pad & 1;
    if (t.begin < 0 || t.count < 1 || t.begin > A.n - t.count) {
      if (tid == 0) set_status(A.ctl, kStBadSplit, 5);
    } else if (t.count <= A.max_leaf) {
      // a leaf made by a top level whose records sit in buffer 1
      if (par)
        for (int k = tid; k < 2 * t.count; k += kBlock)
          A.rec[0][2 * (size_t)t.begin + k] = __ldcg(A.rec[1] + 2 * (size_t)t.begin + k);
    } else {
      if (t.count > kSubMax) {
        if (warp == 0) {
          MidWarp& W = *reinterpret_cast<MidWarp*>(&S.rec[0][0]);
          Task cur = t;
          bool more = true;
          while (more && cur.count > kSubMax) {
            Task nx;
            more = false;
            mid_split(A, W, cur, epoch, ws, nx, more);
            if (more) cur = nx;
          }
          if (lane == 0) {
            S.got = more;
            S.task = cur;
          }
        }
        __syncthreads();
        t = S.task;
        const bool more = S.got;
        __syncthreads();
        if (!more) t.count = 0;
      }
      if (t.count > 0) sub_tree(A, S, t, epoch, ws);
    }
    __syncthreads();
    // the pushes of this task counted first, so this never reads zero early
    if (tid == 0) atomicSub(&A.ctl->qa_pending, 1);
  }
  if (lane == 0) {
    if (ws.n_int) atomicAdd(&A.ctl->n_internal, ws.n_int);
    if (ws.n_leaf) atomicAdd(&A.ctl->n_leaves, ws.n_leaf);
    if (ws.big) atomicMax(&A.ctl->max_leaf_size, ws.big);
    if (ws.deep) atomicMax(&A.ctl->depth2, ws.deep);
  }
}

// The split phase: the first top_ctas CTAs work the chunk items of big nodes
// (CTA per item) and then join the others, which take the subtree queue
// (CTA per subtree).  Both run at once, so subtrees proceed while the big
// nodes of other branches are still being split.
union SplitSmem {
  TopSmem top;
  SubSmem sub;
};

__global__ void __launch_bounds__(kBlock, 2) k_split(BuildArgs A) {
  pdl_wait();
  pdl_launch();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SplitSmem& S = *reinterpret_cast<SplitSmem*>(smem_raw);
  const int epoch = __ldcg(&A.ctl->epoch);
  if ((int)blockIdx.x < A.top_ctas) {
    top_loop(A, S.top, epoch);
    __syncthreads();
  }
  sub_loop(A, S.sub, epoch);
}

// ------------------------------------------------------------------ traversal nodes + leaf order
__device__ __forceinline__ void child_of(const Node2& n, int s, int* ref, float3* lo, float3* hi) {
  const float4 l = s == 0 ? n.a_lo : n.b_lo, h = s == 0 ? n.a_hi : n.b_hi;
  *ref = __float_as_int(l.w);
  *lo = make_float3(l.x, l.y, l.z);
  *hi = make_float3(h.x, h.y, h.z);
}

__device__ __forceinline__ Node2 load_node_cg(const Node2* p) {
  const float4* q = reinterpret_cast<const float4*>(p);
  Node2 n;
  n.a_lo = __ldcg(q);
  n.a_hi = __ldcg(q + 1);
  n.b_lo = __ldcg(q + 2);
  n.b_hi = __ldcg(q + 3);
  return n;
}

// A child reference is usable if it is a leaf or a node written by this build.
__device__ __forceinline__ bool ref_ok(const BuildArgs& A, int ref, int epoch) {
  if (ref == INT_MIN) return false;
  if (ref < 0) return true;
  return ref < A.n - 1 && __ldcg(&A.link2[ref]).y == epoch;
}

// The 4-wide node rooted at binary node x: open the internal child of
// largest surface area until there are 4 children (the first of equal areas
// wins; the opened node's children take its slot and the next free one).
// The 64-byte form of wide node w: per axis the grid origin is the union
// box's lower corner and the step 2^e the smallest with 255 steps covering
// its extent; each lower plane takes the largest byte whose decoded value is
// not above it, each upper plane the smallest not below it (checked with
// qplane itself, so the decoded box contains the exact one); when 255 steps
// fall short after rounding, e grows.
__device__ QNode quantize_node(const WNode& w) {
  const float lo[3][4] = {{w.lox.x, w.lox.y, w.lox.z, w.lox.w}, {w.loy.x, w.loy.y, w.loy.z, w.loy.w},
                          {w.loz.x, w.loz.y, w.loz.z, w.loz.w}};
  const float hi[3][4] = {{w.hix.x, w.hix.y, w.hix.z, w.hix.w}, {w.hiy.x, w.hiy.y, w.hiy.z, w.hiy.w},
                          {w.hiz.x, w.hiz.y, w.hiz.z, w.hiz.w}};
  const int ch[4] = {w.child.x, w.child.y, w.child.z, w.child.w};
  QNode q;
  float org[3];
  unsigned wlo[3], whi[3];
  int exps = 0;
  for (int a = 0; a < 3; ++a) {
    float ulo = INFINITY, uhi = -INFINITY;
    for (int i = 0; i < 4; ++i)
      if (ch[i] != INT_MIN) {
        ulo = fminf(ulo, lo[a][i]);
        uhi = fmaxf(uhi, hi[a][i]);
      }
    if (!(ulo <= uhi)) {  // no child
      ulo = 0.f;
      uhi = 0.f;
    }
    int e = -126;
    const float ext = uhi - ulo;
    if (ext > 0.f) {
      int k;
      frexpf(ext * (1.f / 255.f), &k);  // ext / 255 < 2^k
      e = max(-126, min(127, k));
    }
    unsigned bl = 0, bh = 0;
    for (int attempt = 0; attempt < 8; ++attempt) {
      const float s = qscale(e);
      bool ok = true;
      bl = bh = 0;
      for (int i = 0; i < 4; ++i) {
        unsigned ql = 255, qh = 0;  // empty slot: an empty decoded box
        if (ch[i] != INT_MIN) {
          int l = (int)floorf((lo[a][i] - ulo) / s), h = (int)ceilf((hi[a][i] - ulo) / s);
          l = max(0, min(255, l));
          h = max(0, min(255, h));
          while (l > 0 && qplane((unsigned)l, s, ulo) > lo[a][i]) --l;
          while (h < 255 && qplane((unsigned)h, s, ulo) < hi[a][i]) ++h;
          ok = ok && qplane((unsigned)l, s, ulo) <= lo[a][i] && qplane((unsigned)h, s, ulo) >= hi[a][i];
          ql = (unsigned)l;
          qh = (unsigned)h;
        }
        bl |= ql << (8 * i);
        bh |= qh << (8 * i);
      }
      if (ok || e >= 127) break;
      ++e;
    }
    org[a] = ulo;
    wlo[a] = bl;
    whi[a] = bh;
    exps |= (e + 128) << (8 * a);
  }
  q.ox = org[0];
  q.oy = org[1];
  q.oz = org[2];
  q.exps = exps;
  q.lox = wlo[0];
  q.hix = whi[0];
  q.loy = wlo[1];
  q.hiy = whi[1];
  q.loz = wlo[2];
  q.hiz = whi[2];
  q.parent = w.meta.x;
  q.pad = 0;
  q.child = w.child;
  return q;
}

// The W-wide node rooted at binary node x: open the internal child of
// largest surface area until there are W children (the first of equal areas
// wins; the opened node's children take its slot and the next free one).
// Slots past m are empty.
template <int W>
__device__ int collapse(const BuildArgs& A, int x, int epoch, int* ref, float3* lo, float3* hi) {
  const Node2 nd = load_node_cg(A.node2 + x);
  child_of(nd, 0, &ref[0], &lo[0], &hi[0]);
  child_of(nd, 1, &ref[1], &lo[1], &hi[1]);
  int m = 2;
  for (int q = 0; q < 2; ++q)
    if (!ref_ok(A, ref[q], epoch)) {
      set_status(A.ctl, kStBadLink, 1);
      ref[q] = INT_MIN;
    }
  while (m < W) {
    int pick = -1;
    float best = -1.f;
    for (int q = 0; q < m; ++q)
      if (ref[q] >= 0) {
        const float ar = area(lo[q], hi[q]);
        if (ar > best) {
          best = ar;
          pick = q;
        }
      }
    if (pick < 0) break;
    const Node2 g = load_node_cg(A.node2 + ref[pick]);
    child_of(g, 1, &ref[m], &lo[m], &hi[m]);
    child_of(g, 0, &ref[pick], &lo[pick], &hi[pick]);
    for (int q : {pick, m})
      if (!ref_ok(A, ref[q], epoch)) {
        set_status(A.ctl, kStBadLink, 2);
        ref[q] = INT_MIN;
      }
    ++m;
  }
  for (int q = m; q < W; ++q) ref[q] = INT_MIN;
  for (int q = 0; q < W; ++q)
    if (ref[q] == INT_MIN) {
      lo[q] = make_float3(INFINITY, INFINITY, INFINITY);
      hi[q] = make_float3(-INFINITY, -INFINITY, -INFINITY);
    }
  return m;
}

__device__ void make_wide(const BuildArgs& A, int x, int epoch) {
  int ref[4];
  float3 lo[4], hi[4];
  collapse<4>(A, x, epoch, ref, lo, hi);
  WNode w;
  w.lox = make_float4(lo[0].x, lo[1].x, lo[2].x, lo[3].x);
  w.hix = make_float4(hi[0].x, hi[1].x, hi[2].x, hi[3].x);
  w.loy = make_float4(lo[0].y, lo[1].y, lo[2].y, lo[3].y);
  w.hiy = make_float4(hi[0].y, hi[1].y, hi[2].y, hi[3].y);
  w.loz = make_float4(lo[0].z, lo[1].z, lo[2].z, lo[3].z);
  w.hiz = make_float4(hi[0].z, hi[1].z, hi[2].z, hi[3].z);
  w.child = make_int4(ref[0], ref[1], ref[2], ref[3]);
  w.meta = make_int4(__ldcg(&A.link2[x]).x, 0, 0, 0);
  A.wide[x] = w;
  if (A.qwide) A.qwide[x] = quantize_node(w);
}

__device__ void make_wide8(const BuildArgs& A, int x, int epoch) {
  int ref[8];
  float3 lo[8], hi[8];
  collapse<8>(A, x, epoch, ref, lo, hi);
  WNode8 w;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int b = 4 * h;
    w.lox[h] = make_float4(lo[b].x, lo[b + 1].x, lo[b + 2].x, lo[b + 3].x);
    w.hix[h] = make_float4(hi[b].x, hi[b + 1].x, hi[b + 2].x, hi[b + 3].x);
    w.loy[h] = make_float4(lo[b].y, lo[b + 1].y, lo[b + 2].y, lo[b + 3].y);
    w.hiy[h] = make_float4(hi[b].y, hi[b + 1].y, hi[b + 2].y, hi[b + 3].y);
    w.loz[h] = make_float4(lo[b].z, lo[b + 1].z, lo[b + 2].z, lo[b + 3].z);
    w.hiz[h] = make_float4(hi[b].z, hi[b + 1].z, hi[b + 2].z, hi[b + 3].z);
    w.child[h] = make_int4(ref[b], ref[b + 1], ref[b + 2], ref[b + 3]);
  }
  w.meta[0] = make_int4(__ldcg(&A.link2[x]).x, 0, 0, 0);
  w.meta[1] = make_int4(0, 0, 0, 0);
  A.wide8[x] = w;
}

__global__ void __launch_bounds__(kBlock) k_post(BuildArgs A) {
  pdl_wait();
  pdl_launch();
  const int n = A.n;
  const int epoch = __ldcg(&A.ctl->epoch);
  const int gt = blockIdx.x * kBlock + threadIdx.x, gs = gridDim.x * kBlock;
  if (gt == 0) {
    const int r = __ldcg(&A.ctl->root_ref);
    if (r >= 0) {
      A.ctl->wide_root = r;
    } else {  // the whole scene is one leaf (or empty): a wrapper node in slot 0
      WNode w;
      const float inf = INFINITY;
      w.lox = w.loy = w.loz = make_float4(inf, inf, inf, inf);
      w.hix = w.hiy = w.hiz = make_float4(-inf, -inf, -inf, -inf);
      w.child = make_int4(INT_MIN, INT_MIN, INT_MIN, INT_MIN);
      if (r != INT_MIN && leaf_count(r) > 0) {
        w.lox.x = uval(~__ldcg(&A.ctl->sb[0]));
        w.loy.x = uval(~__ldcg(&A.ctl->sb[1]));
        w.loz.x = uval(~__ldcg(&A.ctl->sb[2]));
        w.hix.x = uval(__ldcg(&A.ctl->sb[3]));
        w.hiy.x = uval(__ldcg(&A.ctl->sb[4]));
        w.hiz.x = uval(__ldcg(&A.ctl->sb[5]));
        w.child.x = r;
      }
      w.meta = make_int4(-1, 0, 0, 0);
      if (A.wide8) {
        WNode8 w8;
        w8.lox[0] = w.lox;
        w8.hix[0] = w.hix;
        w8.loy[0] = w.loy;
        w8.hiy[0] = w.hiy;
        w8.loz[0] = w.loz;
        w8.hiz[0] = w.hiz;
        w8.lox[1] = w8.loy[1] = w8.loz[1] = make_float4(inf, inf, inf, inf);
        w8.hix[1] = w8.hiy[1] = w8.hiz[1] = make_float4(-inf, -inf, -inf, -inf);
        w8.child[0] = w.child;
        w8.child[1] = make_int4(INT_MIN, INT_MIN, INT_MIN, INT_MIN);
        w8.meta[0] = w.meta;
        w8.meta[1] = make_int4(0, 0, 0, 0);
        A.wide8[0] = w8;
      } else {
        A.wide[0] = w;
        if (A.qwide) A.qwide[0] = quantize_node(w);
      }
      A.ctl->wide_root = 0;
    }
  }
  for (int i = gt; i < n; i += gs) {
    const int p = __float_as_int(__ldcg(A.rec[0] + 2 * (size_t)i).w);
    if (p < 0 || p >= A.n_all) {
      set_status(A.ctl, kStBadSplit, 20);
      continue;
    }
    A.order[i] = p;
    A.tri_leaf[3 * (size_t)i] = A.tri[3 * (size_t)p];
    A.tri_leaf[3 * (size_t)i + 1] = A.tri[3 * (size_t)p + 1];
    A.tri_leaf[3 * (size_t)i + 2] = A.tri[3 * (size_t)p + 2];
    if (i < n - 1 && __ldcg(&A.link2[i]).y == epoch) {
      if (A.wide8)
        make_wide8(A, i, epoch);
      else
        make_wide(A, i, epoch);
    }
  }
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Launch with programmatic stream serialization when `pdl` is set: the
// kernel may start while its predecessor drains and waits for it in-kernel.
template <typename... P, typename... Q>
cudaError_t launch(void (*k)(P...), int grid, size_t smem, cudaStream_t st, bool pdl, Q... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

}  // namespace

BuildGeom build_geometry(int64_t n, int nsm) {
  BuildGeom g{};
  const int64_t T = n < 1 ? 1 : n;
  g.big = (int)std::max<int64_t>(kBigMin, (T + 4095) / 4096);
  int64_t rpt = (T + (int64_t)nsm * 512 - 1) / ((int64_t)nsm * 512);
  rpt = std::min<int64_t>(std::max<int64_t>(rpt, 1), kMaxRpt);
  g.rpt = (int)rpt;
  g.chunk = kBlock * g.rpt;
  // Pools of one build (a full pool sends further big nodes to the warps,
  // slower but correct).  Big nodes of one depth are disjoint, so there are at
  // most T / big of them per depth; 16 depths' worth covers the uneven trees
  // of alpha < 1.  Chunk counts: a big node reserves its chunks + 2 for its
  // children; per depth that is at most T / chunk + 3 T / big, where
  // T' / chunk(T') <= max(2 nsm, T / 1024) + 1 for every T' <= T.
  const int64_t nb = (T + g.big - 1) / g.big;
  const int64_t nc = std::max<int64_t>(2 * (int64_t)nsm, (T + 1023) / 1024) + 1;
  g.cap_t = (int)(16 * nb + 256);
  g.cap_c = (int)(16 * nc + 3 * (int64_t)g.cap_t + 64);
  // pushes: at most one per binary node of more than max_leaf triangles plus
  // one per leaf cut from a big node
  g.qa_cap = (int)(2 * T + 16);
  return g;
}

cudaError_t launch_build(rt_scene_s* s, const rt_build_params& p, cudaStream_t st) {
  int n = (int)s->n_tri;
  const int* sel = nullptr;
  cudaError_t e;
  if (p.range > 0.f && p.range < 3.0e38f) {
    // the triangles within the ray action range, in input order; the build
    // is sized for their count, which the host reads back (one small copy)
    const int nb = (n + kBlock - 1) / kBlock;
    if (n > 0) {
      const float3 src = make_float3(p.source[0], p.source[1], p.source[2]);
      const float rr = p.range * 1.00001f;
      k_sel_count<<<nb, kBlock, 0, st>>>(s->tri_in, n, src, rr * rr, s->sel_cnt);
      k_sel_scan<<<1, 1024, 0, st>>>(s->sel_cnt, nb);
      k_sel_write<<<nb, kBlock, 0, st>>>(s->tri_in, n, src, rr * rr, s->sel_cnt, s->sel);
      count_launches(3);
      if ((e = cudaGetLastError())) return e;
      if ((e = cudaMemcpyAsync(s->sel_host, s->sel_cnt + nb, sizeof(int), cudaMemcpyDeviceToHost, st))) return e;
      if ((e = cudaStreamSynchronize(st))) return e;
      n = *s->sel_host;
    }
    sel = s->sel;
  }
  s->n_built = n;
  const int nsm = sm_count();
  const BuildGeom g = build_geometry(n, nsm);
  if (g.cap_t > s->geom.cap_t || g.cap_c > s->geom.cap_c || g.qa_cap > s->geom.qa_cap) return cudaErrorInvalidValue;
  BuildArgs A;
  A.tri = s->tri_in;
  A.sel = sel;
  A.rec[0] = s->rec[0];
  A.rec[1] = s->rec[1];
  A.node2 = s->node2;
  A.link2 = s->link2;
  A.ctl = s->ctl;
  A.qa = s->qa;
  A.qa_ready = s->qa_ready;
  A.ttask = s->top_task;
  A.tdone = s->top_done;
  A.tbins = s->top_bins;
  A.tccnt = s->top_ccnt;
  A.tscnt = s->top_scnt;
  A.titem = s->top_item;
  A.tplan = s->top_plan;
  A.tready = s->top_ready;
  A.wide = s->wide;
  A.qwide = p.quantize ? s->qwide : nullptr;
  A.wide8 = p.width == 8 ? s->wide8 : nullptr;
  A.tri_leaf = s->tri_leaf;
  A.order = s->idx[0];
  A.epoch_dev = s->epoch;
  A.n = n;
  A.n_all = (int)s->n_tri;
  A.K = p.bins;
  A.max_leaf = p.max_leaf;
  A.big = g.big;
  A.chunk = g.chunk;
  A.rpt = g.rpt;
  A.cap_t = s->geom.cap_t;
  A.cap_c = s->geom.cap_c;
  A.qa_cap = s->geom.qa_cap;
  static bool attr = false;
  static int split_per_sm = 2;  // resident split CTAs per SM (at most 2)
  if (!attr) {
    if ((e = cudaFuncSetAttribute(k_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SplitSmem))))
      return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_split, kBlock, sizeof(SplitSmem)))) return e;
    split_per_sm = std::max(1, std::min(2, occ));
    attr = true;
  }
  // the big-node chunks go to the first nsm CTAs, which then join the rest on
  // the subtree queue, so that subtrees proceed while other branches' big
  // nodes are split; when a depth has many more chunks than SMs (large
  // scenes) every CTA takes chunks first
  const int64_t nchunks = (n + g.chunk - 1) / g.chunk;
  A.top_ctas = n > g.big ? (nchunks > 8 * (int64_t)nsm ? split_per_sm * nsm : nsm) : 0;
  const DebugHooks dh = debug_hooks();
  A.spin_limit = dh.spin_limit > 0 ? dh.spin_limit : kSpinLimit;
  A.phantom_tasks = dh.phantom_tasks;
  A.phantom_items = dh.phantom_items;
  if (A.phantom_items && !A.top_ctas) A.top_ctas = nsm;  // someone must wait for the phantom items
  A.cp = CostP{p.alpha, p.t_i, p.t_trav, p.source[0], p.source[1], p.source[2], p.dist_norm};
  if ((e = cudaMemsetAsync(s->ctl, 0, sizeof(BuildCtl), st))) return e;
  const int nch = (n + g.chunk - 1) / g.chunk;
  int gp = (n + kBlock - 1) / kBlock;
  gp = std::max(1, std::min(gp, nsm * 8));
  if ((e = launch(k_prep, gp, 0, st, false, A))) return e;
  if ((e = launch(k_bin_root, std::max(1, std::min(nch, nsm * 4)), 0, st, true, A))) return e;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (s->split_ev[0] && (e = cudaStreamIsCapturing(st, &cs))) return e;
  const unsigned evflags = cs == cudaStreamCaptureStatusNone ? cudaEventRecordDefault : cudaEventRecordExternal;
  if (s->split_ev[0] && (e = cudaEventRecordWithFlags(s->split_ev[0], st, evflags))) return e;
  if ((e = launch(k_split, split_per_sm * nsm, sizeof(SplitSmem), st, true, A))) return e;
  if (s->split_ev[1] && (e = cudaEventRecordWithFlags(s->split_ev[1], st, evflags))) return e;
  if ((e = launch(k_post, gp, 0, st, true, A))) return e;
  count_launches(4);
  return cudaSuccess;
}

}  // namespace rt
