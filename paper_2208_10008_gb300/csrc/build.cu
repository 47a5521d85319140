// BVH construction on the device (Sec. II.B-C of arXiv 2208.10008).
//
// Pipeline, all asynchronous on one stream:
//   k_prep        per-triangle AABB (Eq. 3 boxes) + scene / centroid bounds
//   k_morton      30-bit Morton key of each AABB centre (locality presort)
//   radix sort    4 stable LSD passes (8-bit digits): hist, scan, scatter
//   k_make_recs   32-byte records (box + id) in Morton order
//   k_root        the root task (Fig. 2: "calculate the bounding volume that
//                 contains all triangular facets")
//   k_nodes       one CTA per node of more than kMicro triangles, fed by a
//                 device work queue: bin the AABB centres into `bins` slabs
//                 per axis, evaluate Eq. 2 at every bin plane, take the
//                 minimum (ties: lowest axis, lowest plane), stable-partition
//                 the node's range, emit the children (Fig. 2 recursion)
//   k_micro       one warp per node of at most kMicro triangles: its whole
//                 subtree, Eq. 2 over the splits of the range's order
//   k_collapse    binary tree -> 4-wide traversal nodes (greedy by area)
//   k_gather      triangles copied into leaf order
//
// Node identity: the binary node that splits its range at position s gets id
// s - 1.  Split positions of distinct internal nodes differ, so ids need no
// allocator and the tree is the same whatever order the tasks ran in.
#include <cuda_runtime.h>

#include <cfloat>
#include <climits>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int kPrepBlock = 256;
constexpr int kSortBlock = 256;          // one element per thread per tile

__device__ __forceinline__ void set_status(BuildCtl* ctl, int code, int where) {
  if (atomicCAS(&ctl->status, 0, code) == 0) ctl->status_where = where;
}


// AABB centre, evaluated identically wherever a bin is needed.
__device__ __forceinline__ float centre(float lo, float hi) {
  return __fmul_rn(__fadd_rn(lo, hi), 0.5f);
}

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

struct CostP {
  float alpha, t_i, t_trav, sx, sy, sz;
  int dist_norm;
};

// Eq. 2 (Eq. 1 at alpha = 1): children L (nl triangles), R (nr) of node C.
__device__ float eq2_cost(float3 llo, float3 lhi, int nl, float3 rlo, float3 rhi, int nr,
                          float3 clo, float3 chi, const CostP& p) {
  float sc = area(clo, chi);
  float sah = sc > 0.f ? (area(llo, lhi) / sc * (float)nl + area(rlo, rhi) / sc * (float)nr) * p.t_i
                       : (float)(nl + nr) * p.t_i;
  float ax = 0.5f * (llo.x + lhi.x) - p.sx, ay = 0.5f * (llo.y + lhi.y) - p.sy,
        az = 0.5f * (llo.z + lhi.z) - p.sz;
  float bx = 0.5f * (rlo.x + rhi.x) - p.sx, by = 0.5f * (rlo.y + rhi.y) - p.sy,
        bz = 0.5f * (rlo.z + rhi.z) - p.sz;
  float d2 = 0.5f * ((ax * ax + ay * ay + az * az) + (bx * bx + by * by + bz * bz));
  if (p.dist_norm) {
    float dx = chi.x - clo.x, dy = chi.y - clo.y, dz = chi.z - clo.z;
    float diag2 = dx * dx + dy * dy + dz * dz;
    d2 = (diag2 > 0.f ? d2 / diag2 : 0.f) * (float)(nl + nr) * p.t_i;
  }
  return p.alpha * sah + (1.f - p.alpha) * d2 + p.t_trav;
}

// ------------------------------------------------------------------ prep
__global__ void k_init_ctl(BuildCtl* ctl, int qa_cap, int qb_cap, int qc_cap) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    for (int a = 0; a < 3; ++a) {
      ctl->scene_lo[a] = ford(FLT_MAX);
      ctl->scene_hi[a] = ford(-FLT_MAX);
      ctl->cen_lo[a] = ford(FLT_MAX);
      ctl->cen_hi[a] = ford(-FLT_MAX);
    }
    ctl->qa_cap = qa_cap;
    ctl->qb_cap = qb_cap;
    ctl->qc_cap = qc_cap;
    ctl->root_ref = INT_MIN;
  }
}

__global__ void __launch_bounds__(kPrepBlock) k_prep(const float4* __restrict__ tri, int n,
                                                     float4* __restrict__ plo,
                                                     float4* __restrict__ phi, BuildCtl* ctl) {
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  float clo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, chi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float4 a = tri[3 * i], b = tri[3 * i + 1], c = tri[3 * i + 2];
    float3 l = make_float3(fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)),
                           fminf(a.z, fminf(b.z, c.z)));
    float3 h = make_float3(fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)),
                           fmaxf(a.z, fmaxf(b.z, c.z)));
    plo[i] = make_float4(l.x, l.y, l.z, __int_as_float(i));
    phi[i] = make_float4(h.x, h.y, h.z, 0.f);
    float cc[3] = {centre(l.x, h.x), centre(l.y, h.y), centre(l.z, h.z)};
    float ll[3] = {l.x, l.y, l.z}, hh[3] = {h.x, h.y, h.z};
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(lo[k], ll[k]);
      hi[k] = fmaxf(hi[k], hh[k]);
      clo[k] = fminf(clo[k], cc[k]);
      chi[k] = fmaxf(chi[k], cc[k]);
    }
  }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
      clo[k] = fminf(clo[k], __shfl_xor_sync(0xffffffffu, clo[k], o));
      chi[k] = fmaxf(chi[k], __shfl_xor_sync(0xffffffffu, chi[k], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 3; ++k) {
      atomicMin(&ctl->scene_lo[k], ford(lo[k]));
      atomicMax(&ctl->scene_hi[k], ford(hi[k]));
      atomicMin(&ctl->cen_lo[k], ford(clo[k]));
      atomicMax(&ctl->cen_hi[k], ford(chi[k]));
    }
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

__global__ void k_morton(const float4* __restrict__ plo, const float4* __restrict__ phi, int n,
                         const BuildCtl* ctl, uint32_t* __restrict__ keys,
                         int32_t* __restrict__ idx) {
  float cl[3], sc[3];
  for (int a = 0; a < 3; ++a) {
    cl[a] = iford(ctl->cen_lo[a]);
    float ext = iford(ctl->cen_hi[a]) - cl[a];
    sc[a] = ext > 0.f ? 1023.99f / ext : 0.f;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float4 l = plo[i], h = phi[i];
    float c[3] = {centre(l.x, h.x), centre(l.y, h.y), centre(l.z, h.z)};
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
      float f = (c[a] - cl[a]) * sc[a];
      q[a] = (uint32_t)min(max((int)f, 0), 1023);
    }
    keys[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    idx[i] = i;
  }
}

// ------------------------------------------------------------------ radix sort
__global__ void __launch_bounds__(kSortBlock) k_sort_hist(const uint32_t* __restrict__ keys, int n,
                                                          int shift, uint32_t* __restrict__ hist,
                                                          int nblocks, int chunk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int b = blockIdx.x * chunk, e = min(n, b + chunk);
  for (int i = b + threadIdx.x; i < e; i += kSortBlock) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  __syncthreads();
  hist[blockIdx.x * 256 + threadIdx.x] = h[threadIdx.x];
}

// Exclusive offsets of every (block, digit) counter: hist[b * 256 + d] <-
// (elements with digit < d) + (elements with digit d in blocks < b).  One
// CTA, thread d walks digit d over the blocks (coalesced across threads).
__global__ void __launch_bounds__(256) k_sort_scan(uint32_t* hist, int nblocks) {
  __shared__ uint32_t tot[256];
  __shared__ uint32_t wsum[8];
  const int d = threadIdx.x;
  uint32_t run = 0;
  for (int b = 0; b < nblocks; ++b) {
    uint32_t c = hist[b * 256 + d];
    hist[b * 256 + d] = run;
    run += c;
  }
  // exclusive scan of the digit totals
  uint32_t x = run;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if ((d & 31) >= o) x += y;
  }
  if ((d & 31) == 31) wsum[d >> 5] = x;
  __syncthreads();
  uint32_t wofs = 0;
  for (int w = 0; w < (d >> 5); ++w) wofs += wsum[w];
  tot[d] = wofs + x - run;
  __syncthreads();
  const uint32_t base = tot[d];
  for (int b = 0; b < nblocks; ++b) hist[b * 256 + d] += base;
}

// Stable scatter: tiles of 256 elements, warp-major; ranks from match_any.
__global__ void __launch_bounds__(kSortBlock) k_sort_scatter(
    const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    int32_t* __restrict__ vout, int n, int shift, const uint32_t* __restrict__ hist, int nblocks,
    int chunk) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wh[kSortBlock / 32][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  base[threadIdx.x] = hist[blockIdx.x * 256 + threadIdx.x];
  int b = blockIdx.x * chunk, e = min(n, b + chunk);
  for (int t0 = b; t0 < e; t0 += kSortBlock) {
    for (int k = threadIdx.x; k < (kSortBlock / 32) * 256; k += kSortBlock) (&wh[0][0])[k] = 0u;
    __syncthreads();
    int i = t0 + threadIdx.x;
    bool valid = i < e;
    uint32_t key = valid ? kin[i] : 0u;
    int32_t val = valid ? vin[i] : 0;
    uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wh[w][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = 0;
      int dd = threadIdx.x;
      for (int ww = 0; ww < kSortBlock / 32; ++ww) {
        uint32_t c = wh[ww][dd];
        wh[ww][dd] = run;
        run += c;
      }
      __syncthreads();
      if (valid) {
        uint32_t pos = base[d] + wh[w][d] + rank;
        kout[pos] = key;
        vout[pos] = val;
      }
      __syncthreads();
      base[dd] += run;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ root
__global__ void k_root(BuildCtl* ctl, Task* qa, int* qa_ready, Task* qb, int n, int max_leaf,
                       Node2* node2) {
  if (threadIdx.x || blockIdx.x) return;
  if (n <= max_leaf) {
    ctl->root_ref = leaf_ref(0, n);
    ctl->n_leaves = 1;
    ctl->depth2 = 1;
    ctl->max_leaf_size = n;
    return;
  }
  Task t;
  t.begin = 0;
  t.count = n;
  t.parent = -1;
  t.side = 0;
  t.depth = 1;
  t.pad = 0;
  for (int a = 0; a < 3; ++a) {
    t.clo[a] = iford(ctl->cen_lo[a]);
    t.chi[a] = iford(ctl->cen_hi[a]);
  }
  if (n > kMicro) {
    qa[0] = t;
    ctl->qa_tail = 1;
    ctl->qa_pending = 1;
    __threadfence();
    qa_ready[0] = 1;
  } else {
    qb[0] = t;
    ctl->qb_count = 1;
  }
}

// ------------------------------------------------------------------ split core
// Bins: [axis][bin][8] ints: count, lo xyz, hi xyz (ordered floats), pad.
struct SplitResult {
  int axis, plane, nl;  // axis < 0: median fallback
};

// A bin entry is 9 ints: count, lo xyz, hi xyz (ordered floats), 2 pad.  The
// odd stride puts consecutive bins in different shared-memory banks.
constexpr int kBinEnt = 9;
constexpr int kBinStride = 3 * kMaxBins * kBinEnt;  // ints per bin set

// Reset `nsets` bin sets laid out kBinStride ints apart (first 3*K entries used).
__device__ __forceinline__ void bins_zero(int* bins, int K, int nsets, int tid, int nthreads) {
  const int ent = 3 * K;
  const int lo = ford(FLT_MAX), hi = ford(-FLT_MAX);
  for (int k = tid; k < ent * nsets; k += nthreads) {
    const int w = k >= ent ? k / ent : 0;
    int* e = bins + w * kBinStride + (k - w * ent) * kBinEnt;
    e[0] = 0;
    e[1] = lo;
    e[2] = lo;
    e[3] = lo;
    e[4] = hi;
    e[5] = hi;
    e[6] = hi;
  }
}

__device__ __forceinline__ Task load_task_cg(const Task* p) {
  const int4* q = reinterpret_cast<const int4*>(p);
  int4 a = __ldcg(q), b = __ldcg(q + 1), c = __ldcg(q + 2);
  Task t;
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
  return t;
}

__device__ __forceinline__ void bins_add(int* bins, int K, const float cmin[3], const float scl[3],
                                         float4 lo, float4 hi) {
  float c[3] = {centre(lo.x, hi.x), centre(lo.y, hi.y), centre(lo.z, hi.z)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (scl[a] <= 0.f) continue;
    int* bb = bins + (a * K + bin_of(c[a], cmin[a], scl[a], K)) * kBinEnt;
    atomicAdd(bb, 1);
    atomicMin(bb + 1, ford(lo.x));
    atomicMin(bb + 2, ford(lo.y));
    atomicMin(bb + 3, ford(lo.z));
    atomicMax(bb + 4, ford(hi.x));
    atomicMax(bb + 5, ford(hi.y));
    atomicMax(bb + 6, ford(hi.z));
  }
}

// Per-side accumulator of child bounds during the partition pass.
struct Acc {
  float v[24];  // side s: [s*12 + 0..2] lo, [3..5] hi, [6..8] centroid lo, [9..11] centroid hi
  __device__ void init() {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        v[s * 12 + k] = FLT_MAX;
        v[s * 12 + 3 + k] = -FLT_MAX;
        v[s * 12 + 6 + k] = FLT_MAX;
        v[s * 12 + 9 + k] = -FLT_MAX;
      }
  }
  __device__ void add(int s, float4 lo, float4 hi) {
    float l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float c = centre(l[k], h[k]);
      if (s == 0) {
        v[k] = fminf(v[k], l[k]);
        v[3 + k] = fmaxf(v[3 + k], h[k]);
        v[6 + k] = fminf(v[6 + k], c);
        v[9 + k] = fmaxf(v[9 + k], c);
      } else {
        v[12 + k] = fminf(v[12 + k], l[k]);
        v[15 + k] = fmaxf(v[15 + k], h[k]);
        v[18 + k] = fminf(v[18 + k], c);
        v[21 + k] = fmaxf(v[21 + k], c);
      }
    }
  }
  // 24 independent butterflies, interleaved so their shuffles pipeline
  __device__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float y[24];
#pragma unroll
      for (int k = 0; k < 24; ++k) y[k] = __shfl_xor_sync(0xffffffffu, v[k], o);
#pragma unroll
      for (int k = 0; k < 24; ++k) {
        const bool is_min = (k % 12) < 3 || ((k % 12) >= 6 && (k % 12) < 9);
        v[k] = is_min ? fminf(v[k], y[k]) : fmaxf(v[k], y[k]);
      }
    }
  }
};

__device__ __forceinline__ bool goes_left(float4 lo, float4 hi, const SplitResult& sr, int pos,
                                          const float cmin[3], const float scl[3], int K) {
  if (sr.axis < 0) return pos < sr.nl;
  float c = sr.axis == 0 ? centre(lo.x, hi.x) : (sr.axis == 1 ? centre(lo.y, hi.y) : centre(lo.z, hi.z));
  return bin_of(c, cmin[sr.axis], scl[sr.axis], K) < sr.plane;
}

struct BuildArgs {
  float4* rec[2];    // [2T] each: primitive records (lo.xyz, id) (hi.xyz, 0); a task's
                     // range lives in rec[task.pad], its children go to the other one
  Node2* node2;
  BuildCtl* ctl;
  Task* qa;
  int* qa_ready;
  Task* qb;
  int K;
  int max_leaf;
  CostP cp;
};

// Emit the node for task t split into (left, right), both ranges already in
// place.  Called by one thread.  Returns child tasks needing more work in
// out[0..1] (count in *nout) -- the caller routes them to a tier.
__device__ void emit_node(const BuildArgs& A, const Task& t, int nl, const float* acc,
                          Task* out, int* nout) {
  const int id = t.begin + nl - 1;
  int cnt[2] = {nl, t.count - nl};
  int ref[2];
  *nout = 0;
  int leaves = 0, big = 0;
  for (int s = 0; s < 2; ++s) {
    int b = s == 0 ? t.begin : t.begin + nl;
    if (cnt[s] <= A.max_leaf) {
      ref[s] = leaf_ref(b, cnt[s]);
      ++leaves;
      big = max(big, cnt[s]);
    } else {
      ref[s] = INT_MAX;  // patched by the child when it splits
      Task c;
      c.begin = b;
      c.count = cnt[s];
      c.parent = id;
      c.side = s;
      c.depth = t.depth + 1;
      c.pad = 0;
      for (int k = 0; k < 3; ++k) {
        c.clo[k] = acc[s * 12 + 6 + k];
        c.chi[k] = acc[s * 12 + 9 + k];
      }
      out[(*nout)++] = c;
    }
  }
  Node2 nd;
  nd.a_lo = make_float4(acc[0], acc[1], acc[2], __int_as_float(ref[0]));
  nd.a_hi = make_float4(acc[3], acc[4], acc[5], __int_as_float(cnt[0]));
  nd.b_lo = make_float4(acc[12], acc[13], acc[14], __int_as_float(ref[1]));
  nd.b_hi = make_float4(acc[15], acc[16], acc[17], __int_as_float(cnt[1]));
  // children patch a_lo.w / b_lo.w later; write the whole node first
  A.node2[id] = nd;
  if (t.parent < 0) {
    A.ctl->root_ref = id;
  } else {
    float* slot = t.side == 0 ? &A.node2[t.parent].a_lo.w : &A.node2[t.parent].b_lo.w;
    *slot = __int_as_float(id);
  }
  atomicAdd(&A.ctl->n_internal, 1);
  if (leaves) {
    atomicAdd(&A.ctl->n_leaves, leaves);
    atomicMax(&A.ctl->max_leaf_size, big);
    atomicMax(&A.ctl->depth2, t.depth + 1);
  } else {
    atomicMax(&A.ctl->depth2, t.depth);
  }
}

__device__ void push_a(const BuildArgs& A, const Task& c) {
  int s = atomicAdd(&A.ctl->qa_tail, 1);
  if (s >= A.ctl->qa_cap) {
    set_status(A.ctl, kStQueueOverflow, 1);
    return;
  }
  atomicAdd(&A.ctl->qa_pending, 1);
  A.qa[s] = c;
  __threadfence();
  atomicExch(&A.qa_ready[s], 1);
}

__device__ void push_b(const BuildArgs& A, const Task& c) {
  int s = atomicAdd(&A.ctl->qb_count, 1);
  if (s >= A.ctl->qb_cap) {
    set_status(A.ctl, kStQueueOverflow, 2);
    return;
  }
  A.qb[s] = c;
}

// The K-1 planes of axis `a` evaluated by one warp.  Lane 0 accumulates the
// prefix unions of the bins and lane 1 the suffix unions into `scan` (shared,
// 2 x K entries of 7 floats); then lane p evaluates plane p from prefix p-1
// and suffix p.  Every lane gets the best (cost, candidate, left count);
// candidate = a * (K - 1) + plane - 1.  The full prefix is the node box
// (every triangle sits in exactly one bin of an active axis).
__device__ __forceinline__ void warp_axis_best(const int* bins, int K, int n, int a, const CostP& cp,
                                               float* scan, float* best, int* bestc, int* bestnl) {
  const int lane = threadIdx.x & 31;
  if (lane < 2) {
    const bool fwd = lane == 0;
    float c = 0.f, l0 = FLT_MAX, l1 = FLT_MAX, l2 = FLT_MAX, h0 = -FLT_MAX, h1 = -FLT_MAX, h2 = -FLT_MAX;
    for (int i = 0; i < K; ++i) {
      const int b = fwd ? i : K - 1 - i;
      const int* e = bins + (a * K + b) * kBinEnt;
      const int cnt = e[0];
      if (cnt) {
        c += (float)cnt;
        l0 = fminf(l0, iford(e[1]));
        l1 = fminf(l1, iford(e[2]));
        l2 = fminf(l2, iford(e[3]));
        h0 = fmaxf(h0, iford(e[4]));
        h1 = fmaxf(h1, iford(e[5]));
        h2 = fmaxf(h2, iford(e[6]));
      }
      float* o = scan + ((fwd ? 0 : K) + b) * 7;
      o[0] = c;
      o[1] = l0;
      o[2] = l1;
      o[3] = l2;
      o[4] = h0;
      o[5] = h1;
      o[6] = h2;
    }
  }
  __syncwarp();
  *best = INFINITY;
  *bestc = INT_MAX;
  *bestnl = 0;
  if (lane >= 1 && lane < K) {
    const float* L = scan + (lane - 1) * 7;  // bins 0..lane-1
    const float* R = scan + (K + lane) * 7;  // bins lane..K-1
    const float* N = scan + (K - 1) * 7;     // all bins: the node box
    const int lc = (int)L[0];
    if (lc > 0 && lc < n) {
      *best = eq2_cost(make_float3(L[1], L[2], L[3]), make_float3(L[4], L[5], L[6]), lc,
                       make_float3(R[1], R[2], R[3]), make_float3(R[4], R[5], R[6]), n - lc,
                       make_float3(N[1], N[2], N[3]), make_float3(N[4], N[5], N[6]), cp);
      *bestc = a * (K - 1) + lane - 1;
      *bestnl = lc;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, *best, o);
    const int oc = __shfl_xor_sync(0xffffffffu, *bestc, o);
    const int on = __shfl_xor_sync(0xffffffffu, *bestnl, o);
    if (ov < *best || (ov == *best && oc < *bestc)) {
      *best = ov;
      *bestc = oc;
      *bestnl = on;
    }
  }
}

__device__ __forceinline__ SplitResult make_split(int K, int n, float best, int bestc, int bestnl) {
  SplitResult sr;
  if (bestc == INT_MAX || !(best < INFINITY)) {
    sr.axis = -1;  // no usable plane: split the range in the middle
    sr.plane = 0;
    sr.nl = n / 2;
  } else {
    sr.axis = bestc / (K - 1);
    sr.plane = 1 + bestc % (K - 1);
    sr.nl = bestnl;
  }
  return sr;
}

// ------------------------------------------------------------------ micro subtrees
// A node of at most 32 * E triangles (E = 1, 2 or 4) is finished by one warp
// in registers: lane j holds records E*j .. E*j + E-1 of the node's range (in
// the order the stable partitions kept, i.e. Morton order within the node).
// Every split of the subtree is the minimum of Eq. 2 over all splits of that
// order, evaluated from lane-local prefix/suffix unions of the records' boxes
// and one warp scan of the lane totals; ranges never move, so there is no
// partition step.
struct Box6 {
  float l0, l1, l2, h0, h1, h2;
};
__device__ __forceinline__ Box6 box_empty() { return {FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX}; }
__device__ __forceinline__ Box6 box_join(const Box6& a, const Box6& b) {
  return {fminf(a.l0, b.l0), fminf(a.l1, b.l1), fminf(a.l2, b.l2),
          fmaxf(a.h0, b.h0), fmaxf(a.h1, b.h1), fmaxf(a.h2, b.h2)};
}
__device__ __forceinline__ Box6 box_shfl_up(const Box6& a, int o) {
  return {__shfl_up_sync(0xffffffffu, a.l0, o), __shfl_up_sync(0xffffffffu, a.l1, o),
          __shfl_up_sync(0xffffffffu, a.l2, o), __shfl_up_sync(0xffffffffu, a.h0, o),
          __shfl_up_sync(0xffffffffu, a.h1, o), __shfl_up_sync(0xffffffffu, a.h2, o)};
}
__device__ __forceinline__ Box6 box_shfl_down(const Box6& a, int o) {
  return {__shfl_down_sync(0xffffffffu, a.l0, o), __shfl_down_sync(0xffffffffu, a.l1, o),
          __shfl_down_sync(0xffffffffu, a.l2, o), __shfl_down_sync(0xffffffffu, a.h0, o),
          __shfl_down_sync(0xffffffffu, a.h1, o), __shfl_down_sync(0xffffffffu, a.h2, o)};
}
__device__ __forceinline__ Box6 box_shfl(const Box6& a, int src) {
  return {__shfl_sync(0xffffffffu, a.l0, src), __shfl_sync(0xffffffffu, a.l1, src),
          __shfl_sync(0xffffffffu, a.l2, src), __shfl_sync(0xffffffffu, a.h0, src),
          __shfl_sync(0xffffffffu, a.h1, src), __shfl_sync(0xffffffffu, a.h2, src)};
}

template <int E>
__device__ void micro_build(const BuildArgs& A, const float4 (&rlo)[E], const float4 (&rhi)[E], int n,
                            int gbase, int parent, int side, int depth) {
  const int lane = threadIdx.x & 31;
  // uniform stack of pending ranges: (b, e, parent, side | depth << 1); the
  // larger child is stacked, so at most log2(32 E) + 1 entries
  int4 st[10];
  int sp = 0;
  st[sp++] = make_int4(0, n, parent, side | (depth << 1));
  int n_int = 0, n_leaf = 0, big = 0, deep = 0;
  while (sp > 0) {
    const int4 tk = st[--sp];
    const int b = tk.x, e = tk.y, par = tk.z, sd = tk.w & 1, dep = tk.w >> 1;
    // lane-local inclusive prefix / suffix of the in-range records
    Box6 pre[E], suf[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int q = E * lane + i;
      const bool in = q >= b && q < e;
      Box6 x = in ? Box6{rlo[i].x, rlo[i].y, rlo[i].z, rhi[i].x, rhi[i].y, rhi[i].z} : box_empty();
      pre[i] = i ? box_join(pre[i - 1], x) : x;
    }
#pragma unroll
    for (int i = E - 1; i >= 0; --i) {
      const int q = E * lane + i;
      const bool in = q >= b && q < e;
      Box6 x = in ? Box6{rlo[i].x, rlo[i].y, rlo[i].z, rhi[i].x, rhi[i].y, rhi[i].z} : box_empty();
      suf[i] = i < E - 1 ? box_join(suf[i + 1], x) : x;
    }
    // warp scans of the lane totals: inclusive prefix / suffix, then exclusive
    Box6 ip = pre[E - 1], is = suf[0];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Box6 u = box_shfl_up(ip, o), d = box_shfl_down(is, o);
      if (lane >= o) ip = box_join(ip, u);
      if (lane + o < 32) is = box_join(is, d);
    }
    Box6 xp = box_shfl_up(ip, 1), xs = box_shfl_down(is, 1);
    if (lane == 0) xp = box_empty();
    if (lane == 31) xs = box_empty();
    const Box6 node = box_shfl(ip, 31);
    const float3 clo = make_float3(node.l0, node.l1, node.l2), chi = make_float3(node.h0, node.h1, node.h2);
    // candidate: last left record q (b <= q < e - 1)
    float best = INFINITY;
    int bq = 1 << 20;
    Box6 bl = box_empty(), br = box_empty();
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int q = E * lane + i;
      if (q >= b && q + 1 < e) {
        const Box6 L = box_join(xp, pre[i]);
        const Box6 R = box_join(xs, i + 1 < E ? suf[i + 1 < E ? i + 1 : i] : box_empty());
        const float c = eq2_cost(make_float3(L.l0, L.l1, L.l2), make_float3(L.h0, L.h1, L.h2), q - b + 1,
                                 make_float3(R.l0, R.l1, R.l2), make_float3(R.h0, R.h1, R.h2), e - q - 1,
                                 clo, chi, A.cp);
        if (c < best) {  // increasing q within the lane: strict < keeps the lowest
          best = c;
          bq = q;
          bl = L;
          br = R;
        }
      }
    }
    float wb = best;
    int wq = bq;
    for (int o = 16; o > 0; o >>= 1) {
      const float oc = __shfl_xor_sync(0xffffffffu, wb, o);
      const int oq = __shfl_xor_sync(0xffffffffu, wq, o);
      if (oc < wb || (oc == wb && oq < wq)) {
        wb = oc;
        wq = oq;
      }
    }
    const int q = wq < (1 << 20) ? wq : (b + e) / 2 - 1;  // all costs non-finite: middle
    const int j = q + 1;                                  // first record of the right child
    const int id = gbase + q;
    const int nl = j - b, nr = e - j;
    const int rl = nl <= A.max_leaf ? leaf_ref(gbase + b, nl) : INT_MAX;
    const int rr = nr <= A.max_leaf ? leaf_ref(gbase + j, nr) : INT_MAX;
    const bool writer = wq < (1 << 20) ? (bq == wq) : (lane == 0);
    if (writer) {
      Box6 L = bl, R = br;
      if (!(wq < (1 << 20))) {  // middle split: boxes recomputed by lane 0 below
        L = box_empty();
        R = box_empty();
      }
      Node2 nd;
      nd.a_lo = make_float4(L.l0, L.l1, L.l2, __int_as_float(rl));
      nd.a_hi = make_float4(L.h0, L.h1, L.h2, __int_as_float(nl));
      nd.b_lo = make_float4(R.l0, R.l1, R.l2, __int_as_float(rr));
      nd.b_hi = make_float4(R.h0, R.h1, R.h2, __int_as_float(nr));
      A.node2[id] = nd;
      if (par < 0)
        A.ctl->root_ref = id;
      else
        *(sd == 0 ? &A.node2[par].a_lo.w : &A.node2[par].b_lo.w) = __int_as_float(id);
    }
    if (!(wq < (1 << 20))) {
      // degenerate (non-finite costs): compute the two child boxes by reduction
      Box6 L = box_empty(), R = box_empty();
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int qq = E * lane + i;
        Box6 x = Box6{rlo[i].x, rlo[i].y, rlo[i].z, rhi[i].x, rhi[i].y, rhi[i].z};
        if (qq >= b && qq < j) L = box_join(L, x);
        if (qq >= j && qq < e) R = box_join(R, x);
      }
      for (int o = 16; o > 0; o >>= 1) {
        L = box_join(L, Box6{__shfl_xor_sync(0xffffffffu, L.l0, o), __shfl_xor_sync(0xffffffffu, L.l1, o),
                             __shfl_xor_sync(0xffffffffu, L.l2, o), __shfl_xor_sync(0xffffffffu, L.h0, o),
                             __shfl_xor_sync(0xffffffffu, L.h1, o), __shfl_xor_sync(0xffffffffu, L.h2, o)});
        R = box_join(R, Box6{__shfl_xor_sync(0xffffffffu, R.l0, o), __shfl_xor_sync(0xffffffffu, R.l1, o),
                             __shfl_xor_sync(0xffffffffu, R.l2, o), __shfl_xor_sync(0xffffffffu, R.h0, o),
                             __shfl_xor_sync(0xffffffffu, R.h1, o), __shfl_xor_sync(0xffffffffu, R.h2, o)});
      }
      if (lane == 0) {
        A.node2[id].a_lo = make_float4(L.l0, L.l1, L.l2, __int_as_float(rl));
        A.node2[id].a_hi = make_float4(L.h0, L.h1, L.h2, __int_as_float(nl));
        A.node2[id].b_lo = make_float4(R.l0, R.l1, R.l2, __int_as_float(rr));
        A.node2[id].b_hi = make_float4(R.h0, R.h1, R.h2, __int_as_float(nr));
      }
    }
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
    // stack the larger internal child first so the smaller is taken next
    const int4 cl = make_int4(b, j, id, 0 | ((dep + 1) << 1));
    const int4 cr = make_int4(j, e, id, 1 | ((dep + 1) << 1));
    const bool il = rl == INT_MAX, ir = rr == INT_MAX;
    if (il && ir) {
      if (nl >= nr) {
        st[sp++] = cl;
        st[sp++] = cr;
      } else {
        st[sp++] = cr;
        st[sp++] = cl;
      }
    } else if (il) {
      st[sp++] = cl;
    } else if (ir) {
      st[sp++] = cr;
    }
  }
  if (lane == 0) {
    atomicAdd(&A.ctl->n_internal, n_int);
    atomicAdd(&A.ctl->n_leaves, n_leaf);
    atomicMax(&A.ctl->max_leaf_size, big);
    atomicMax(&A.ctl->depth2, deep);
  }
}

// ------------------------------------------------------------------ node kernel
// Every node of more than kMicro triangles is split by one CTA (Fig. 2, one
// recursion step): bin the AABB centres of its triangles into `bins` slabs
// per axis (warp-private bins, each lane on its own sub-chunk of its warp's
// segment, so neighbouring triangles -- which share bins -- do not contend),
// evaluate Eq. 2 at every bin plane with one warp per axis, then partition
// the range stably into the other record buffer (count pass, scan over the
// warps, scatter pass).  Nodes of at most kStage triangles are first staged
// in shared memory.  A CTA keeps the larger child as its next task and hands
// the other to the device queue; children of at most kMicro triangles go to
// the micro list.
constexpr int kNodeBlock = 256;
constexpr int kNodeWarps = kNodeBlock / 32;
constexpr int kStage = 2048;
constexpr int kUnrollA = 4;

struct NodeSmem {
  float4 rec[2 * kStage];
  int wbins[kNodeWarps][kBinStride];
  int bins[kBinStride];
  float scan[3][2 * kMaxBins * 7];
  Task task, cont;
  SplitResult sr;
  float ax_cost[3];
  int ax_c[3], ax_nl[3];
  int wleft[kNodeWarps];
  float acc[kNodeWarps][24];
  float fin[24];
  int have, have_cont;
};

__device__ __forceinline__ float4 ld_rec(bool staged, const float4* srec, const float4* grec, int k) {
  return staged ? srec[k] : __ldcg(grec + k);
}

__global__ void __launch_bounds__(kNodeBlock) k_nodes(BuildArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NodeSmem& S = *reinterpret_cast<NodeSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = A.K;
  if (tid == 0) S.have_cont = 0;
  __syncthreads();
  for (;;) {
    if (tid == 0) {
      S.have = 0;
      if (S.have_cont) {
        S.task = S.cont;
        S.have_cont = 0;
        S.have = 1;
      } else if (A.ctl->status == 0) {
        const int s = atomicAdd(&A.ctl->qa_head, 1);
        int seen = -1;
        for (int it = 0;; ++it) {
          if (s < A.ctl->qa_cap && *(volatile int*)&A.qa_ready[s]) {
            __threadfence();
            S.task = load_task_cg(&A.qa[s]);
            S.have = 1;
            break;
          }
          if (*(volatile int*)&A.ctl->qa_pending == 0 || *(volatile int*)&A.ctl->status != 0) break;
          const int tail = *(volatile int*)&A.ctl->qa_tail;
          if (tail != seen) {  // the queue moved: restart the no-progress budget
            seen = tail;
            it = 0;
          }
          if (it > kSpinLimit) {
            set_status(A.ctl, kStQueueTimeout, 1);
            break;
          }
          __nanosleep(128);
        }
      }
    }
    __syncthreads();
    if (!S.have) return;
    const Task t = S.task;
    const int par = t.pad & 1;
    // records of this range were written by other CTAs of this kernel: global
    // reads go through L2 (ld.global.cg), never a stale L1 line
    const float4* grec = A.rec[par] + 2 * (size_t)t.begin;
    float4* dst = A.rec[par ^ 1] + 2 * (size_t)t.begin;
    const bool staged = t.count <= kStage;
    if (staged)
      for (int k0 = tid; k0 < 2 * t.count; k0 += 4 * kNodeBlock) {
        float4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (k0 + j * kNodeBlock < 2 * t.count) v[j] = __ldcg(grec + k0 + j * kNodeBlock);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (k0 + j * kNodeBlock < 2 * t.count) S.rec[k0 + j * kNodeBlock] = v[j];
      }
    const int seg = (t.count + kNodeWarps - 1) / kNodeWarps;
    const int sb = min(warp * seg, t.count), se = min(sb + seg, t.count);
    float cmin[3], scl[3];
    for (int a = 0; a < 3; ++a) {
      cmin[a] = t.clo[a];
      scl[a] = bin_scale(t.clo[a], t.chi[a], K);
    }
    // 1. bin
    bins_zero(&S.wbins[0][0], K, kNodeWarps, tid, kNodeBlock);
    __syncthreads();
    {
      const int c = (se - sb + 31) >> 5;
      const int lb = sb + lane * c, le = min(lb + c, se);
      for (int k0 = lb; k0 < le; k0 += kUnrollA) {
        float4 lo[kUnrollA], hi[kUnrollA];
#pragma unroll
        for (int j = 0; j < kUnrollA; ++j)
          if (k0 + j < le) {
            lo[j] = ld_rec(staged, S.rec, grec, 2 * (k0 + j));
            hi[j] = ld_rec(staged, S.rec, grec, 2 * (k0 + j) + 1);
          }
#pragma unroll
        for (int j = 0; j < kUnrollA; ++j)
          if (k0 + j < le) bins_add(S.wbins[warp], K, cmin, scl, lo[j], hi[j]);
      }
    }
    __syncthreads();
    for (int q = tid; q < 3 * K * 7; q += kNodeBlock) {
      const int ent = q / 7, f = q - ent * 7;
      const int e = ent * kBinEnt + f;
      int v = S.wbins[0][e];
      for (int w = 1; w < kNodeWarps; ++w) {
        const int x = S.wbins[w][e];
        v = f == 0 ? v + x : (f <= 3 ? min(v, x) : max(v, x));
      }
      S.bins[e] = v;
    }
    __syncthreads();
    // 2. Eq. 2 at every plane, one warp per axis
    if (warp < 3) {
      float best = INFINITY;
      int bestc = INT_MAX, bestnl = 0;
      if (scl[warp] > 0.f) warp_axis_best(S.bins, K, t.count, warp, A.cp, S.scan[warp], &best, &bestc, &bestnl);
      if (lane == 0) {
        S.ax_cost[warp] = best;
        S.ax_c[warp] = bestc;
        S.ax_nl[warp] = bestnl;
      }
    }
    __syncthreads();
    if (tid == 0) {
      float best = INFINITY;
      int bestc = INT_MAX, bestnl = 0;
      for (int a = 0; a < 3; ++a)
        if (S.ax_cost[a] < best || (S.ax_cost[a] == best && S.ax_c[a] < bestc)) {
          best = S.ax_cost[a];
          bestc = S.ax_c[a];
          bestnl = S.ax_nl[a];
        }
      S.sr = make_split(K, t.count, best, bestc, bestnl);
    }
    __syncthreads();
    const SplitResult sr = S.sr;
    // 3. lefts per warp segment (kUnrollA chunks of 32 in flight)
    int nleft = 0;
    for (int k0 = sb; k0 < se; k0 += 32 * kUnrollA) {
      float4 lo[kUnrollA], hi[kUnrollA];
#pragma unroll
      for (int j = 0; j < kUnrollA; ++j) {
        const int k = k0 + 32 * j + lane;
        if (k < se) {
          lo[j] = ld_rec(staged, S.rec, grec, 2 * k);
          hi[j] = ld_rec(staged, S.rec, grec, 2 * k + 1);
        }
      }
#pragma unroll
      for (int j = 0; j < kUnrollA; ++j) {
        const int k = k0 + 32 * j + lane;
        nleft += __popc(__ballot_sync(0xffffffffu, k < se && goes_left(lo[j], hi[j], sr, k, cmin, scl, K)));
      }
    }
    if (lane == 0) S.wleft[warp] = nleft;
    __syncthreads();
    int lbase = 0;
    for (int w = 0; w < warp; ++w) lbase += S.wleft[w];
    int rbase = sb - lbase;  // rights before this segment
    // 4. stable scatter into the other buffer, accumulating child bounds
    Acc acc;
    acc.init();
    for (int k0 = sb; k0 < se; k0 += 32 * kUnrollA) {
      float4 lo[kUnrollA], hi[kUnrollA];
#pragma unroll
      for (int j = 0; j < kUnrollA; ++j) {
        const int k = k0 + 32 * j + lane;
        if (k < se) {
          lo[j] = ld_rec(staged, S.rec, grec, 2 * k);
          hi[j] = ld_rec(staged, S.rec, grec, 2 * k + 1);
        }
      }
#pragma unroll
      for (int j = 0; j < kUnrollA; ++j) {
        const int c0 = k0 + 32 * j;
        if (c0 >= se) break;
        const int k = c0 + lane;
        const bool valid = k < se;
        const bool left = valid && goes_left(lo[j], hi[j], sr, k, cmin, scl, K);
        const unsigned m = __ballot_sync(0xffffffffu, left);
        const int rank = __popc(m & ((1u << lane) - 1u));
        if (valid) {
          const int d = left ? lbase + rank : sr.nl + rbase + (lane - rank);
          dst[2 * d] = lo[j];
          dst[2 * d + 1] = hi[j];
          acc.add(left ? 0 : 1, lo[j], hi[j]);
        }
        const int tot = __popc(m);
        lbase += tot;
        rbase += min(32, se - c0) - tot;
      }
    }
    acc.warp_reduce();
    if (lane == 0)
      for (int k = 0; k < 24; ++k) S.acc[warp][k] = acc.v[k];
    __syncthreads();
    if (tid < 24) {
      const bool is_min = (tid % 12) < 3 || ((tid % 12) >= 6 && (tid % 12) < 9);
      float v = S.acc[0][tid];
      for (int w = 1; w < kNodeWarps; ++w) v = is_min ? fminf(v, S.acc[w][tid]) : fmaxf(v, S.acc[w][tid]);
      S.fin[tid] = v;
    }
    if (warp == kNodeWarps - 1 && lane == 0 && lbase != sr.nl) set_status(A.ctl, kStBadSplit, 1);
    // leaves keep their records in buffer 0
    if (par == 0) {
      const int ln = sr.nl, rn = t.count - sr.nl;
      if (ln <= A.max_leaf)
        for (int k = tid; k < 2 * ln; k += kNodeBlock) A.rec[0][2 * (size_t)t.begin + k] = __ldcg(dst + k);
      if (rn <= A.max_leaf)
        for (int k = tid; k < 2 * rn; k += kNodeBlock)
          A.rec[0][2 * ((size_t)t.begin + ln) + k] = __ldcg(dst + 2 * ln + k);
    }
    __syncthreads();
    // 5. node + children: the larger big child stays here, the rest is handed out
    if (tid == 0) {
      Task out[2];
      int nout;
      emit_node(A, t, sr.nl, S.fin, out, &nout);
      int keep = -1;
      for (int i = 0; i < nout; ++i) {
        out[i].pad = par ^ 1;
        if (out[i].count > kMicro && (keep < 0 || out[i].count > out[keep].count)) keep = i;
      }
      for (int i = 0; i < nout; ++i) {
        if (i == keep) continue;
        if (out[i].count > kMicro)
          push_a(A, out[i]);
        else
          push_b(A, out[i]);
      }
      if (keep >= 0) {
        S.cont = out[keep];
        S.have_cont = 1;
        atomicAdd(&A.ctl->qa_pending, 1);
      }
      __threadfence();
      atomicSub(&A.ctl->qa_pending, 1);
    }
    __syncthreads();
  }
}

// One warp per micro task: the subtree of a node of at most kMicro triangles.
template <int E>
__device__ __forceinline__ void micro_task(const BuildArgs& A, const Task& t) {
  const int lane = threadIdx.x & 31;
  const int par = t.pad & 1;
  float4 lo[E], hi[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int q = E * lane + i;
    lo[i] = hi[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < t.count) {
      const float4* g = A.rec[par] + 2 * ((size_t)t.begin + q);
      lo[i] = g[0];
      hi[i] = g[1];
      if (par) {  // the final record order lives in buffer 0
        A.rec[0][2 * ((size_t)t.begin + q)] = lo[i];
        A.rec[0][2 * ((size_t)t.begin + q) + 1] = hi[i];
      }
    }
  }
  micro_build<E>(A, lo, hi, t.count, t.begin, t.parent, t.side, t.depth);
}

__global__ void __launch_bounds__(256) k_micro(BuildArgs A) {
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int total = min(*(volatile int*)&A.ctl->qb_count, A.ctl->qb_cap);
  for (int ti = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ti < total; ti += nwarps) {
    const Task t = A.qb[ti];
    if (t.count <= 32)
      micro_task<1>(A, t);
    else if (t.count <= 64)
      micro_task<2>(A, t);
    else
      micro_task<4>(A, t);
  }
}

// ------------------------------------------------------------------ collapse
struct CollapseArgs {
  const Node2* node2;
  WNode* wide;
  BuildCtl* ctl;
  int4* q;
  int* ready;
  int cap;
  int n_tri;  // binary node ids are < n_tri - 1; anything else is a broken link
};

// A binary child link is usable only if it is a leaf or a valid node id.
__device__ __forceinline__ bool link_ok(int ref, int n_tri) { return ref < 0 || ref < n_tri - 1; }

__global__ void k_collapse_init(CollapseArgs C) {
  if (threadIdx.x || blockIdx.x) return;
  int r = C.ctl->root_ref;
  C.ctl->n_wide = 1;
  C.ctl->depth_wide = 1;
  C.ctl->qc_tail = 0;
  if (r < 0) {  // the whole scene is one leaf (or empty)
    WNode w;
    float inf = INFINITY;
    w.lox = w.loy = w.loz = make_float4(inf, inf, inf, inf);
    w.hix = w.hiy = w.hiz = make_float4(-inf, -inf, -inf, -inf);
    w.child = make_int4(INT_MIN, INT_MIN, INT_MIN, INT_MIN);
    if (r != INT_MIN && leaf_count(r) > 0) {
      float lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        lo[a] = iford(C.ctl->scene_lo[a]);
        hi[a] = iford(C.ctl->scene_hi[a]);
      }
      w.lox.x = lo[0];
      w.loy.x = lo[1];
      w.loz.x = lo[2];
      w.hix.x = hi[0];
      w.hiy.x = hi[1];
      w.hiz.x = hi[2];
      w.child.x = r;
    }
    w.meta = make_int4(-1, 0, 0, 0);
    C.wide[0] = w;
    return;
  }
  if (!link_ok(r, C.n_tri)) {
    set_status(C.ctl, kStBadSplit, 13);
    return;
  }
  C.q[0] = make_int4(r, 0, -1, 0);  // (binary node, -, parent wide node, slot)
  C.ctl->qc_tail = 1;
}

__device__ __forceinline__ void child_of(const Node2& n, int s, int* ref, float3* lo, float3* hi) {
  float4 l = s == 0 ? n.a_lo : n.b_lo, h = s == 0 ? n.a_hi : n.b_hi;
  *ref = __float_as_int(l.w);
  *lo = make_float3(l.x, l.y, l.z);
  *hi = make_float3(h.x, h.y, h.z);
}

// Binary tree -> 4-wide nodes, top-down, one level of the wide tree at a
// time in a single CTA.  Queue item i becomes wide node i: a wide node opens
// the internal child of largest surface area until it has 4 children; its
// internal children are appended to the queue at positions from a block
// scan, so the layout is breadth-first and the same on every run.
constexpr int kCollapseThreads = 1024;

__global__ void __launch_bounds__(kCollapseThreads) k_collapse(CollapseArgs C) {
  __shared__ int s_warp[kCollapseThreads / 32];
  __shared__ int s_tail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (C.ctl->qc_tail == 0) return;  // leaf root: done by k_collapse_init
  int lb = 0, le = 1, depth = 1;
  if (tid == 0) s_tail = 1;
  __syncthreads();
  while (lb < le) {
    for (int c0 = lb; c0 < le; c0 += kCollapseThreads) {
      const int i = c0 + tid;
      const bool valid = i < le;
      int ref[kWidth];
      float3 lo[kWidth], hi[kWidth];
      int m = 0;
      int4 item = make_int4(0, 0, 0, 0);
      if (valid) {
        item = __ldcg(&C.q[i]);
        Node2 n = C.node2[item.x];
        child_of(n, 0, &ref[0], &lo[0], &hi[0]);
        child_of(n, 1, &ref[1], &lo[1], &hi[1]);
        m = 2;
        for (int q = 0; q < 2; ++q)
          if (!link_ok(ref[q], C.n_tri)) {
            set_status(C.ctl, kStBadSplit, 11);
            ref[q] = INT_MIN;
          }
        while (m < kWidth) {
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
          Node2 g = C.node2[ref[pick]];
          child_of(g, 1, &ref[m], &lo[m], &hi[m]);
          child_of(g, 0, &ref[pick], &lo[pick], &hi[pick]);
          for (int q : {pick, m})
            if (!link_ok(ref[q], C.n_tri)) {
              set_status(C.ctl, kStBadSplit, 12);
              ref[q] = INT_MIN;
            }
          ++m;
        }
      }
      // positions of this chunk's internal children: block exclusive scan
      int cnt = 0;
      for (int q = 0; q < m; ++q) cnt += ref[q] >= 0 ? 1 : 0;
      int x = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_warp[warp] = x;
      __syncthreads();
      int base = 0, total = 0;
      for (int w = 0; w < kCollapseThreads / 32; ++w) {
        const int v = s_warp[w];
        if (w < warp) base += v;
        total += v;
      }
      const int tail0 = s_tail;
      int pos = tail0 + base + x - cnt;
      if (valid) {
        float lx[4], ly[4], lz[4], hx[4], hy[4], hz[4];
        int ch[4];
        for (int q = 0; q < kWidth; ++q) {
          if (q < m && ref[q] != INT_MIN) {
            lx[q] = lo[q].x;
            ly[q] = lo[q].y;
            lz[q] = lo[q].z;
            hx[q] = hi[q].x;
            hy[q] = hi[q].y;
            hz[q] = hi[q].z;
            if (ref[q] >= 0) {
              if (pos >= C.cap) {
                set_status(C.ctl, kStWideOverflow, 1);
                ch[q] = INT_MIN;
                continue;
              }
              C.q[pos] = make_int4(ref[q], 0, i, q);
              ch[q] = pos++;
            } else {
              ch[q] = ref[q];
            }
          } else {
            lx[q] = ly[q] = lz[q] = INFINITY;
            hx[q] = hy[q] = hz[q] = -INFINITY;
            ch[q] = INT_MIN;
          }
        }
        WNode w;
        w.lox = make_float4(lx[0], lx[1], lx[2], lx[3]);
        w.hix = make_float4(hx[0], hx[1], hx[2], hx[3]);
        w.loy = make_float4(ly[0], ly[1], ly[2], ly[3]);
        w.hiy = make_float4(hy[0], hy[1], hy[2], hy[3]);
        w.loz = make_float4(lz[0], lz[1], lz[2], lz[3]);
        w.hiz = make_float4(hz[0], hz[1], hz[2], hz[3]);
        w.child = make_int4(ch[0], ch[1], ch[2], ch[3]);
        w.meta = make_int4(item.z, item.w, 0, 0);
        C.wide[i] = w;
      }
      __syncthreads();
      if (tid == 0) s_tail = tail0 + total;
      __syncthreads();
    }
    lb = le;
    le = min(s_tail, C.cap);
    if (lb < le) ++depth;
  }
  if (tid == 0) {
    C.ctl->n_wide = le;
    C.ctl->depth_wide = depth;
    C.ctl->qc_tail = le;
  }
}

// Records in Morton order (the build's starting order).
__global__ void k_make_recs(const float4* __restrict__ plo, const float4* __restrict__ phi,
                            const int32_t* __restrict__ idx, int n, float4* __restrict__ rec) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int p = idx[k];
    rec[2 * (size_t)k] = plo[p];
    rec[2 * (size_t)k + 1] = phi[p];
  }
}

// Triangles in leaf order (the final record order carries the ids).
__global__ void k_gather(const float4* __restrict__ tri_in, const float4* __restrict__ rec, int n,
                         float4* __restrict__ tri_leaf, int32_t* __restrict__ order) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int p = __float_as_int(rec[2 * (size_t)k].w);
    order[k] = p;
    tri_leaf[3 * (size_t)k] = tri_in[3 * (size_t)p];
    tri_leaf[3 * (size_t)k + 1] = tri_in[3 * (size_t)p + 1];
    tri_leaf[3 * (size_t)k + 2] = tri_in[3 * (size_t)p + 2];
  }
}

// Elements per radix-sort block: at least one tile, about two blocks per SM.
int sort_chunk(int n, int nsm) {
  int c = (n + 2 * nsm - 1) / (2 * nsm);
  c = (c + kSortBlock - 1) / kSortBlock * kSortBlock;
  return c < 4 * kSortBlock ? 4 * kSortBlock : c;
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

}  // namespace

cudaError_t launch_build(rt_scene_s* s, const rt_build_params& p, cudaStream_t st) {
  const int n = (int)s->n_tri;
  const int nsm = sm_count();
  const int qa_cap = n + 4;  // a peeling chain can make almost every node a tier-A task
  const int qb_cap = n + 1;
  const int qc_cap = n + 1;
  cudaError_t e;
  int n_launched = 0;
  if ((e = cudaMemsetAsync(s->ctl, 0, sizeof(BuildCtl), st))) return e;
  if ((e = cudaMemsetAsync(s->qa_ready, 0, sizeof(int) * qa_cap, st))) return e;
  k_init_ctl<<<1, 32, 0, st>>>(s->ctl, qa_cap, qb_cap, qc_cap);
    ++n_launched;
  if (n > 0) {
    int g = (n + kPrepBlock - 1) / kPrepBlock;
    g = g < nsm * 8 ? g : nsm * 8;
    k_prep<<<g, kPrepBlock, 0, st>>>(s->tri_in, n, s->prim_lo, s->prim_hi, s->ctl);
    ++n_launched;
    k_morton<<<g, kPrepBlock, 0, st>>>(s->prim_lo, s->prim_hi, n, s->ctl, s->keys[0], s->idx[0]);
    ++n_launched;
    const int chunk = sort_chunk(n, nsm);
    const int nb = (n + chunk - 1) / chunk;
    for (int pass = 0; pass < 4; ++pass) {
      int src = pass & 1, dst = src ^ 1;
      k_sort_hist<<<nb, kSortBlock, 0, st>>>(s->keys[src], n, 8 * pass, s->sort_hist, nb, chunk);
    ++n_launched;
      k_sort_scan<<<1, 256, 0, st>>>(s->sort_hist, nb);
    ++n_launched;
      k_sort_scatter<<<nb, kSortBlock, 0, st>>>(s->keys[src], s->idx[src], s->keys[dst], s->idx[dst],
                                                n, 8 * pass, s->sort_hist, nb, chunk);
    ++n_launched;
    }
  }
  if (n > 0) {
    int g = (n + 255) / 256;
    g = g < nsm * 8 ? g : nsm * 8;
    k_make_recs<<<g, 256, 0, st>>>(s->prim_lo, s->prim_hi, s->idx[0], n, s->rec[0]);
    ++n_launched;
  }
  k_root<<<1, 32, 0, st>>>(s->ctl, s->qa, s->qa_ready, s->qb, n, p.max_leaf, s->node2);
  ++n_launched;
  BuildArgs A;
  A.rec[0] = s->rec[0];
  A.rec[1] = s->rec[1];
  A.node2 = s->node2;
  A.ctl = s->ctl;
  A.qa = s->qa;
  A.qa_ready = s->qa_ready;
  A.qb = s->qb;
  A.K = p.bins;
  A.max_leaf = p.max_leaf;
  A.cp = CostP{p.alpha, p.t_i, p.t_trav, p.source[0], p.source[1], p.source[2], p.dist_norm};
  if (n > kMicro) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_nodes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(NodeSmem));
      attr = true;
    }
    k_nodes<<<nsm, kNodeBlock, sizeof(NodeSmem), st>>>(A);
    ++n_launched;
  }
  if (n > p.max_leaf) {
    k_micro<<<2 * nsm, 256, 0, st>>>(A);
    ++n_launched;
  }
  CollapseArgs C{s->node2, s->wide, s->ctl, s->qc, s->qc_ready, qc_cap, n};
  k_collapse_init<<<1, 32, 0, st>>>(C);
  ++n_launched;
  if (n > p.max_leaf) {
    k_collapse<<<1, kCollapseThreads, 0, st>>>(C);
    ++n_launched;
  }
  if (n > 0) {
    int g = (n + 255) / 256;
    g = g < nsm * 8 ? g : nsm * 8;
    k_gather<<<g, 256, 0, st>>>(s->tri_in, s->rec[0], n, s->tri_leaf, s->idx[0]);
    ++n_launched;
  }
  count_launches(n_launched);
  return cudaGetLastError();
}

}  // namespace rt
