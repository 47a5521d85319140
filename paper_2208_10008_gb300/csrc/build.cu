// BVH construction on the device (Sec. II.B-C of arXiv 2208.10008).
//
// Pipeline, all asynchronous on one stream:
//   k_prep        per-triangle AABB (Eq. 3 boxes) + scene / centroid bounds
//   k_morton      30-bit Morton key of each AABB centre (locality presort)
//   radix sort    4 stable LSD passes (8-bit digits): hist, scan, scatter
//   k_root        the root task (Fig. 2: "calculate the bounding volume that
//                 contains all triangular facets")
//   k_tier_a      one CTA per node of more than kTierASmall triangles, fed by
//                 a device work queue: bin AABB centres into `bins` slabs per
//                 axis, evaluate Eq. 2 at every bin plane, take the minimum
//                 (ties: lowest axis, lowest plane), stable-partition the
//                 node's index range, emit children (Fig. 2 recursion)
//   k_tier_b      one warp per remaining subtree, depth first
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
constexpr int kSortChunk = 256 * 32;     // elements per block per pass
constexpr int kTierABlock = 256;
constexpr int kTierAWarps = kTierABlock / 32;
constexpr int kTierBBlock = 256;
constexpr int kTierBWarps = kTierBBlock / 32;
constexpr int kCollapseBlock = 128;

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
                                                          int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int b = blockIdx.x * kSortChunk, e = min(n, b + kSortChunk);
  for (int i = b + threadIdx.x; i < e; i += kSortBlock) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m counters in one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* hist, int m) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < m; base += 1024) {
    int i = base + threadIdx.x;
    uint32_t v = i < m ? hist[i] : 0u;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) warp_sums[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t w = warp_sums[threadIdx.x];
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (threadIdx.x >= o) w += y;
      }
      warp_sums[threadIdx.x] = w;
    }
    __syncthreads();
    uint32_t wofs = (threadIdx.x >> 5) ? warp_sums[(threadIdx.x >> 5) - 1] : 0u;
    if (i < m) hist[i] = carry + wofs + x - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += wofs + x;
    __syncthreads();
  }
}

// Stable scatter: tiles of 256 elements, warp-major; ranks from match_any.
__global__ void __launch_bounds__(kSortBlock) k_sort_scatter(
    const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    int32_t* __restrict__ vout, int n, int shift, const uint32_t* __restrict__ hist, int nblocks) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wh[kSortBlock / 32][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  base[threadIdx.x] = hist[threadIdx.x * nblocks + blockIdx.x];
  int b = blockIdx.x * kSortChunk, e = min(n, b + kSortChunk);
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
  if (n > kTierASmall) {
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

constexpr int kBinStride = 3 * kMaxBins * 8;  // ints per bin set

// Reset `nsets` bin sets laid out kBinStride ints apart (first 3*K*8 used).
__device__ __forceinline__ void bins_zero(int* bins, int K, int nsets, int tid, int nthreads) {
  const int per = 3 * K * 8;
  for (int k = tid; k < per * nsets; k += nthreads) {
    int w = k / per, e = k - w * per;
    int f = e & 7;
    bins[w * kBinStride + e] = f == 0 ? 0 : (f <= 3 ? ford(FLT_MAX) : (f <= 6 ? ford(-FLT_MAX) : 0));
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
    int* bb = bins + (a * K + bin_of(c[a], cmin[a], scl[a], K)) * 8;
    atomicAdd(bb, 1);
    atomicMin(bb + 1, ford(lo.x));
    atomicMin(bb + 2, ford(lo.y));
    atomicMin(bb + 3, ford(lo.z));
    atomicMax(bb + 4, ford(hi.x));
    atomicMax(bb + 5, ford(hi.y));
    atomicMax(bb + 6, ford(hi.z));
  }
}

// Cost of candidate c (axis c / (K-1), plane 1 + c % (K-1)); +inf when invalid.
__device__ float eval_candidate(const int* bins, int K, int c, int n, const float scl[3],
                                const CostP& cp, float3 nlo, float3 nhi) {
  int a = c / (K - 1), p = 1 + c % (K - 1);
  if (scl[a] <= 0.f) return INFINITY;
  const int* ba = bins + a * K * 8;
  int nl = 0;
  float3 llo = make_float3(FLT_MAX, FLT_MAX, FLT_MAX), lhi = make_float3(-FLT_MAX, -FLT_MAX, -FLT_MAX);
  float3 rlo = llo, rhi = lhi;
  for (int b = 0; b < K; ++b) {
    const int* e = ba + b * 8;
    int cnt = e[0];
    if (cnt == 0) continue;
    float3 lo = make_float3(iford(e[1]), iford(e[2]), iford(e[3]));
    float3 hi = make_float3(iford(e[4]), iford(e[5]), iford(e[6]));
    if (b < p) {
      nl += cnt;
      llo = make_float3(fminf(llo.x, lo.x), fminf(llo.y, lo.y), fminf(llo.z, lo.z));
      lhi = make_float3(fmaxf(lhi.x, hi.x), fmaxf(lhi.y, hi.y), fmaxf(lhi.z, hi.z));
    } else {
      rlo = make_float3(fminf(rlo.x, lo.x), fminf(rlo.y, lo.y), fminf(rlo.z, lo.z));
      rhi = make_float3(fmaxf(rhi.x, hi.x), fmaxf(rhi.y, hi.y), fmaxf(rhi.z, hi.z));
    }
  }
  if (nl == 0 || nl == n) return INFINITY;
  return eq2_cost(llo, lhi, nl, rlo, rhi, n - nl, nlo, nhi, cp);
}

__device__ __forceinline__ int left_count(const int* bins, int K, int axis, int plane) {
  int nl = 0;
  for (int b = 0; b < plane; ++b) nl += bins[(axis * K + b) * 8];
  return nl;
}

// Node box = union of all bins of any active axis (every triangle is in
// exactly one bin per active axis).
__device__ void node_box(const int* bins, int K, const float scl[3], float3* lo, float3* hi) {
  *lo = make_float3(FLT_MAX, FLT_MAX, FLT_MAX);
  *hi = make_float3(-FLT_MAX, -FLT_MAX, -FLT_MAX);
  int a = scl[0] > 0.f ? 0 : (scl[1] > 0.f ? 1 : 2);
  for (int b = 0; b < K; ++b) {
    const int* e = bins + (a * K + b) * 8;
    if (e[0] == 0) continue;
    *lo = make_float3(fminf(lo->x, iford(e[1])), fminf(lo->y, iford(e[2])), fminf(lo->z, iford(e[3])));
    *hi = make_float3(fmaxf(hi->x, iford(e[4])), fmaxf(hi->y, iford(e[5])), fmaxf(hi->z, iford(e[6])));
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
  __device__ void warp_reduce() {
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      bool is_min = (k % 12) < 3 || ((k % 12) >= 6 && (k % 12) < 9);
      for (int o = 16; o > 0; o >>= 1) {
        float y = __shfl_xor_sync(0xffffffffu, v[k], o);
        v[k] = is_min ? fminf(v[k], y) : fmaxf(v[k], y);
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
  float4* rec;       // [2T] primitive records in build order: (lo.xyz, id) (hi.xyz, 0)
  float4* rec_tmp;   // [2T] partition scratch
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

// Best candidate of a bin set: (cost, candidate) minimum over the calling
// threads' share, reduced within the warp (ties: lowest candidate index, i.e.
// lowest axis, then lowest plane).
__device__ __forceinline__ void warp_best(const int* bins, int K, int n, const float scl[3],
                                          const CostP& cp, float3 nlo, float3 nhi, int first,
                                          int stride, float* best, int* bestc) {
  *best = INFINITY;
  *bestc = INT_MAX;
  for (int c = first; c < 3 * (K - 1); c += stride) {
    float v = eval_candidate(bins, K, c, n, scl, cp, nlo, nhi);
    if (v < *best) {
      *best = v;
      *bestc = c;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    float ov = __shfl_xor_sync(0xffffffffu, *best, o);
    int oc = __shfl_xor_sync(0xffffffffu, *bestc, o);
    if (ov < *best || (ov == *best && oc < *bestc)) {
      *best = ov;
      *bestc = oc;
    }
  }
}

__device__ __forceinline__ SplitResult make_split(const int* bins, int K, int n, float best, int bestc) {
  SplitResult sr;
  if (bestc == INT_MAX || !(best < INFINITY)) {
    sr.axis = -1;  // no usable plane: split the range in the middle
    sr.plane = 0;
    sr.nl = n / 2;
  } else {
    sr.axis = bestc / (K - 1);
    sr.plane = 1 + bestc % (K - 1);
    sr.nl = left_count(bins, K, sr.axis, sr.plane);
  }
  return sr;
}

// ------------------------------------------------------------------ tier A
// One CTA per node of more than kTierASmall triangles.  Records are read
// coalesced, kUnrollA per thread in flight.
constexpr int kUnrollA = 4;

__global__ void __launch_bounds__(kTierABlock) k_tier_a(BuildArgs A) {
  __shared__ int wbins[kTierAWarps][kBinStride];
  __shared__ int bins[kBinStride];
  __shared__ Task task;
  __shared__ int s_slot;
  __shared__ float s_cost[kTierAWarps];
  __shared__ int s_cand[kTierAWarps];
  __shared__ SplitResult s_sr;
  __shared__ int s_wcount[kTierAWarps];
  __shared__ float s_acc[kTierAWarps][24];
  __shared__ float s_fin[24];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = A.K;
  for (;;) {
    if (tid == 0) {
      int slot = -1;
      if (A.ctl->status == 0) {
        int s = atomicAdd(&A.ctl->qa_head, 1);
        int seen = -1;
        for (int it = 0;; ++it) {
          if (s < A.ctl->qa_cap && *(volatile int*)&A.qa_ready[s]) {
            __threadfence();
            slot = s;
            break;
          }
          const int pend = *(volatile int*)&A.ctl->qa_pending;
          if (pend == 0 || *(volatile int*)&A.ctl->status != 0) break;
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
      s_slot = slot;
      if (slot >= 0) task = load_task_cg(&A.qa[slot]);
    }
    __syncthreads();
    if (s_slot < 0) return;
    const Task t = task;
    // records of this range were written by other CTAs of this kernel: every
    // read below goes through L2 (ld.global.cg), never a stale L1 line
    const float4* rec = A.rec + 2 * (size_t)t.begin;
    float4* tmp = A.rec_tmp + 2 * (size_t)t.begin;
    float cmin[3], scl[3];
    for (int a = 0; a < 3; ++a) {
      cmin[a] = t.clo[a];
      scl[a] = bin_scale(t.clo[a], t.chi[a], K);
    }
    // 1. bin (warp-private bins, then merge)
    bins_zero(&wbins[0][0], K, kTierAWarps, tid, kTierABlock);
    __syncthreads();
    for (int k0 = 0; k0 < t.count; k0 += kUnrollA * kTierABlock) {
      float4 lo[kUnrollA], hi[kUnrollA];
#pragma unroll
      for (int j = 0; j < kUnrollA; ++j) {
        int k = k0 + j * kTierABlock + tid;
        if (k < t.count) {
          lo[j] = __ldcg(rec + 2 * k);
          hi[j] = __ldcg(rec + 2 * k + 1);
        }
      }
#pragma unroll
      for (int j = 0; j < kUnrollA; ++j)
        if (k0 + j * kTierABlock + tid < t.count) bins_add(wbins[warp], K, cmin, scl, lo[j], hi[j]);
    }
    __syncthreads();
    for (int e = tid; e < 3 * K * 8; e += kTierABlock) {
      int f = e & 7;
      int v = wbins[0][e];
      for (int w = 1; w < kTierAWarps; ++w) {
        int x = wbins[w][e];
        v = f == 0 ? v + x : (f <= 3 ? min(v, x) : (f <= 6 ? max(v, x) : 0));
      }
      bins[e] = v;
    }
    __syncthreads();
    // 2. Eq. 2 at every plane
    float3 nlo, nhi;
    node_box(bins, K, scl, &nlo, &nhi);
    float best;
    int bestc;
    warp_best(bins, K, t.count, scl, A.cp, nlo, nhi, tid, kTierABlock, &best, &bestc);
    if (lane == 0) {
      s_cost[warp] = best;
      s_cand[warp] = bestc;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < kTierAWarps; ++w)
        if (s_cost[w] < best || (s_cost[w] == best && s_cand[w] < bestc)) {
          best = s_cost[w];
          bestc = s_cand[w];
        }
      s_sr = make_split(bins, K, t.count, best, bestc);
    }
    __syncthreads();
    const SplitResult sr = s_sr;
    // 3. stable partition into tmp, accumulating child bounds
    Acc acc;
    acc.init();
    int lbase = 0, rbase = 0;
    for (int t0 = 0; t0 < t.count; t0 += kTierABlock) {
      int k = t0 + tid;
      bool valid = k < t.count;
      float4 lo = valid ? __ldcg(rec + 2 * k) : make_float4(0, 0, 0, 0);
      float4 hi = valid ? __ldcg(rec + 2 * k + 1) : make_float4(0, 0, 0, 0);
      bool left = valid && goes_left(lo, hi, sr, k, cmin, scl, K);
      unsigned m = __ballot_sync(0xffffffffu, left);
      int rank = __popc(m & ((1u << lane) - 1u));
      if (lane == 0) s_wcount[warp] = __popc(m);
      __syncthreads();
      int woff = 0, tot = 0;
      for (int w = 0; w < kTierAWarps; ++w) {
        int c = s_wcount[w];
        if (w < warp) woff += c;
        tot += c;
      }
      if (valid) {
        int lpos = woff + rank;  // lefts before k in this tile
        int dst = left ? lbase + lpos : sr.nl + rbase + (k - t0 - lpos);
        tmp[2 * dst] = lo;
        tmp[2 * dst + 1] = hi;
        acc.add(left ? 0 : 1, lo, hi);
      }
      lbase += tot;
      rbase += min(kTierABlock, t.count - t0) - tot;
      __syncthreads();
    }
    acc.warp_reduce();
    if (lane == 0)
      for (int k = 0; k < 24; ++k) s_acc[warp][k] = acc.v[k];
    __syncthreads();
    if (tid < 24) {
      bool is_min = (tid % 12) < 3 || ((tid % 12) >= 6 && (tid % 12) < 9);
      float v = s_acc[0][tid];
      for (int w = 1; w < kTierAWarps; ++w) v = is_min ? fminf(v, s_acc[w][tid]) : fmaxf(v, s_acc[w][tid]);
      s_fin[tid] = v;
    }
    if (tid == 0 && lbase != sr.nl) set_status(A.ctl, kStBadSplit, 1);
    {
      float4* __restrict__ dst = A.rec + 2 * (size_t)t.begin;
      for (int k = tid; k < 2 * t.count; k += kTierABlock) dst[k] = __ldcg(tmp + k);
    }
    __syncthreads();
    // 4. node + children
    if (tid == 0) {
      Task out[2];
      int nout;
      emit_node(A, t, sr.nl, s_fin, out, &nout);
      for (int i = 0; i < nout; ++i) {
        if (out[i].count > kTierASmall)
          push_a(A, out[i]);
        else
          push_b(A, out[i]);
      }
      __threadfence();
      atomicSub(&A.ctl->qa_pending, 1);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ tier B
// One CTA per subtree of at most kTierASmall triangles.  The subtree's
// records are copied to shared memory once; its nodes are then split by the
// CTA's warps in parallel, each warp taking whole nodes from a shared stack
// (and a short private stack when the shared one is full).
constexpr int kTierBShared = 128;  // shared task stack entries
constexpr int kTierBPriv = 16;     // private entries per warp (>= log2 kTierASmall + 2)

struct TierBSmem {
  float4 rec[2 * kTierASmall];
  uint16_t idx[2][kTierASmall];
  int bins[kTierBWarps][kBinStride];
  Task shared_stack[kTierBShared];
  Task priv[kTierBWarps][kTierBPriv];
  Task cur[kTierBWarps];
  int sp, pending, lock, pad;
};

// Critical sections are a few instructions long; the bound only guards
// against a logic error turning into a hang.
__device__ __forceinline__ bool smem_lock(int* l) {
  for (int it = 0; atomicCAS(l, 0, 1) != 0; ++it) {
    if (it > kSpinLimit) return false;
    __nanosleep(32);
  }
  __threadfence_block();
  return true;
}
__device__ __forceinline__ void smem_unlock(int* l) {
  __threadfence_block();
  atomicExch(l, 0);
}

__global__ void __launch_bounds__(kTierBBlock) k_tier_b(BuildArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TierBSmem& S = *reinterpret_cast<TierBSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = A.K;
  int* bins = S.bins[warp];
  const int total = min(*(volatile int*)&A.ctl->qb_count, A.ctl->qb_cap);
  for (int ti = blockIdx.x; ti < total; ti += gridDim.x) {
    const Task root = A.qb[ti];
    const int gb = root.begin, n = root.count;
    for (int k = tid; k < 2 * n; k += kTierBBlock) S.rec[k] = __ldcg(A.rec + 2 * (size_t)gb + k);
    for (int k = tid; k < n; k += kTierBBlock) S.idx[0][k] = (uint16_t)k;
    if (tid == 0) {
      Task r = root;
      r.begin = 0;
      S.shared_stack[0] = r;
      S.sp = 1;
      S.pending = 1;
      S.lock = 0;
    }
    __syncthreads();
    int psp = 0;  // private stack depth (uniform in the warp)
    for (int spin = 0;;) {
      // lane 0 alone looks at the shared state; the warp follows its decision
      int got = 0, done = 0;
      if (lane == 0) {
        if (psp > 0) {
          S.cur[warp] = S.priv[warp][psp - 1];
          got = 1;
        } else {
          if (smem_lock(&S.lock)) {
            if (S.sp > 0) {
              S.cur[warp] = S.shared_stack[--S.sp];
              got = 1;
            }
            smem_unlock(&S.lock);
          } else {
            set_status(A.ctl, kStQueueTimeout, 4);
            done = 1;
          }
        }
        if (!got && *(volatile int*)&S.pending == 0) done = 1;
      }
      got = __shfl_sync(0xffffffffu, got, 0);
      done = __shfl_sync(0xffffffffu, done, 0);
      if (got && psp > 0) --psp;
      if (!got) {
        if (done) break;
        if (++spin > kSpinLimit) {
          set_status(A.ctl, kStQueueTimeout, 3);
          break;
        }
        __nanosleep(64);
        continue;
      }
      spin = 0;
      __syncwarp();
      const Task t = S.cur[warp];
      float cmin[3], scl[3];
      for (int a = 0; a < 3; ++a) {
        cmin[a] = t.clo[a];
        scl[a] = bin_scale(t.clo[a], t.chi[a], K);
      }
      bins_zero(bins, K, 1, lane, 32);
      __syncwarp();
      for (int k = lane; k < t.count; k += 32) {
        const int li = S.idx[0][t.begin + k];
        bins_add(bins, K, cmin, scl, S.rec[2 * li], S.rec[2 * li + 1]);
      }
      __syncwarp();
      float3 nlo, nhi;
      node_box(bins, K, scl, &nlo, &nhi);
      float best;
      int bestc;
      warp_best(bins, K, t.count, scl, A.cp, nlo, nhi, lane, 32, &best, &bestc);
      const SplitResult sr = make_split(bins, K, t.count, best, bestc);
      Acc acc;
      acc.init();
      int lbase = 0, rbase = 0;
      for (int t0 = 0; t0 < t.count; t0 += 32) {
        const int k = t0 + lane;
        const bool valid = k < t.count;
        const int li = valid ? S.idx[0][t.begin + k] : 0;
        const float4 lo = S.rec[2 * li], hi = S.rec[2 * li + 1];
        const bool left = valid && goes_left(lo, hi, sr, k, cmin, scl, K);
        const unsigned m = __ballot_sync(0xffffffffu, left);
        const int rank = __popc(m & ((1u << lane) - 1u));
        if (valid) {
          const int dst = left ? lbase + rank : sr.nl + rbase + (lane - rank);
          S.idx[1][t.begin + dst] = (uint16_t)li;
          acc.add(left ? 0 : 1, lo, hi);
        }
        const int tot = __popc(m);
        lbase += tot;
        rbase += min(32, t.count - t0) - tot;
      }
      acc.warp_reduce();
      if (lane == 0 && lbase != sr.nl) set_status(A.ctl, kStBadSplit, 2);
      __syncwarp();
      for (int k = lane; k < t.count; k += 32) S.idx[0][t.begin + k] = S.idx[1][t.begin + k];
      __syncwarp();
      if (lane == 0) {
        Task g = t;
        g.begin = gb + t.begin;
        Task out[2];
        int nout = 0;
        emit_node(A, g, sr.nl, acc.v, out, &nout);
        if (nout) atomicAdd(&S.pending, nout);
        // larger child to the shared stack (work for idle warps), smaller
        // child kept by this warp; a full shared stack keeps both here
        int order[2] = {0, 1};
        if (nout == 2 && out[0].count < out[1].count) {
          order[0] = 1;
          order[1] = 0;
        }
        for (int q = 0; q < nout; ++q) {
          Task c = out[order[q]];
          c.begin -= gb;
          bool shared = false;
          if (q == 0 && nout == 2) {
            if (smem_lock(&S.lock)) {
              if (S.sp < kTierBShared) {
                S.shared_stack[S.sp++] = c;
                shared = true;
              }
              smem_unlock(&S.lock);
            }
          }
          if (!shared) {
            if (psp < kTierBPriv) {
              S.priv[warp][psp++] = c;
            } else {
              set_status(A.ctl, kStQueueOverflow, 4);
              atomicSub(&S.pending, 1);
            }
          }
        }
        __threadfence_block();
        atomicSub(&S.pending, 1);
      }
      psp = __shfl_sync(0xffffffffu, psp, 0);
      __syncwarp();
    }
    __syncthreads();
    for (int k = tid; k < n; k += kTierBBlock) {
      const int li = S.idx[0][k];
      A.rec[2 * ((size_t)gb + k)] = S.rec[2 * li];
      A.rec[2 * ((size_t)gb + k) + 1] = S.rec[2 * li + 1];
    }
    __syncthreads();
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
  C.q[0] = make_int4(r, 0, -1, 0 | (1 << 4));
  C.ctl->qc_tail = 1;
  C.ctl->qc_pending = 1;
  __threadfence();
  C.ready[0] = 1;
}

__device__ __forceinline__ void child_of(const Node2& n, int s, int* ref, float3* lo, float3* hi) {
  float4 l = s == 0 ? n.a_lo : n.b_lo, h = s == 0 ? n.a_hi : n.b_hi;
  *ref = __float_as_int(l.w);
  *lo = make_float3(l.x, l.y, l.z);
  *hi = make_float3(h.x, h.y, h.z);
}

__global__ void __launch_bounds__(kCollapseBlock) k_collapse(CollapseArgs C) {
  for (;;) {
    int slot = -1;
    if (*(volatile int*)&C.ctl->status != 0) return;
    int s = atomicAdd(&C.ctl->qc_head, 1);
    int seen = -1;
    for (int it = 0;; ++it) {
      if (s < C.cap && *(volatile int*)&C.ready[s]) {
        __threadfence();
        slot = s;
        break;
      }
      if (*(volatile int*)&C.ctl->qc_pending == 0 || *(volatile int*)&C.ctl->status != 0) break;
      const int tail = *(volatile int*)&C.ctl->qc_tail;
      if (tail != seen) {
        seen = tail;
        it = 0;
      }
      if (it > kSpinLimit) {
        set_status(C.ctl, kStQueueTimeout, 2);
        break;
      }
      __nanosleep(256);
    }
    if (slot < 0) return;
    int4 item = __ldcg(&C.q[slot]);
    const int wid = item.y, depth = item.w >> 4;
    // greedy expansion: open the internal child with the largest surface area
    int ref[kWidth];
    float3 lo[kWidth], hi[kWidth];
    int m = 2;
    if (!link_ok(item.x, C.n_tri) || item.x < 0) {
      set_status(C.ctl, kStBadSplit, 10);
      ref[0] = ref[1] = INT_MIN;
      lo[0] = lo[1] = make_float3(INFINITY, INFINITY, INFINITY);
      hi[0] = hi[1] = make_float3(-INFINITY, -INFINITY, -INFINITY);
    } else {
      Node2 n = C.node2[item.x];
      child_of(n, 0, &ref[0], &lo[0], &hi[0]);
      child_of(n, 1, &ref[1], &lo[1], &hi[1]);
    }
    for (int i = 0; i < 2; ++i)
      if (!link_ok(ref[i], C.n_tri)) {
        set_status(C.ctl, kStBadSplit, 11);
        ref[i] = INT_MIN;
      }
    while (m < kWidth) {
      int pick = -1;
      float best = -1.f;
      for (int i = 0; i < m; ++i)
        if (ref[i] >= 0) {
          float a = area(lo[i], hi[i]);
          if (a > best) {
            best = a;
            pick = i;
          }
        }
      if (pick < 0) break;
      Node2 n = C.node2[ref[pick]];
      child_of(n, 1, &ref[m], &lo[m], &hi[m]);
      child_of(n, 0, &ref[pick], &lo[pick], &hi[pick]);
      for (int i : {pick, m})
        if (!link_ok(ref[i], C.n_tri)) {
          set_status(C.ctl, kStBadSplit, 12);
          ref[i] = INT_MIN;
        }
      ++m;
    }
    WNode w;
    float lx[4], ly[4], lz[4], hx[4], hy[4], hz[4];
    int ch[4];
    for (int i = 0; i < kWidth; ++i) {
      if (i < m) {
        lx[i] = lo[i].x;
        ly[i] = lo[i].y;
        lz[i] = lo[i].z;
        hx[i] = hi[i].x;
        hy[i] = hi[i].y;
        hz[i] = hi[i].z;
        if (ref[i] == INT_MIN) {
          lx[i] = ly[i] = lz[i] = INFINITY;
          hx[i] = hy[i] = hz[i] = -INFINITY;
          ch[i] = INT_MIN;
        } else if (ref[i] >= 0) {
          int c = atomicAdd(&C.ctl->n_wide, 1);
          if (c >= C.cap) {
            set_status(C.ctl, kStWideOverflow, 1);
            ch[i] = INT_MIN;
            continue;
          }
          ch[i] = c;
          int qs = atomicAdd(&C.ctl->qc_tail, 1);
          atomicAdd(&C.ctl->qc_pending, 1);
          C.q[qs] = make_int4(ref[i], c, wid, i | ((depth + 1) << 4));
          __threadfence();
          atomicExch(&C.ready[qs], 1);
        } else {
          ch[i] = ref[i];
        }
      } else {
        lx[i] = ly[i] = lz[i] = INFINITY;
        hx[i] = hy[i] = hz[i] = -INFINITY;
        ch[i] = INT_MIN;
      }
    }
    w.lox = make_float4(lx[0], lx[1], lx[2], lx[3]);
    w.hix = make_float4(hx[0], hx[1], hx[2], hx[3]);
    w.loy = make_float4(ly[0], ly[1], ly[2], ly[3]);
    w.hiy = make_float4(hy[0], hy[1], hy[2], hy[3]);
    w.loz = make_float4(lz[0], lz[1], lz[2], lz[3]);
    w.hiz = make_float4(hz[0], hz[1], hz[2], hz[3]);
    w.child = make_int4(ch[0], ch[1], ch[2], ch[3]);
    w.meta = make_int4(item.z, item.w & 15, 0, 0);
    C.wide[wid] = w;
    atomicMax(&C.ctl->depth_wide, depth);
    __threadfence();
    atomicSub(&C.ctl->qc_pending, 1);
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
  if ((e = cudaMemsetAsync(s->qc_ready, 0, sizeof(int) * qc_cap, st))) return e;
  k_init_ctl<<<1, 32, 0, st>>>(s->ctl, qa_cap, qb_cap, qc_cap);
    ++n_launched;
  if (n > 0) {
    int g = (n + kPrepBlock - 1) / kPrepBlock;
    g = g < nsm * 8 ? g : nsm * 8;
    k_prep<<<g, kPrepBlock, 0, st>>>(s->tri_in, n, s->prim_lo, s->prim_hi, s->ctl);
    ++n_launched;
    k_morton<<<g, kPrepBlock, 0, st>>>(s->prim_lo, s->prim_hi, n, s->ctl, s->keys[0], s->idx[0]);
    ++n_launched;
    const int nb = (n + kSortChunk - 1) / kSortChunk;
    for (int pass = 0; pass < 4; ++pass) {
      int src = pass & 1, dst = src ^ 1;
      k_sort_hist<<<nb, kSortBlock, 0, st>>>(s->keys[src], n, 8 * pass, s->sort_hist, nb);
    ++n_launched;
      k_sort_scan<<<1, 1024, 0, st>>>(s->sort_hist, 256 * nb);
    ++n_launched;
      k_sort_scatter<<<nb, kSortBlock, 0, st>>>(s->keys[src], s->idx[src], s->keys[dst], s->idx[dst],
                                                n, 8 * pass, s->sort_hist, nb);
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
  A.rec = s->rec[0];
  A.rec_tmp = s->rec[1];
  A.node2 = s->node2;
  A.ctl = s->ctl;
  A.qa = s->qa;
  A.qa_ready = s->qa_ready;
  A.qb = s->qb;
  A.K = p.bins;
  A.max_leaf = p.max_leaf;
  A.cp = CostP{p.alpha, p.t_i, p.t_trav, p.source[0], p.source[1], p.source[2], p.dist_norm};
  if (n > kTierASmall) {
    k_tier_a<<<nsm, kTierABlock, 0, st>>>(A);
    ++n_launched;
  }
  if (n > p.max_leaf) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_tier_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TierBSmem));
      attr = true;
    }
    k_tier_b<<<nsm * 2, kTierBBlock, sizeof(TierBSmem), st>>>(A);
    ++n_launched;
  }
  CollapseArgs C{s->node2, s->wide, s->ctl, s->qc, s->qc_ready, qc_cap, n};
  k_collapse_init<<<1, 32, 0, st>>>(C);
  ++n_launched;
  if (n > p.max_leaf) {
    k_collapse<<<nsm * 2, kCollapseBlock, 0, st>>>(C);
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
