// Receiving-sphere reception (Sec. III.C, Eq. 4 of arXiv 2208.10008).
//
// A path segment t in [tmin, tend) of ray (o, d) receives at point p when the
// foot of the perpendicular from p lies on the segment and p is within the
// receiving sphere's radius r = l delta / sqrt(3) of the ray, l being the
// path length from the source (range0 - tmax + t*: every bounce leaves the
// remaining range in tmax).
//
// Receivers sit in a uniform grid, each entered into every cell its largest
// sphere (radius r_max, widened by a small margin) overlaps, so a segment
// only has to look at the cells it passes through: the foot of a received
// receiver lies on the segment within r_max of it.  One thread per ray
// clips its segment to the grid box and steps from cell to cell
// (Amanatides-Woo); a receiver seen in several cells is reported once (a
// short list per ray).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <vector>

#include "rt_internal.cuh"

namespace rt {
int set_error(int code, const char* msg);  // records the message for rt_last_error
}

struct rt_rxset_s {
  float lo[3] = {0.f, 0.f, 0.f};
  float h = 1.f;
  int dims[3] = {1, 1, 1};
  int m = 0;
  float r_max = 0.f;
  int* cell_start = nullptr;  // [cells + 1]
  int* items = nullptr;       // receiver index per entry
  float4* pos = nullptr;      // [m] (x, y, z, 0)
};

namespace {

constexpr int kRecvBlock = 256;
constexpr int kRecvSeen = 16;  // receivers a ray remembers to report each once

struct RecvArgs {
  const float4* rays;
  const float4* hits;
  int n;
  const int* n_dev;
  float3 lo;
  float h, inv_h;
  int nx, ny, nz;
  const int* cell_start;
  const int* items;
  const float4* pos;
  float k;  // delta / sqrt(3)
  const float* delta_ray;  // nullable: per-ray delta
  float k_cap;             // largest k the set supports
  float range0;
  int max_records;
  int4* out;
  int* count;
  unsigned long long* stats;  // nullable: cells visited, entries tested
};

__device__ __forceinline__ bool finite3(float a, float b, float c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

template <bool kStats>
__global__ void __launch_bounds__(kRecvBlock) k_receive(RecvArgs A) {
  const int i = blockIdx.x * kRecvBlock + threadIdx.x;
  const int n = A.n_dev ? min(A.n, __ldg(A.n_dev)) : A.n;
  if (i >= n) return;
  const float4 ra = __ldg(A.rays + 2 * i), rb = __ldg(A.rays + 2 * i + 1);
  const float ht = __ldg(&A.hits[i].x);
  const float tmin = ra.w, tmax = rb.w;
  const float tend = ht < tmax ? ht : tmax;
  if (!finite3(ra.x, ra.y, ra.z) || !finite3(rb.x, rb.y, rb.z) || !isfinite(tmin) || !isfinite(tmax) ||
      !(tend > tmin))
    return;
  const float ox = ra.x, oy = ra.y, oz = ra.z, dx = rb.x, dy = rb.y, dz = rb.z;
  const float dd = dx * dx + dy * dy + dz * dz;
  if (!(dd > 0.f)) return;
  const float inv_dd = 1.f / dd;
  const float lprev = A.range0 - tmax;
  const float kr = A.delta_ray ? fminf(__ldg(A.delta_ray + i) * 0.57735026918962576f, A.k_cap) : A.k;
  // clip [tmin, tend] to the grid box
  const float hx = A.lo.x + A.nx * A.h, hy = A.lo.y + A.ny * A.h, hz = A.lo.z + A.nz * A.h;
  float ta = tmin, tb = tend;
  {
    const float o3[3] = {ox, oy, oz}, d3[3] = {dx, dy, dz};
    const float l3[3] = {A.lo.x, A.lo.y, A.lo.z}, h3[3] = {hx, hy, hz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (d3[a] == 0.f) {
        if (o3[a] < l3[a] || o3[a] > h3[a]) return;
      } else {
        const float inv = 1.f / d3[a];
        float t0 = (l3[a] - o3[a]) * inv, t1 = (h3[a] - o3[a]) * inv;
        if (t0 > t1) {
          const float w = t0;
          t0 = t1;
          t1 = w;
        }
        ta = fmaxf(ta, t0);
        tb = fminf(tb, t1);
      }
    }
  }
  if (!(ta <= tb)) return;
  // entry cell and stepping state per axis
  int c[3], step[3], dim[3] = {A.nx, A.ny, A.nz};
  float tn[3], dt[3];
  {
    const float o3[3] = {ox, oy, oz}, d3[3] = {dx, dy, dz};
    const float l3[3] = {A.lo.x, A.lo.y, A.lo.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float pe = o3[a] + ta * d3[a];
      c[a] = min(max((int)floorf((pe - l3[a]) * A.inv_h), 0), dim[a] - 1);
      if (d3[a] > 0.f) {
        step[a] = 1;
        tn[a] = (l3[a] + (c[a] + 1) * A.h - o3[a]) / d3[a];
        dt[a] = A.h / d3[a];
      } else if (d3[a] < 0.f) {
        step[a] = -1;
        tn[a] = (l3[a] + c[a] * A.h - o3[a]) / d3[a];
        dt[a] = -A.h / d3[a];
      } else {
        step[a] = 0;
        tn[a] = INFINITY;
        dt[a] = INFINITY;
      }
    }
  }
  int seen[kRecvSeen];
  int ns = 0;
  unsigned n_cells = 0, n_entries = 0;
  const int max_steps = A.nx + A.ny + A.nz + 3;
  for (int it = 0; it < max_steps; ++it) {
    const int cell = (c[2] * A.ny + c[1]) * A.nx + c[0];
    const int e0 = __ldg(A.cell_start + cell), e1 = __ldg(A.cell_start + cell + 1);
    if (kStats) {
      ++n_cells;
      n_entries += (unsigned)(e1 - e0);
    }
    for (int e = e0; e < e1; ++e) {
      const int j = __ldg(A.items + e);
      const float4 p = __ldg(A.pos + j);
      const float qx = p.x - ox, qy = p.y - oy, qz = p.z - oz;
      const float ts = (qx * dx + qy * dy + qz * dz) * inv_dd;
      if (!(ts >= tmin && ts < tend)) continue;
      const float ex = qx - ts * dx, ey = qy - ts * dy, ez = qz - ts * dz;
      const float dist = sqrtf(ex * ex + ey * ey + ez * ez);
      const float l = lprev + ts;
      if (!(dist <= l * kr)) continue;
      bool dup = false;
      for (int q = 0; q < ns; ++q) dup = dup || seen[q] == j;
      if (dup) continue;
      if (ns < kRecvSeen) seen[ns++] = j;
      const int slot = atomicAdd(A.count, 1);
      if (slot < A.max_records) A.out[slot] = make_int4(i, j, __float_as_int(l), __float_as_int(dist));
    }
    // next cell: the axis whose boundary comes first
    const int a = tn[0] <= tn[1] ? (tn[0] <= tn[2] ? 0 : 2) : (tn[1] <= tn[2] ? 1 : 2);
    if (tn[a] > tb) break;
    c[a] += step[a];
    if (c[a] < 0 || c[a] >= dim[a]) break;
    tn[a] += dt[a];
  }
  if (kStats) {
    atomicAdd(A.stats, (unsigned long long)n_cells);
    atomicAdd(A.stats + 1, (unsigned long long)n_entries);
  }
}

}  // namespace

static int rt_rxset_create_body(const float* rx, int32_t m, float r_max, rt_rxset* out) {
  if (!rx || !out) return rt::set_error(RT_EINVAL, "NULL argument");
  *out = nullptr;
  // each receiver lands in at most 8 cells: 2^26 keeps the int cell offsets exact
  if (m < 1 || m > (1 << 26)) return rt::set_error(RT_EINVAL, "m must be 1..2^26");
  if (!(r_max > 0.f) || !std::isfinite(r_max)) return rt::set_error(RT_EINVAL, "r_max must be positive and finite");
  double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int32_t j = 0; j < m; ++j)
    for (int a = 0; a < 3; ++a) {
      const float v = rx[3 * (int64_t)j + a];
      if (!std::isfinite(v)) return rt::set_error(RT_EINVAL, "non-finite receiver position");
      lo[a] = std::min(lo[a], (double)v);
      hi[a] = std::max(hi[a], (double)v);
    }
  // cells at least two sphere radii wide, about one receiver per cell when
  // receivers are sparse, at most 2^24 cells
  const double R0 = (double)r_max * 1.001;
  double ext[3], vol = 1.0;
  for (int a = 0; a < 3; ++a) {
    ext[a] = hi[a] - lo[a] + 2.0 * R0;
    vol *= ext[a];
  }
  double h = std::max(2.0 * R0, std::cbrt(vol / m));
  for (;;) {
    double cells = 1.0;
    for (int a = 0; a < 3; ++a) cells *= std::max(1.0, std::ceil(ext[a] / h));
    if (cells <= (double)(1 << 24)) break;
    h *= 1.25;
  }
  const double R = R0 + 1e-3 * h;  // insertion radius: the sphere plus a rounding margin
  rt_rxset_s* s = new rt_rxset_s();
  struct Undo {  // frees the half-made set on an error return or exception
    rt_rxset_s* s;
    ~Undo() {
      if (s) rt_rxset_destroy(s);
    }
  } undo{s};
  s->h = (float)h;
  s->m = m;
  s->r_max = r_max;
  for (int a = 0; a < 3; ++a) {
    s->lo[a] = (float)(lo[a] - R);
    s->dims[a] = std::max(1, (int)std::ceil((hi[a] - lo[a] + 2.0 * R) / h));
  }
  const int64_t ncell = (int64_t)s->dims[0] * s->dims[1] * s->dims[2];
  // the cells of receiver j: those its widened sphere's bounding cube overlaps
  auto for_cells = [&](int32_t j, auto&& f) {
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
      const double v = rx[3 * (int64_t)j + a];
      c0[a] = std::max(0, (int)std::floor((v - R - s->lo[a]) / h));
      c1[a] = std::min(s->dims[a] - 1, (int)std::floor((v + R - s->lo[a]) / h));
    }
    for (int z = c0[2]; z <= c1[2]; ++z)
      for (int y = c0[1]; y <= c1[1]; ++y)
        for (int x = c0[0]; x <= c1[0]; ++x) f(((int64_t)z * s->dims[1] + y) * s->dims[0] + x);
  };
  std::vector<int> start(ncell + 1, 0);
  for (int32_t j = 0; j < m; ++j) for_cells(j, [&](int64_t c) { ++start[c + 1]; });
  for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
  std::vector<int> fill(start.begin(), start.end() - 1), items(std::max(1, start[ncell]), 0);
  for (int32_t j = 0; j < m; ++j) for_cells(j, [&](int64_t c) { items[fill[c]++] = j; });
  std::vector<float4> pos(m);
  for (int32_t j = 0; j < m; ++j)
    pos[j] = make_float4(rx[3 * (int64_t)j], rx[3 * (int64_t)j + 1], rx[3 * (int64_t)j + 2], 0.f);
  cudaError_t e = cudaMalloc((void**)&s->cell_start, (ncell + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->items, items.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->pos, m * sizeof(float4));
  if (e == cudaSuccess) e = cudaMemcpy(s->cell_start, start.data(), (ncell + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->pos, pos.data(), m * sizeof(float4), cudaMemcpyHostToDevice);
  if (e != cudaSuccess)
    return rt::set_error(e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA, cudaGetErrorString(e));
  undo.s = nullptr;
  *out = s;
  return RT_OK;
}

extern "C" int rt_rxset_create(const float* rx, int32_t m, float r_max, rt_rxset* out) {
  return rt::abi_guard([&] { return rt_rxset_create_body(rx, m, r_max, out); });
}

extern "C" int rt_rxset_destroy(rt_rxset s) {
  if (!s) return rt::set_error(RT_EINVAL, "receiver set is NULL");
  cudaFree(s->cell_start);
  cudaFree(s->items);
  cudaFree(s->pos);
  delete s;
  return RT_OK;
}

extern "C" int rt_receive(rt_rxset s, const rt_ray* rays, const rt_hit* hits, int64_t n, const int32_t* n_dev,
                          const rt_receive_params* p, rt_rx_record* out, int32_t* count, void* stream) {
  if (!s || !p || !count) return rt::set_error(RT_EINVAL, "NULL argument");
  if (n < 0 || n > INT_MAX) return rt::set_error(RT_EINVAL, "n out of range");
  if (n > 0 && (!rays || !hits)) return rt::set_error(RT_EINVAL, "NULL rays or hits");
  if (((uintptr_t)rays & 15) || ((uintptr_t)hits & 15) || ((uintptr_t)out & 15))
    return rt::set_error(RT_EINVAL, "rays, hits and records must be 16-byte aligned");
  if (!(p->delta > 0.f) || !std::isfinite(p->delta) || !(p->range0 > 0.f) || !std::isfinite(p->range0))
    return rt::set_error(RT_EINVAL, "delta and range0 must be positive and finite");
  if (p->max_records < 0 || (p->max_records > 0 && !out)) return rt::set_error(RT_EINVAL, "bad record buffer");
  if ((uintptr_t)p->stats_dev & 7) return rt::set_error(RT_EINVAL, "stats_dev must be 8-byte aligned");
  const float k = (float)(p->delta / std::sqrt(3.0));
  if ((double)p->range0 * k > (double)s->r_max * 1.0001)
    return rt::set_error(RT_EINVAL, "range0 * delta / sqrt(3) exceeds the receiver set's r_max");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return rt::set_error(RT_ECUDA, cudaGetErrorString(e));
  if (n == 0) return RT_OK;
  RecvArgs A;
  A.rays = reinterpret_cast<const float4*>(rays);
  A.hits = reinterpret_cast<const float4*>(hits);
  A.n = (int)n;
  A.n_dev = n_dev;
  A.lo = make_float3(s->lo[0], s->lo[1], s->lo[2]);
  A.h = s->h;
  A.inv_h = 1.f / s->h;
  A.nx = s->dims[0];
  A.ny = s->dims[1];
  A.nz = s->dims[2];
  A.cell_start = s->cell_start;
  A.items = s->items;
  A.pos = s->pos;
  A.k = k;
  A.delta_ray = p->delta_ray_dev;
  A.k_cap = (float)((double)s->r_max * 1.0001 / (double)p->range0);
  A.range0 = p->range0;
  A.max_records = p->max_records;
  A.out = reinterpret_cast<int4*>(out);
  A.count = count;
  A.stats = p->stats_dev;
  const int grid = (int)((n + kRecvBlock - 1) / kRecvBlock);
  if (A.stats)
    k_receive<true><<<grid, kRecvBlock, 0, st>>>(A);
  else
    k_receive<false><<<grid, kRecvBlock, 0, st>>>(A);
  rt::count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rt::set_error(RT_ECUDA, cudaGetErrorString(e));
  return RT_OK;
}

extern "C" int rt_abi_struct_sizes(int64_t* sizes, int32_t n) {
  const int64_t v[12] = {sizeof(rt_ray),         sizeof(rt_hit),           sizeof(rt_build_params),
                         sizeof(rt_trace_params), sizeof(rt_bvh_info_t),    sizeof(rt_tune_result),
                         sizeof(rt_rx_record),    sizeof(rt_receive_params), sizeof(rt_batch_desc),
                         sizeof(rt_batch_stats),  sizeof(rt_request),       sizeof(rt_session_stats)};
  for (int32_t i = 0; sizes && i < n && i < 12; ++i) sizes[i] = v[i];
  return 12;
}
