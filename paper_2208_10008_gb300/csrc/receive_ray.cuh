// Receiving-sphere test of one path segment (Sec. III.C, Eq. 4), shared by
// the reception kernel and the one-launch batch pipeline.
#pragma once

#include <cuda_runtime.h>

#include "rtbvh.h"

namespace rt {

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

// The receiving spheres met by the segment of ray i of `rays` / `hits` (the
// caller checks i against the ray count), records to out / count, the
// ray's delta from `delta` when not null; the grid and the constants from A.
template <bool kStats>
__device__ __forceinline__ void receive_one(const RecvArgs& A, const int i, const float4* __restrict__ rays,
                                            const float4* __restrict__ hits, const float* __restrict__ delta,
                                            int4* __restrict__ out, int* __restrict__ count) {
  const float4 ra = __ldg(rays + 2 * i), rb = __ldg(rays + 2 * i + 1);
  const float ht = __ldg(&hits[i].x);
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
  const float kr = delta ? fminf(__ldg(delta + i) * 0.57735026918962576f, A.k_cap) : A.k;
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
      const int slot = atomicAdd(count, 1);
      if (slot < A.max_records) out[slot] = make_int4(i, j, __float_as_int(l), __float_as_int(dist));
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

// The grid, the constants and the checks of rt_receive for the receiver set
// and parameters; rays, hits, counts and records are the caller's.  Returns
// an RT_* code (message set).
int receive_args(const struct rt_rxset_s* s, const rt_receive_params* p, RecvArgs* A);

}  // namespace rt
