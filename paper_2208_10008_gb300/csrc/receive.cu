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
#include "receive_ray.cuh"

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

using rt::RecvArgs;
using rt::receive_one;

constexpr int kRecvBlock = 256;

template <bool kStats>
__global__ void __launch_bounds__(kRecvBlock) k_receive(RecvArgs A) {
  const int i = blockIdx.x * kRecvBlock + threadIdx.x;
  const int n = A.n_dev ? min(A.n, __ldg(A.n_dev)) : A.n;
  if (i >= n) return;
  receive_one<kStats>(A, i, A.rays, A.hits, A.delta_ray, A.out, A.count);
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

namespace rt {
int receive_args(const rt_rxset_s* s, const rt_receive_params* p, RecvArgs* A) {
  if (!s || !p) return rt::set_error(RT_EINVAL, "NULL argument");
  if (!(p->delta > 0.f) || !std::isfinite(p->delta) || !(p->range0 > 0.f) || !std::isfinite(p->range0))
    return rt::set_error(RT_EINVAL, "delta and range0 must be positive and finite");
  if (p->max_records < 0) return rt::set_error(RT_EINVAL, "bad record buffer");
  if ((uintptr_t)p->stats_dev & 7) return rt::set_error(RT_EINVAL, "stats_dev must be 8-byte aligned");
  const float k = (float)(p->delta / std::sqrt(3.0));
  if ((double)p->range0 * k > (double)s->r_max * 1.0001)
    return rt::set_error(RT_EINVAL, "range0 * delta / sqrt(3) exceeds the receiver set's r_max");
  A->rays = nullptr;
  A->hits = nullptr;
  A->n = 0;
  A->n_dev = nullptr;
  A->lo = make_float3(s->lo[0], s->lo[1], s->lo[2]);
  A->h = s->h;
  A->inv_h = 1.f / s->h;
  A->nx = s->dims[0];
  A->ny = s->dims[1];
  A->nz = s->dims[2];
  A->cell_start = s->cell_start;
  A->items = s->items;
  A->pos = s->pos;
  A->k = k;
  A->delta_ray = p->delta_ray_dev;
  A->k_cap = (float)((double)s->r_max * 1.0001 / (double)p->range0);
  A->range0 = p->range0;
  A->max_records = p->max_records;
  A->out = nullptr;
  A->count = nullptr;
  A->stats = p->stats_dev;
  return RT_OK;
}
}  // namespace rt

extern "C" int rt_receive(rt_rxset s, const rt_ray* rays, const rt_hit* hits, int64_t n, const int32_t* n_dev,
                          const rt_receive_params* p, rt_rx_record* out, int32_t* count, void* stream) {
  if (!s || !p || !count) return rt::set_error(RT_EINVAL, "NULL argument");
  if (n < 0 || n > INT_MAX) return rt::set_error(RT_EINVAL, "n out of range");
  if (n > 0 && (!rays || !hits)) return rt::set_error(RT_EINVAL, "NULL rays or hits");
  if (((uintptr_t)rays & 15) || ((uintptr_t)hits & 15) || ((uintptr_t)out & 15))
    return rt::set_error(RT_EINVAL, "rays, hits and records must be 16-byte aligned");
  if (p->max_records > 0 && !out) return rt::set_error(RT_EINVAL, "bad record buffer");
  RecvArgs A;
  const int rc = rt::receive_args(s, p, &A);
  if (rc != RT_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return rt::set_error(RT_ECUDA, cudaGetErrorString(e));
  if (n == 0) return RT_OK;
  A.rays = reinterpret_cast<const float4*>(rays);
  A.hits = reinterpret_cast<const float4*>(hits);
  A.n = (int)n;
  A.n_dev = n_dev;
  A.out = reinterpret_cast<int4*>(out);
  A.count = count;
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
