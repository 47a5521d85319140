// Ray launch (Sec. III.A) and specular bounce with compaction (Sec. III.B).
//
// k_gen_fibonacci / k_gen_icosphere write rays from a source point towards
//   Fibonacci-sphere points or the vertices of a subdivided regular
//   icosahedron (f = 2^level segments per edge, 10 f^2 + 2 directions), in
//   float32, in launch order (fib_slot, ico_slot_point): the 32 rays of a
//   warp are neighbours on the sphere and walk the same nodes.
// k_reflect_* turn every hit ray into its specular reflection r = d -
//   2 (d.n) n about the unit geometric normal of the hit triangle, starting at
//   the hit point with the remaining range tmax - t and the hit triangle to
//   be skipped, and compact the survivors into the next order's ray queue in
//   input order (count per block, scan, scatter: deterministic).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int kRayBlock = 256;

// 0.38196601125010515... = (3 - sqrt 5) / 2 as a 64-bit binary fraction, so
// that the fractional part of i * g (the azimuth in turns) is exact integer
// arithmetic for every i.
constexpr unsigned long long kGoldenFrac = 0x61C8864680B583EAull;

// Direction i of an n-point Fibonacci launch.
__device__ __forceinline__ float3 fib_dir(long long i, long long n) {
  // z = 1 - (2i + 1)/n = (n - 2i - 1)/n and rho = sqrt(1 - z^2) =
  // sqrt((2i + 1)(2n - 2i - 1)) / n, each from exact integers (no
  // cancellation near the poles), in float32 with every step rounded to
  // nearest: each integer, the product, the root and the quotient add at
  // most half an ulp, so z and rho lie within 4 ulp (< 2.5e-7) of their
  // exact values
  const float fn = __ll2float_rn(n);
  const float z = __fdiv_rn(__ll2float_rn(n - 2 * i - 1), fn);
  const float rho = __fdiv_rn(__fsqrt_rn(__fmul_rn(__ll2float_rn(2 * i + 1), __ll2float_rn(2 * n - 2 * i - 1))), fn);
  // azimuth in turns, i (3 - sqrt 5)/2 mod 1, reduced to [-1/2, 1/2) in
  // exact integer arithmetic before the one rounding to float
  const unsigned long long turns = (unsigned long long)i * kGoldenFrac;  // mod 2^64
  const float a = (float)(int)(unsigned)(turns >> 32) * 2.3283064365386963e-10f;  // 2^-32
  float s, c;
  sincospif(2.f * a, &s, &c);
  return make_float3(__fmul_rn(rho, c), __fmul_rn(rho, s), z);
}

__global__ void k_gen_fibonacci(float ox, float oy, float oz, long long n, long long w, long long c, float tmin,
                                float tmax, float4* __restrict__ rays) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float3 d = fib_dir(fib_slot(i, n, w, c), n);
    rays[2 * i] = make_float4(ox, oy, oz, tmin);
    rays[2 * i + 1] = make_float4(d.x, d.y, d.z, tmax);
  }
}

// Icosahedron tables (vertices, edges, faces) for the device generator.
struct Ico {
  float v[12][3];
  int e[30][2];
  int f[20][3];
};
__constant__ Ico c_ico;

// Direction towards point p of the icosahedron with every edge cut into f
// segments, normalised; every operation rounded explicitly (the same bits in
// every kernel that generates it).
__device__ __forceinline__ float3 ico_dir(const IcoPt& p, long long f) {
  const float inv_f = __frcp_rn((float)f);
  float p0, p1, p2;
  if (p.kind == 0) {
    p0 = c_ico.v[p.a][0];
    p1 = c_ico.v[p.a][1];
    p2 = c_ico.v[p.a][2];
  } else if (p.kind == 1) {
    const float t = __fmul_rn((float)p.i, inv_f), u = __fsub_rn(1.f, t);
    const float* a = c_ico.v[c_ico.e[p.a][0]];
    const float* b = c_ico.v[c_ico.e[p.a][1]];
    p0 = __fadd_rn(__fmul_rn(a[0], u), __fmul_rn(b[0], t));
    p1 = __fadd_rn(__fmul_rn(a[1], u), __fmul_rn(b[1], t));
    p2 = __fadd_rn(__fmul_rn(a[2], u), __fmul_rn(b[2], t));
  } else {
    const float wi = __fmul_rn((float)p.i, inv_f), wj = __fmul_rn((float)p.j, inv_f);
    const float w0 = __fsub_rn(__fsub_rn(1.f, wi), wj);
    const float* a = c_ico.v[c_ico.f[p.a][0]];
    const float* b = c_ico.v[c_ico.f[p.a][1]];
    const float* c = c_ico.v[c_ico.f[p.a][2]];
    p0 = __fadd_rn(__fadd_rn(__fmul_rn(a[0], w0), __fmul_rn(b[0], wi)), __fmul_rn(c[0], wj));
    p1 = __fadd_rn(__fadd_rn(__fmul_rn(a[1], w0), __fmul_rn(b[1], wi)), __fmul_rn(c[1], wj));
    p2 = __fadd_rn(__fadd_rn(__fmul_rn(a[2], w0), __fmul_rn(b[2], wi)), __fmul_rn(c[2], wj));
  }
  const float il = rsqrtf(__fadd_rn(__fadd_rn(__fmul_rn(p0, p0), __fmul_rn(p1, p1)), __fmul_rn(p2, p2)));
  return make_float3(__fmul_rn(p0, il), __fmul_rn(p1, il), __fmul_rn(p2, il));
}

__global__ void k_gen_icosphere(float ox, float oy, float oz, int fseg, long long n, float tmin, float tmax,
                                float4* __restrict__ rays) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const float3 d = ico_dir(ico_slot_point(k, fseg), fseg);
    rays[2 * k] = make_float4(ox, oy, oz, tmin);
    rays[2 * k + 1] = make_float4(d.x, d.y, d.z, tmax);
  }
}

// The launches of many transmitters in one kernel: transmitter t's rays
// occupy [off[t], off[t + 1]) (each the same rays its own launch writes);
// param[t] holds the icosphere level, or the band width w and step c of a
// Fibonacci launch as w << 32 | c.
__global__ void k_gen_batch(int kind, const float* __restrict__ tx, const long long* __restrict__ off,
                            const long long* __restrict__ param, int n_tx, float tmin, float tmax,
                            float4* __restrict__ rays) {
  const long long total = off[n_tx];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_tx - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= i)
        lo = mid;
      else
        hi = mid - 1;
    }
    const long long j = i - off[lo];
    float3 d;
    if (kind == RT_RAYS_FIBONACCI) {
      const long long n = off[lo + 1] - off[lo];
      const unsigned long long wc = (unsigned long long)param[lo];
      d = fib_dir(fib_slot(j, n, (long long)(wc >> 32), (long long)(wc & 0xffffffffull)), n);
    } else {
      d = ico_dir(ico_slot_point(j, 1ll << param[lo]), 1ll << param[lo]);
    }
    rays[2 * i] = make_float4(tx[3 * lo], tx[3 * lo + 1], tx[3 * lo + 2], tmin);
    rays[2 * i + 1] = make_float4(d.x, d.y, d.z, tmax);
  }
}

// ------------------------------------------------------------------ bounce
struct ReflectArgs {
  const float4* rays;
  const float4* hits;
  const int* n_dev;      // nullable: count on the device (else n)
  long long n;
  const float4* tri_in;  // input-order triangles
  float4* out_rays;
  int* out_skip;
  int* out_src;          // nullable
  int* out_count;
  int* block_counts;
  long long cap;
};

__device__ __forceinline__ bool survives(const ReflectArgs& A, long long i, float4* hit) {
  *hit = A.hits[i];
  const int id = __float_as_int(hit->y);
  const float4 rb = A.rays[2 * i + 1];
  return id >= 0 && rb.w - hit->x > 0.f;
}

__device__ __forceinline__ long long count_of(const ReflectArgs& A) {
  return A.n_dev ? (long long)*A.n_dev : A.n;
}

__global__ void __launch_bounds__(kRayBlock) k_reflect_count(ReflectArgs A) {
  __shared__ int wsum[kRayBlock / 32];
  const long long n = count_of(A);
  const long long i = blockIdx.x * (long long)kRayBlock + threadIdx.x;
  float4 h;
  const bool keep = i < n && survives(A, i, &h);
  __syncwarp();
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kRayBlock / 32; ++w) t += wsum[w];
    A.block_counts[blockIdx.x] = t;
  }
}

// Exclusive scan of the block counts (one CTA) and the total.
__global__ void __launch_bounds__(1024) k_reflect_scan(ReflectArgs A, int nblocks) {
  __shared__ int carry;
  __shared__ int ws[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nblocks; b0 += 1024) {
    const int b = b0 + threadIdx.x;
    const int v = b < nblocks ? A.block_counts[b] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
      if (w < (int)(threadIdx.x >> 5)) off += ws[w];
      tot += ws[w];
    }
    if (b < nblocks) A.block_counts[b] = carry + off + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *A.out_count = (int)min((long long)carry, A.cap);
}

__global__ void __launch_bounds__(kRayBlock) k_reflect_scatter(ReflectArgs A) {
  __shared__ int wsum[kRayBlock / 32];
  const long long n = count_of(A);
  const long long i = blockIdx.x * (long long)kRayBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
  const bool keep = i < n && survives(A, i, &h);
  __syncwarp();
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  if (lane == 0) wsum[warp] = __popc(m);
  __syncthreads();
  if (!keep) return;
  int pos = A.block_counts[blockIdx.x];
  for (int w = 0; w < warp; ++w) pos += wsum[w];
  pos += __popc(m & ((1u << lane) - 1u));
  if (pos >= A.cap) return;
  const float4 ra = A.rays[2 * i], rb = A.rays[2 * i + 1];
  const int id = __float_as_int(h.y);
  float4 o0, o1;
  reflect_ray(ra, rb, h.x, A.tri_in[3 * (size_t)id], A.tri_in[3 * (size_t)id + 1], A.tri_in[3 * (size_t)id + 2], &o0,
              &o1);
  A.out_rays[2 * (size_t)pos] = o0;
  A.out_rays[2 * (size_t)pos + 1] = o1;
  A.out_skip[pos] = id;
  if (A.out_src) A.out_src[pos] = (int)i;
}

std::once_flag g_ico_once;
bool g_ico_ok = false;

// The regular icosahedron with vertices (0, +-1, +-phi) and cyclic shifts;
// edges and faces found as vertex pairs / triples at the edge length 2,
// listed in lexicographic order of their sorted indices.
void init_ico() {
  Ico h;
  const double g = (1.0 + std::sqrt(5.0)) / 2.0;
  double v[12][3];
  int k = 0;
  for (double a : {-1.0, 1.0})
    for (double b : {-g, g}) {
      const double tri[3][3] = {{0.0, a, b}, {a, b, 0.0}, {b, 0.0, a}};
      for (auto& p : tri) {
        v[k][0] = p[0];
        v[k][1] = p[1];
        v[k][2] = p[2];
        ++k;
      }
    }
  auto adj = [&](int i, int j) {
    const double dx = v[i][0] - v[j][0], dy = v[i][1] - v[j][1], dz = v[i][2] - v[j][2];
    return std::fabs(std::sqrt(dx * dx + dy * dy + dz * dz) - 2.0) < 1e-9;
  };
  int ne = 0, nf = 0;
  for (int i = 0; i < 12; ++i)
    for (int j = i + 1; j < 12; ++j) {
      if (!adj(i, j)) continue;
      if (ne < 30) {
        h.e[ne][0] = i;
        h.e[ne][1] = j;
      }
      ++ne;
      for (int l = j + 1; l < 12; ++l)
        if (adj(j, l) && adj(i, l)) {
          if (nf < 20) {
            h.f[nf][0] = i;
            h.f[nf][1] = j;
            h.f[nf][2] = l;
          }
          ++nf;
        }
    }
  for (int i = 0; i < 12; ++i)
    for (int a = 0; a < 3; ++a) h.v[i][a] = (float)v[i][a];
  g_ico_ok = ne == 30 && nf == 20 && cudaMemcpyToSymbol(c_ico, &h, sizeof(h)) == cudaSuccess;
}

int grid_for(long long n, int nsm) {
  long long g = (n + kRayBlock - 1) / kRayBlock;
  const long long gmax = (long long)nsm * 16;
  if (g > gmax) g = gmax;
  return g < 1 ? 1 : (int)g;
}

int sms() {
  static int n = 0;
  if (!n) {
    int d = 0;
    cudaGetDevice(&d);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

void fib_launch_order(long long n, long long* w, long long* c) {
  // Fibonacci numbers F_k (F_1 = F_2 = 1); w = F_k, the largest with
  // F_k^2 <= 80 n (k >= 3), which makes a band about sqrt(80 n) points long
  // and 2 sqrt(80 / n) high in z: a warp's 32 neighbours in azimuth then
  // cover a patch about as wide as it is high.  The points j g mod 1
  // (g = (3 - sqrt 5) / 2), j < F_k, follow one another in the order
  // j -> j + c mod F_k with c the even-indexed one of F_(k-1) and F_(k-2)
  // (three-gap theorem; the continued fraction of g has all partial
  // quotients 1 after the first two).
  long long f2 = 1, f1 = 1, f = 2;  // F_(k-2), F_(k-1), F_k for k = 3
  int k = 3;
  const long long lim = 80 * (n > 0 ? n : 0);
  while ((f1 + f) <= lim / (f1 + f)) {
    f2 = f1;
    f1 = f;
    f = f1 + f2;
    ++k;
  }
  *w = f;
  *c = ((k - 1) & 1) == 0 ? f1 : f2;
}

cudaError_t launch_gen_rays(int kind, const float* o, long long param, float tmin, float tmax, rt_ray* rays,
                            long long count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (kind == RT_RAYS_FIBONACCI) {
    long long w = 1, c = 1;
    fib_launch_order(count, &w, &c);
    k_gen_fibonacci<<<grid_for(count, sms()), kRayBlock, 0, st>>>(o[0], o[1], o[2], count, w, c, tmin, tmax,
                                                                   reinterpret_cast<float4*>(rays));
  } else {
    std::call_once(g_ico_once, init_ico);
    if (!g_ico_ok) return cudaErrorInitializationError;
    k_gen_icosphere<<<grid_for(count, sms()), kRayBlock, 0, st>>>(o[0], o[1], o[2], 1 << param, count, tmin,
                                                                   tmax, reinterpret_cast<float4*>(rays));
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gen_batch(int kind, const float* tx_dev, const long long* off_dev, const long long* param_dev,
                             int n_tx, long long total, float tmin, float tmax, rt_ray* rays, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  if (kind == RT_RAYS_ICOSPHERE) {
    std::call_once(g_ico_once, init_ico);
    if (!g_ico_ok) return cudaErrorInitializationError;
  }
  k_gen_batch<<<grid_for(total, sms()), kRayBlock, 0, st>>>(kind, tx_dev, off_dev, param_dev, n_tx, tmin, tmax,
                                                             reinterpret_cast<float4*>(rays));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_reflect(const rt_scene_s* s, const rt_ray* rays, const rt_hit* hits, long long n,
                           const int* n_dev, rt_ray* out_rays, int* out_skip, int* out_src, int* out_count,
                           int* block_counts, long long cap, cudaStream_t st) {
  ReflectArgs A;
  A.rays = reinterpret_cast<const float4*>(rays);
  A.hits = reinterpret_cast<const float4*>(hits);
  A.n_dev = n_dev;
  A.n = n;
  A.tri_in = s->tri_in;
  A.out_rays = reinterpret_cast<float4*>(out_rays);
  A.out_skip = out_skip;
  A.out_src = out_src;
  A.out_count = out_count;
  A.block_counts = block_counts;
  A.cap = cap;
  const int nb = (int)((n + kRayBlock - 1) / kRayBlock);
  if (nb == 0) return cudaMemsetAsync(out_count, 0, sizeof(int), st);
  k_reflect_count<<<nb, kRayBlock, 0, st>>>(A);
  k_reflect_scan<<<1, 1024, 0, st>>>(A, nb);
  k_reflect_scatter<<<nb, kRayBlock, 0, st>>>(A);
  count_launches(3);
  return cudaGetLastError();
}

}  // namespace rt
