// Instrumentation with no counterpart in the paper: the read bandwidth of the
// L2 cache, the ceiling of a walk whose nodes and triangles stay resident
// there.  One launch reads a device buffer that fits in the L2 `reps` times
// with 16-byte loads that are cached in L2 only (ld.global.cg), so every
// load after the first pass is an L2 hit; the loaded words feed a
// reduction whose result is stored only on a condition that never holds, so
// no load can be dropped.
#include <cuda_runtime.h>

#include "rt_internal.cuh"

namespace {

constexpr int kProbeBlock = 512;
constexpr int kUnroll = 4;

__global__ void __launch_bounds__(kProbeBlock) k_l2_read(const float4* __restrict__ buf, long long n4, int reps,
                                                        unsigned* sink) {
  unsigned acc = 0;
  const long long nt = (long long)gridDim.x * kProbeBlock;
  const long long t0 = (long long)blockIdx.x * kProbeBlock + threadIdx.x;
  for (int r = 0; r < reps; ++r) {
    long long i = t0;
    for (; i + (kUnroll - 1) * nt < n4; i += kUnroll * nt) {
      float4 v[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) v[u] = __ldcg(buf + i + u * nt);
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        acc ^= __float_as_uint(v[u].x) ^ __float_as_uint(v[u].y) ^ __float_as_uint(v[u].z) ^ __float_as_uint(v[u].w);
    }
    for (; i < n4; i += nt) {
      const float4 v = __ldcg(buf + i);
      acc ^= __float_as_uint(v.x) ^ __float_as_uint(v.y) ^ __float_as_uint(v.z) ^ __float_as_uint(v.w);
    }
    acc = acc * 0x9e3779b9u + (unsigned)r;
  }
  if (acc == 0x2545f491u && sink) sink[blockIdx.x] = acc;
}

}  // namespace

extern "C" int rt_probe_l2_read(const void* buf_dev, int64_t bytes, int32_t reps, uint32_t* sink_dev,
                                void* stream) {
  if (!buf_dev || bytes < 16 || (bytes & 15) || ((uintptr_t)buf_dev & 15) || reps < 1)
    return rt::set_error(RT_EINVAL, "rt_probe_l2_read: 16-byte aligned buffer of a multiple of 16 bytes, reps >= 1");
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return rt::set_error(RT_ECUDA, "device query failed");
  const long long n4 = bytes / 16;
  long long grid = (long long)nsm * 4;  // 2048 threads on every SM
  if (grid * kProbeBlock > n4) grid = (n4 + kProbeBlock - 1) / kProbeBlock;
  k_l2_read<<<(int)grid, kProbeBlock, 0, (cudaStream_t)stream>>>(static_cast<const float4*>(buf_dev), n4, reps,
                                                                  sink_dev);
  rt::count_launches(1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rt::set_error(RT_ECUDA, cudaGetErrorString(e));
  return RT_OK;
}
