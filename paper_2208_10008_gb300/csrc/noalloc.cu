// rt_trace_closest_noalloc: closest-hit tracing that never allocates device
// memory.
//
// rt_trace_closest keeps a per-scene scratch area for the rays its float32
// pass hands to the float64 re-test, and grows it with cudaMalloc the first
// time a larger batch arrives.  Some callers cannot let a library do that:
// a serving runtime that owns every byte of device memory through its own
// pool and budgets it per tenant, or a latency-critical loop where an
// allocation (which may synchronise the whole device) would stall other
// streams.  This entry point gives them the same result with the scratch
// taken from one fixed array compiled into the library instead.
//
// The array below is the only scratch this call uses.  It is a file-scope
// device variable, so every GPU that loads the library holds it (10 MiB)
// until the process exits.  Host code cannot use the array's name as a
// device address; its address on each device is looked up with
// cudaGetSymbolAddress the first time the call runs on that device, with
// that device current, and cached for the life of the process (a device
// reset, which invalidates every scene, invalidates this address too).
#include <cuda_runtime.h>

#include <mutex>

#include "rt_internal.cuh"

namespace {

constexpr int64_t kMaxRays = RT_NOALLOC_MAX_RAYS;
// counter block (4 ints, padded to 64) + queue (kMaxRays) + candidate lists
constexpr int64_t kScratchInts = 64 + kMaxRays + kMaxRays * (rt::kTraceCand + 1);

static __device__ __align__(256) int g_noalloc_scratch[kScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int* g_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" int rt_trace_closest_noalloc(rt_scene scene, const rt_ray* rays_dev, int64_t n, rt_hit* hits_dev,
                                        const rt_trace_params* params, void* stream) {
  return rt::abi_guard([&]() -> int {
    if (!scene) return rt::set_error(RT_EINVAL, "scene is NULL");
    if (n < 0) return rt::set_error(RT_EINVAL, "n out of range");
    if (n > kMaxRays)
      return rt::set_error(RT_EINVAL,
                           "rt_trace_closest_noalloc: n exceeds RT_NOALLOC_MAX_RAYS (262144); split the batch");
    if (n > 0 && (!rays_dev || !hits_dev)) return rt::set_error(RT_EINVAL, "NULL buffer");
    if (((uintptr_t)rays_dev & 15) || ((uintptr_t)hits_dev & 15))
      return rt::set_error(RT_EINVAL, "rays/hits must be 16-byte aligned");
    if (params && params->block != 0 && params->block != 64 && params->block != 128 && params->block != 256)
      return rt::set_error(RT_EINVAL, "block must be 0, 64, 128 or 256");
    if (params && ((params->stack != 0 && params->stack != 16 && params->stack != 32 && params->stack != 64)))
      return rt::set_error(RT_EINVAL, "stack must be 0, 16, 32 or 64");
    if (params && (params->flags & RT_QUANTIZED_NODES) && !scene->q_built)
      return rt::set_error(RT_EINVAL, "RT_QUANTIZED_NODES needs a build with quantize = 1");
    if (!scene->built) return rt::set_error(RT_ENOTBUILT, "BVH not built");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
      return rt::set_error(RT_ECUDA, "cudaGetDevice failed or device index too large");
    // the kernels run on the current device against the scene's tree and this
    // device's copy of the array: the scene must live here
    if (dev != scene->device)
      return rt::set_error(RT_EINVAL, "the scene was uploaded on another device; make that device current");
    int* base = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_mu);
      if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
          cudaGetLastError();
          return rt::set_error(RT_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
        }
        g_addr[dev] = static_cast<int*>(p);
      }
      base = g_addr[dev];
    }
    rt::TraceScratch scr;
    scr.counter = base;          // zeroed by launch_trace on the stream
    scr.queue = base + 64;
    scr.cand = base + 64 + kMaxRays;
    scr.cap = kMaxRays;
    cudaError_t e = rt::launch_trace(scene, rays_dev, n, hits_dev, nullptr, params, scr, (cudaStream_t)stream);
    if (e != cudaSuccess) return rt::set_error(RT_ECUDA, cudaGetErrorString(e));
    return RT_OK;
  });
}
