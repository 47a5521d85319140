// Autotuner of the build and walk parameters (rt_autotune in rtbvh.h).
//
// The knobs are the ones that trade build time against walk time without
// changing any hit: the traversal node width, the leaf size, the number of
// bins per axis, and the ray tile (rays per CTA) and stack depth of the
// float32 walk.  Every configuration is built
// and timed with CUDA events on the caller's stream (median of 5, L2 flushed
// before each timing by a 256 MB write, so that the ranking is the one of
// cold-cache steps), and the scene is left built with the winner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>

#include "rt_internal.cuh"

namespace rt {
int set_error(int code, const char* msg);  // records the message for rt_last_error
}

namespace {

struct Events {
  cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
  ~Events() {
    for (cudaEvent_t x : e)
      if (x) cudaEventDestroy(x);
  }
};

constexpr int kTuneReps = 5;
constexpr size_t kFlushBytes = size_t(256) << 20;  // twice the L2

// Device time of `fn` (enqueueing on st), median of kTuneReps, each after
// an untimed write of `flush` (nullable) that evicts the L2; negative on
// failure.
template <class F>
float median_ms(cudaStream_t st, const Events& ev, void* flush, F fn, int* err) {
  float t[kTuneReps];
  for (int r = 0; r < kTuneReps; ++r) {
    if (flush && cudaMemsetAsync(flush, r, kFlushBytes, st) != cudaSuccess) return -1.f;
    if (cudaEventRecord(ev.e[0], st) != cudaSuccess) return -1.f;
    *err = fn();
    if (*err) return -1.f;
    if (cudaEventRecord(ev.e[1], st) != cudaSuccess || cudaEventSynchronize(ev.e[1]) != cudaSuccess) return -1.f;
    if (cudaEventElapsedTime(&t[r], ev.e[0], ev.e[1]) != cudaSuccess) return -1.f;
  }
  std::sort(t, t + kTuneReps);
  return t[kTuneReps / 2];
}

}  // namespace

extern "C" int rt_autotune(rt_scene s, const rt_build_params* base, const rt_ray* rays, int64_t n,
                           float build_weight, rt_tune_result* out, void* stream) {
  if (!s || !base || !rays || !out) return rt::set_error(RT_EINVAL, "NULL argument");
  if (n < 1 || n > INT_MAX) return rt::set_error(RT_EINVAL, "n_rays out of range");
  if (!(build_weight >= 0.f) || build_weight > 1e6f) return rt::set_error(RT_EINVAL, "build_weight must be >= 0");
  if (((uintptr_t)rays & 15)) return rt::set_error(RT_EINVAL, "rays must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  Events ev;
  for (cudaEvent_t& x : ev.e)
    if (cudaEventCreate(&x) != cudaSuccess) return rt::set_error(RT_ECUDA, "create events");
  rt_hit* hits = nullptr;
  if (cudaMalloc((void**)&hits, sizeof(rt_hit) * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    return rt::set_error(RT_ENOMEM, "hit buffer");
  }
  void* flush = nullptr;  // without it (no memory) the timings are warm-cache
  if (cudaMalloc(&flush, kFlushBytes) != cudaSuccess) {
    cudaGetLastError();
    flush = nullptr;
  }
  // Two stages.  The tree (node width x leaf size x bins), each build timed
  // and its walk timed with the default tile and stack; then the walk of the
  // chosen tree (ray tile x stack depth).
  const int widths[] = {4, 8}, leaves[] = {2, 4, 6, 8}, binsv[] = {8, 16, 32};
  const int tiles[] = {64, 128, 256}, stacks[] = {16, 32, 64};
  rt_tune_result best{};
  best.score_ms = FLT_MAX;
  best.default_score_ms = -1.f;
  best.block = 128;
  best.stack = 64;
  int err = 0, tried = 0;
  for (int wd : widths) {
    for (int ml : leaves) {
      for (int bn : binsv) {
        rt_build_params p = *base;
        p.width = wd;
        p.max_leaf = ml;
        p.bins = bn;
        p.quantize = 0;
        err = rt_bvh_build(s, &p, stream);  // warm: the first build sizes the scene's buffers
        if (err) goto done;
        const float tb = median_ms(st, ev, flush, [&] { return rt_bvh_build(s, &p, stream); }, &err);
        if (tb < 0.f) goto fail_cuda;
        rt_trace_params tp{};
        err = rt_trace_closest(s, rays, n, hits, &tp, stream);
        if (err) goto done;
        const float tt =
            median_ms(st, ev, flush, [&] { return rt_trace_closest(s, rays, n, hits, &tp, stream); }, &err);
        if (tt < 0.f) goto fail_cuda;
        const float score = build_weight * tb + tt;
        ++tried;
        if (wd == 4 && ml == 4 && bn == 16) best.default_score_ms = score;
        if (score < best.score_ms) {
          best.width = wd;
          best.max_leaf = ml;
          best.bins = bn;
          best.build_ms = tb;
          best.trace_ms = tt;
          best.score_ms = score;
        }
      }
    }
  }
  {
    rt_build_params p = *base;
    p.width = best.width;
    p.max_leaf = best.max_leaf;
    p.bins = best.bins;
    p.quantize = 0;
    err = rt_bvh_build(s, &p, stream);
    if (err) goto done;
    for (int tile : tiles) {
      for (int sd : stacks) {
        if (tile == 128 && sd == 64) continue;  // timed in the first stage
        rt_trace_params tp{};
        tp.block = tile;
        tp.stack = sd;
        err = rt_trace_closest(s, rays, n, hits, &tp, stream);
        if (err) goto done;
        const float tt =
            median_ms(st, ev, flush, [&] { return rt_trace_closest(s, rays, n, hits, &tp, stream); }, &err);
        if (tt < 0.f) goto fail_cuda;
        ++tried;
        const float score = build_weight * best.build_ms + tt;
        if (score < best.score_ms) {
          best.block = tile;
          best.stack = sd;
          best.trace_ms = tt;
          best.score_ms = score;
        }
      }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) goto fail_cuda;
  }
  best.n_tried = tried;
  *out = best;
done:
  cudaFree(hits);
  if (flush) cudaFree(flush);
  return err;
fail_cuda:
  cudaFree(hits);
  if (flush) cudaFree(flush);
  if (err) return err;
  return rt::set_error(RT_ECUDA, "timing failed");
}
