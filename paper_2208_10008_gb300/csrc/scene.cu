// C-ABI entry points of librtbvh (declared in include/rtbvh.h): scene
// lifetime, triangle upload, build / trace dispatch and the host-buffer
// pipeline.  Device work lives in build.cu and trace.cu.
#include <cuda_runtime.h>

#include <atomic>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "rt_internal.cuh"

namespace rt {
static std::atomic<uint64_t> g_launches{0};
void count_launches(int k) { g_launches.fetch_add((uint64_t)(int64_t)k, std::memory_order_relaxed); }

static std::atomic<int> g_spin_limit{0}, g_phantom_tasks{0}, g_phantom_items{0};
static std::atomic<long long> g_fail_alloc{0};  // allocations left before the injected failure (0: off)
DebugHooks debug_hooks() {
  return DebugHooks{g_spin_limit.load(), g_phantom_tasks.load(), g_phantom_items.load()};
}
// True when the injected allocation failure is due now.
bool alloc_should_fail() {
  long long v = g_fail_alloc.load();
  while (v > 0) {
    if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 1;
  }
  return false;
}
}  // namespace rt

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  int code = e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;
  return fail(code, "%s: %s", what, cudaGetErrorString(e));
}

#define RT_CUDA(call, what)                  \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

template <class T>
cudaError_t dev_alloc(T** p, size_t count) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) count = 1;
  if (rt::alloc_should_fail()) return cudaErrorMemoryAllocation;
  return cudaMalloc((void**)p, count * sizeof(T));
}

// float[9] per triangle -> 3 float4 (v0.xyz, id) (v1.xyz, 0) (v2.xyz, 0)
__global__ void k_pack(const float* __restrict__ raw, int n, float4* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float* p = raw + 9 * (size_t)i;
    out[3 * (size_t)i] = make_float4(p[0], p[1], p[2], __int_as_float(i));
    out[3 * (size_t)i + 1] = make_float4(p[3], p[4], p[5], 0.f);
    out[3 * (size_t)i + 2] = make_float4(p[6], p[7], p[8], 0.f);
  }
}

// The child references of every traversal node slot (width of them per
// slot, in slot order), for the host's count of the reachable nodes: 16 or
// 32 bytes per node instead of the whole 128- or 256-byte node.
__global__ void k_child_refs(const rt::WNode* __restrict__ w4, const rt::WNode8* __restrict__ w8, int64_t slots,
                             int4* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < slots;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (w8) {
      out[2 * k] = w8[k].child[0];
      out[2 * k + 1] = w8[k].child[1];
    } else {
      out[k] = w4[k].child;
    }
  }
}

void free_scene_buffers(rt_scene_s* s) {
  void* ptrs[] = {s->tri_in, s->idx[0], s->idx[1], s->rec[0], s->rec[1], s->node2, s->wide, s->link2, s->epoch,
                  s->tri_leaf, s->qa, s->qa_ready, s->top_task, s->top_done, s->top_bins, s->top_ccnt,
                  s->top_scnt, s->top_item, s->top_plan, s->top_ready, s->ctl, s->scratch.counter, s->scratch.queue, s->scratch.cand,
                  s->host_scr[0].counter, s->host_scr[0].queue, s->host_scr[0].cand,
                  s->host_scr[1].counter, s->host_scr[1].queue, s->host_scr[1].cand, s->reflect_blocks,
                  s->stage_rays[0], s->stage_rays[1], s->stage_hits[0], s->stage_hits[1], s->sel, s->sel_cnt,
                  s->qwide, s->wide8};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s->sel_host) cudaFreeHost(s->sel_host);
}

int sm_count_dev() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

int alloc_capacity(rt_scene_s* s, int64_t m);

// Size every per-triangle buffer for n triangles (grow only).  On failure
// the scene is left empty (no triangles, no buffers, not built), never half
// sized.
int ensure_capacity(rt_scene_s* s, int64_t n) {
  if (n <= s->cap_tri && s->ctl) return RT_OK;
  const int r = alloc_capacity(s, n < 1 ? 1 : n);
  if (r) {
    void* per_tri[] = {s->tri_in, s->idx[0], s->rec[0], s->rec[1], s->node2, s->link2, s->wide, s->tri_leaf,
                       s->qa, s->qa_ready, s->top_task, s->top_done, s->top_bins, s->top_ccnt, s->top_scnt,
                       s->top_item, s->top_plan, s->top_ready, s->sel, s->sel_cnt};
    for (void* p : per_tri)
      if (p) cudaFree(p);
    s->tri_in = s->tri_leaf = nullptr;
    s->idx[0] = nullptr;
    s->rec[0] = s->rec[1] = nullptr;
    s->node2 = nullptr;
    s->link2 = nullptr;
    s->wide = nullptr;
    s->qa = nullptr;
    s->qa_ready = nullptr;
    s->top_task = nullptr;
    s->top_done = nullptr;
    s->top_bins = s->top_ccnt = s->top_scnt = nullptr;
    s->top_item = nullptr;
    s->top_plan = nullptr;
    s->top_ready = nullptr;
    s->sel = s->sel_cnt = nullptr;
    s->cap_tri = 0;
    s->n_tri = 0;
    s->built = false;
    s->geom = rt::BuildGeom{};
  }
  return r;
}

// Buffers whose old contents must never match a new build's epoch start
// zeroed.
int alloc_capacity(rt_scene_s* s, int64_t m) {
  const rt::BuildGeom g = rt::build_geometry(m, sm_count_dev());
  RT_CUDA(dev_alloc(&s->tri_in, 3 * m), "alloc triangles");
  RT_CUDA(dev_alloc(&s->idx[0], m), "alloc index");
  for (int k = 0; k < 2; ++k) RT_CUDA(dev_alloc(&s->rec[k], 2 * m), "alloc build records");
  RT_CUDA(dev_alloc(&s->node2, m), "alloc binary nodes");
  RT_CUDA(dev_alloc(&s->link2, m), "alloc binary links");
  RT_CUDA(cudaMemset(s->link2, 0, sizeof(int2) * m), "clear binary links");
  RT_CUDA(dev_alloc(&s->wide, m + 1), "alloc wide nodes");
  RT_CUDA(dev_alloc(&s->tri_leaf, 3 * m), "alloc leaf triangles");
  RT_CUDA(dev_alloc(&s->qa, g.qa_cap), "alloc task queue");
  RT_CUDA(dev_alloc(&s->qa_ready, g.qa_cap), "alloc task queue");
  RT_CUDA(cudaMemset(s->qa_ready, 0, sizeof(int) * g.qa_cap), "clear task queue");
  RT_CUDA(dev_alloc(&s->top_task, (size_t)g.cap_t), "alloc top tasks");
  RT_CUDA(dev_alloc(&s->top_done, (size_t)g.cap_t), "alloc top tasks");
  RT_CUDA(dev_alloc(&s->top_bins, (size_t)g.cap_t * 3 * rt::kMaxBins * 13), "alloc top bins");
  RT_CUDA(dev_alloc(&s->top_ccnt, (size_t)g.cap_c * 3 * rt::kMaxBins), "alloc top counts");
  RT_CUDA(dev_alloc(&s->top_scnt, (size_t)g.cap_c * 3 * rt::kMaxBins), "alloc top counts");
  RT_CUDA(dev_alloc(&s->top_item, (size_t)g.cap_c), "alloc top items");
  RT_CUDA(dev_alloc(&s->top_plan, 2 * (size_t)g.cap_t), "alloc top plans");
  RT_CUDA(dev_alloc(&s->top_ready, (size_t)g.cap_c), "alloc top items");
  RT_CUDA(cudaMemset(s->top_ready, 0, sizeof(int) * g.cap_c), "clear top items");
  RT_CUDA(dev_alloc(&s->sel, m), "alloc range selection");
  RT_CUDA(dev_alloc(&s->sel_cnt, m / 256 + 2), "alloc range selection");
  if (!s->sel_host) RT_CUDA(cudaMallocHost((void**)&s->sel_host, sizeof(int)), "alloc pinned count");
  if (!s->epoch) {
    RT_CUDA(cudaMalloc((void**)&s->epoch, sizeof(int)), "alloc epoch");
    RT_CUDA(cudaMemset(s->epoch, 0, sizeof(int)), "clear epoch");
  }
  if (!s->ctl) RT_CUDA(cudaMalloc((void**)&s->ctl, sizeof(rt::BuildCtl)), "alloc control block");
  s->geom = g;
  s->cap_tri = m;
  return RT_OK;
}

int ensure_scratch(rt::TraceScratch& scr, int64_t n) {
  if (scr.counter && scr.cap >= n) return RT_OK;
  if (!scr.counter) RT_CUDA(cudaMalloc((void**)&scr.counter, 4 * sizeof(int)), "alloc trace counter");
  if (scr.queue) cudaFree(scr.queue);
  if (scr.cand) cudaFree(scr.cand);
  scr.queue = nullptr;
  scr.cand = nullptr;
  int64_t cap = n < 1024 ? 1024 : n;
  RT_CUDA(cudaMalloc((void**)&scr.queue, cap * sizeof(int)), "alloc re-test queue");
  RT_CUDA(cudaMalloc((void**)&scr.cand, cap * (rt::kTraceCand + 1) * sizeof(int)), "alloc re-test candidates");
  scr.cap = cap;
  return RT_OK;
}

int load_triangles(rt_scene_s* s, const float* tris, int64_t n, int is_dev, cudaStream_t st) {
  if (n > 0) {
    int r = ensure_capacity(s, n);
    if (r) return r;
    const float* raw = tris;
    if (!is_dev) {
      // stage the raw floats in the leaf buffer (48 B per triangle >= 36 B)
      RT_CUDA(cudaMemcpyAsync(s->tri_leaf, tris, (size_t)n * 9 * sizeof(float), cudaMemcpyHostToDevice, st),
              "copy triangles");
      raw = reinterpret_cast<const float*>(s->tri_leaf);
    }
    int g = (int)((n + 255) / 256);
    if (g > 4096) g = 4096;
    k_pack<<<g, 256, 0, st>>>(raw, (int)n, s->tri_in);
    rt::count_launches(1);
    RT_CUDA(cudaGetLastError(), "pack triangles");
  } else {
    int r = ensure_capacity(s, 1);
    if (r) return r;
  }
  s->n_tri = n;
  s->built = false;
  return RT_OK;
}

int check_params(const rt_build_params* p) {
  if (!p) return fail(RT_EINVAL, "params is NULL");
  if (!(p->alpha >= 0.f && p->alpha <= 1.f)) return fail(RT_EINVAL, "alpha must be in [0, 1]");
  if (!(p->t_i > 0.f)) return fail(RT_EINVAL, "t_i must be > 0");
  if (!(p->t_trav >= 0.f)) return fail(RT_EINVAL, "t_trav must be >= 0");
  for (int a = 0; a < 3; ++a)
    if (!(p->source[a] == p->source[a]) || p->source[a] > 3.0e38f || p->source[a] < -3.0e38f)
      return fail(RT_EINVAL, "source must be finite");
  if (p->max_leaf < 1 || p->max_leaf > rt::kMaxLeaf) return fail(RT_EINVAL, "max_leaf must be 1..15");
  if (p->bins < 4 || p->bins > rt::kMaxBins) return fail(RT_EINVAL, "bins must be 4..32");
  if (p->width != 4 && p->width != 8) return fail(RT_EINVAL, "width must be 4 or 8");
  if (p->dist_norm < 0 || p->dist_norm > 2) return fail(RT_EINVAL, "dist_norm must be 0, 1 or 2");
  if (!(p->range >= 0.f)) return fail(RT_EINVAL, "range must be >= 0");
  if (p->quantize != 0 && p->quantize != 1) return fail(RT_EINVAL, "quantize must be 0 or 1");
  if (p->quantize && p->width != 4) return fail(RT_EINVAL, "quantised nodes are 4-wide: quantize needs width 4");
  return RT_OK;
}

}  // namespace

namespace rt {
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace rt

extern "C" {

int rt_version(void) { return 100; }

uint64_t rt_launch_count(void) { return rt::g_launches.load(std::memory_order_relaxed); }

const char* rt_last_error(void) { return g_err; }

int rt_scene_upload(const float* tris, int64_t n_tri, int is_device_ptr, void* stream, rt_scene* out) {
  g_err[0] = 0;
  if (!out) return fail(RT_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_tri < 0 || n_tri > (int64_t(1) << 27)) return fail(RT_EINVAL, "n_tri out of range: %lld", (long long)n_tri);
  if (n_tri > 0 && !tris) return fail(RT_EINVAL, "tris is NULL");
  rt_scene_s* s = new (std::nothrow) rt_scene_s();
  if (!s) return fail(RT_ENOMEM, "host allocation failed");
  cudaGetDevice(&s->device);
  int r = load_triangles(s, tris, n_tri, is_device_ptr, (cudaStream_t)stream);
  if (r) {
    free_scene_buffers(s);
    delete s;
    return r;
  }
  cudaError_t e = cudaEventCreate(&s->ev_build0);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev_build1);
  if (e != cudaSuccess) {
    free_scene_buffers(s);
    delete s;
    return cuda_fail(e, "create events");
  }
  *out = s;
  return RT_OK;
}

int rt_scene_update(rt_scene s, const float* tris, int64_t n_tri, int is_device_ptr, void* stream) {
  g_err[0] = 0;
  if (!s) return fail(RT_EINVAL, "scene is NULL");
  if (n_tri < 0 || n_tri > (int64_t(1) << 27)) return fail(RT_EINVAL, "n_tri out of range");
  if (n_tri > 0 && !tris) return fail(RT_EINVAL, "tris is NULL");
  return load_triangles(s, tris, n_tri, is_device_ptr, (cudaStream_t)stream);
}

int rt_scene_destroy(rt_scene s) {
  g_err[0] = 0;
  if (!s) return fail(RT_EINVAL, "scene is NULL");
  cudaDeviceSynchronize();
  free_scene_buffers(s);
  for (int k = 0; k < 2; ++k)
    if (s->host_streams[k]) cudaStreamDestroy(s->host_streams[k]);
  if (s->host_ev) cudaEventDestroy(s->host_ev);
  if (s->ev_build0) cudaEventDestroy(s->ev_build0);
  if (s->ev_build1) cudaEventDestroy(s->ev_build1);
  delete s;
  return RT_OK;
}

int rt_bvh_build(rt_scene s, const rt_build_params* p, void* stream) {
  g_err[0] = 0;
  if (!s) return fail(RT_EINVAL, "scene is NULL");
  if (!s->tri_in || !s->ctl) return fail(RT_EINVAL, "scene has no buffers (a failed upload or update)");
  int r = check_params(p);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  const bool ranged = p->range > 0.f && p->range < 3.0e38f;
  if (capturing && ranged)
    return fail(RT_EINVAL, "a build with a range reads its triangle count back and cannot be captured");
  if (p->quantize && s->qwide_cap < s->cap_tri + 1) {  // the 64-byte nodes, on first use
    if (capturing) return fail(RT_EINVAL, "the first build with quantize = 1 allocates and cannot be captured");
    if (s->qwide) cudaFree(s->qwide);
    s->qwide = nullptr;
    s->qwide_cap = 0;
    RT_CUDA(dev_alloc(&s->qwide, s->cap_tri + 1), "alloc quantised nodes");
    s->qwide_cap = s->cap_tri + 1;
  }
  if (p->width == 8 && s->wide8_cap < s->cap_tri + 1) {  // the 8-wide nodes, on first use
    if (capturing) return fail(RT_EINVAL, "the first build with width = 8 allocates and cannot be captured");
    if (s->wide8) cudaFree(s->wide8);
    s->wide8 = nullptr;
    s->wide8_cap = 0;
    RT_CUDA(dev_alloc(&s->wide8, s->cap_tri + 1), "alloc 8-wide nodes");
    s->wide8_cap = s->cap_tri + 1;
  }
  s->q_built = false;
  if (!capturing) RT_CUDA(cudaEventRecord(s->ev_build0, st), "record event");
  RT_CUDA(rt::launch_build(s, *p, st), "launch build");
  s->q_built = p->quantize != 0;
  if (!capturing) RT_CUDA(cudaEventRecord(s->ev_build1, st), "record event");
  s->params = *p;
  s->built = true;
  return RT_OK;
}

int rt_debug_inject(int hook, int64_t value) {
  g_err[0] = 0;
  if (value < 0 || value > INT_MAX) return fail(RT_EINVAL, "value out of range");
  switch (hook) {
    case RT_DEBUG_SPIN_LIMIT:
      rt::g_spin_limit.store((int)value);
      return RT_OK;
    case RT_DEBUG_PHANTOM_TASK:
      rt::g_phantom_tasks.store((int)value);
      return RT_OK;
    case RT_DEBUG_PHANTOM_ITEM:
      rt::g_phantom_items.store((int)value);
      return RT_OK;
    case RT_DEBUG_FAIL_ALLOC:
      rt::g_fail_alloc.store(value);
      return RT_OK;
    default:
      return fail(RT_EINVAL, "unknown hook %d", hook);
  }
}

int rt_scene_set_split_events(rt_scene s, void* ev_begin, void* ev_end) {
  g_err[0] = 0;
  if (!s) return fail(RT_EINVAL, "scene is NULL");
  if ((ev_begin == nullptr) != (ev_end == nullptr)) return fail(RT_EINVAL, "give both events or neither");
  s->split_ev[0] = (cudaEvent_t)ev_begin;
  s->split_ev[1] = (cudaEvent_t)ev_end;
  return RT_OK;
}

static int rt_bvh_info_body(rt_scene s, void* stream, rt_bvh_info_t* info) {
  g_err[0] = 0;
  if (!s || !info) return fail(RT_EINVAL, "NULL argument");
  if (!s->built) return fail(RT_ENOTBUILT, "BVH not built");
  RT_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "synchronize");
  rt::BuildCtl c;
  RT_CUDA(cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost), "read control block");
  info->n_tri = s->n_tri;
  info->n_built = s->n_built;
  info->n_bvh2_internal = c.n_internal;
  info->n_leaves = c.n_leaves;
  info->depth2 = c.depth2;
  info->max_leaf_size = c.max_leaf_size;
  info->status = c.status;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, s->ev_build0, s->ev_build1) != cudaSuccess) {
    cudaGetLastError();
    ms = -1.f;
  }
  info->build_ms = ms;
  if (c.status == rt::kStQueueTimeout)
    return fail(RT_ETIMEOUT, "a work-queue wait of the build ran out (at %d)", c.status_where);
  if (c.status != 0) return fail(RT_EINTERNAL, "device status %d at %d", c.status, c.status_where);
  // traversal nodes reachable from the root, and their depth
  const int64_t slots = s->n_tri > 1 ? s->n_tri : 1;
  const int width = s->params.width == 8 ? 8 : 4;
  std::vector<int32_t> ch((size_t)slots * width);
  {
    // gathered on the device: only the references cross to the host
    int4* refs = nullptr;
    RT_CUDA(dev_alloc(&refs, slots * (width / 4)), "alloc child references");
    const int64_t blocks = (slots + 255) / 256;
    const int grid = (int)(blocks < 4 * (int64_t)sm_count_dev() ? blocks : 4 * (int64_t)sm_count_dev());
    cudaStream_t st = (cudaStream_t)stream;
    k_child_refs<<<grid, 256, 0, st>>>(width == 8 ? nullptr : s->wide, width == 8 ? s->wide8 : nullptr, slots, refs);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ch.data(), refs, sizeof(int32_t) * (size_t)slots * width, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(refs);
    RT_CUDA(e, "read child references");
  }
  std::vector<std::pair<int32_t, int32_t>> st{{c.wide_root, 1}};
  int64_t nw = 0;
  int32_t dw = 0;
  while (!st.empty()) {
    const auto it = st.back();
    st.pop_back();
    if (it.first < 0 || it.first >= slots || nw > slots) return fail(RT_EINTERNAL, "bad wide node %d", it.first);
    ++nw;
    if (it.second > dw) dw = it.second;
    for (int k = 0; k < width; ++k) {
      const int32_t c2 = ch[(size_t)it.first * width + k];
      if (c2 >= 0) st.push_back({c2, it.second + 1});
    }
  }
  info->n_wide = nw;
  info->depth_wide = dw;
  return RT_OK;
}

int rt_bvh_info(rt_scene s, void* stream, rt_bvh_info_t* info) {
  return rt::abi_guard([&] { return rt_bvh_info_body(s, stream, info); });
}

static int rt_bvh_export_body(rt_scene s, void* stream, int32_t* child, int64_t* leaf_first, int64_t* leaf_count,
                  int32_t* prims, float* boxes) {
  g_err[0] = 0;
  if (!s || !child || !leaf_first || !leaf_count || !prims) return fail(RT_EINVAL, "NULL argument");
  if (!s->built) return fail(RT_ENOTBUILT, "BVH not built");
  RT_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "synchronize");
  rt::BuildCtl c;
  RT_CUDA(cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost), "read control block");
  const int64_t n = s->n_built;
  for (int64_t k = n; k < s->n_tri; ++k) prims[k] = -1;  // triangles outside a range build's tree
  std::vector<rt::Node2> nodes((size_t)(n > 0 ? n : 1));
  std::vector<int32_t> idx((size_t)(n > 0 ? n : 1));
  if (n > 0) {
    RT_CUDA(cudaMemcpy(nodes.data(), s->node2, sizeof(rt::Node2) * n, cudaMemcpyDeviceToHost), "read nodes");
    RT_CUDA(cudaMemcpy(idx.data(), s->idx[0], sizeof(int32_t) * n, cudaMemcpyDeviceToHost), "read index");
  }
  for (int64_t k = 0; k < n; ++k) prims[k] = idx[k];
  // renumber: internal nodes in depth-first order, leaves in order of discovery
  int64_t ni = 0, nl = 0;
  auto add_leaf = [&](int32_t ref) {
    leaf_first[nl] = rt::leaf_first(ref);
    leaf_count[nl] = rt::leaf_count(ref);
    return -1 - (int32_t)(nl++);
  };
  if (c.root_ref < 0) {
    if (c.root_ref != INT_MIN) add_leaf(c.root_ref);
    return RT_OK;
  }
  struct Item {
    int32_t id;
    int64_t slot;  // where to write our neutral id (-1: root)
  };
  std::vector<Item> st{{c.root_ref, -1}};
  while (!st.empty()) {
    Item it = st.back();
    st.pop_back();
    if (it.id < 0 || it.id >= n) return fail(RT_EINTERNAL, "bad node id %d", it.id);
    int64_t me = ni++;
    if (ni > c.n_internal) return fail(RT_EINTERNAL, "more internal nodes than counted");
    if (it.slot >= 0) child[it.slot] = (int32_t)me;
    const rt::Node2& nd = nodes[it.id];
    int32_t refs[2];
    memcpy(&refs[0], &nd.a_lo.w, 4);
    memcpy(&refs[1], &nd.b_lo.w, 4);
    if (boxes) {
      float b[12] = {nd.a_lo.x, nd.a_lo.y, nd.a_lo.z, nd.a_hi.x, nd.a_hi.y, nd.a_hi.z,
                     nd.b_lo.x, nd.b_lo.y, nd.b_lo.z, nd.b_hi.x, nd.b_hi.y, nd.b_hi.z};
      memcpy(boxes + 12 * me, b, sizeof(b));
    }
    for (int k = 1; k >= 0; --k) {
      if (refs[k] >= 0 && refs[k] != INT_MAX)
        st.push_back({refs[k], 2 * me + k});
      else if (refs[k] == INT_MAX)
        return fail(RT_EINTERNAL, "child never written");
      else
        child[2 * me + k] = add_leaf(refs[k]);
    }
  }
  return RT_OK;
}

int rt_bvh_export(rt_scene s, void* stream, int32_t* child, int64_t* leaf_first, int64_t* leaf_count,
                  int32_t* prims, float* boxes) {
  return rt::abi_guard([&] { return rt_bvh_export_body(s, stream, child, leaf_first, leaf_count, prims, boxes); });
}

static int trace_common(rt_scene s, const rt_ray* rays, int64_t n, rt_hit* hits, uint8_t* occl,
                        const rt_trace_params* params, void* stream) {
  if (!s) return fail(RT_EINVAL, "scene is NULL");
  if (n < 0 || n > INT_MAX) return fail(RT_EINVAL, "n out of range");
  if (n > 0 && (!rays || (!hits && !occl))) return fail(RT_EINVAL, "NULL buffer");
  if (((uintptr_t)rays & 15) || ((uintptr_t)hits & 15)) return fail(RT_EINVAL, "rays/hits must be 16-byte aligned");
  if (params && params->block != 0 && params->block != 64 && params->block != 128 && params->block != 256)
    return fail(RT_EINVAL, "block must be 0, 64, 128 or 256");
  if (params && ((params->stack != 0 && params->stack != 16 && params->stack != 32 && params->stack != 64)))
    return fail(RT_EINVAL, "stack must be 0, 16, 32 or 64");
  if (params && (params->flags & RT_QUANTIZED_NODES) && !s->q_built)
    return fail(RT_EINVAL, "RT_QUANTIZED_NODES needs a build with quantize = 1");
  if (!s->built) return fail(RT_ENOTBUILT, "BVH not built");
  int r = ensure_scratch(s->scratch, n);
  if (r) return r;
  RT_CUDA(rt::launch_trace(s, rays, n, hits, occl, params, s->scratch, (cudaStream_t)stream), "launch trace");
  return RT_OK;
}

int rt_trace_closest(rt_scene s, const rt_ray* rays_dev, int64_t n, rt_hit* hits_dev,
                     const rt_trace_params* params, void* stream) {
  g_err[0] = 0;
  if (n > 0 && !hits_dev) return fail(RT_EINVAL, "hits is NULL");
  return trace_common(s, rays_dev, n, hits_dev, nullptr, params, stream);
}

int rt_trace_any(rt_scene s, const rt_ray* rays_dev, int64_t n, uint8_t* occluded_dev,
                 const rt_trace_params* params, void* stream) {
  g_err[0] = 0;
  if (n > 0 && !occluded_dev) return fail(RT_EINVAL, "occluded is NULL");
  return trace_common(s, rays_dev, n, nullptr, occluded_dev, params, stream);
}

int64_t rt_ray_count(int kind, int64_t param) {
  if (kind == RT_RAYS_FIBONACCI) return param >= 0 ? param : -1;
  if (kind == RT_RAYS_ICOSPHERE) {
    if (param < 0 || param > 12) return -1;
    const int64_t f = int64_t(1) << param;
    return 10 * f * f + 2;
  }
  return -1;
}

int64_t rt_launch_index(int kind, int64_t param, int64_t slot) {
  const int64_t n = rt_ray_count(kind, param);
  if (n < 0 || slot < 0 || slot >= n) return -1;
  if (kind == RT_RAYS_ICOSPHERE) {
    const long long f = 1ll << param;
    return rt::ico_index(rt::ico_slot_point(slot, f), f);
  }
  long long w = 1, c = 1;
  rt::fib_launch_order(n, &w, &c);
  return rt::fib_slot(slot, n, w, c);
}

int rt_gen_rays(int kind, const float* origin, int64_t param, float tmin, float tmax, rt_ray* rays_dev,
                int64_t capacity, void* stream) {
  g_err[0] = 0;
  const int64_t n = rt_ray_count(kind, param);
  if (n < 0) return fail(RT_EINVAL, "bad launch kind or param");
  if (n > INT_MAX) return fail(RT_EINVAL, "too many rays");
  if (!origin || (n > 0 && !rays_dev)) return fail(RT_EINVAL, "NULL argument");
  if (capacity < n) return fail(RT_EINVAL, "capacity %lld < %lld rays", (long long)capacity, (long long)n);
  if ((uintptr_t)rays_dev & 15) return fail(RT_EINVAL, "rays must be 16-byte aligned");
  RT_CUDA(rt::launch_gen_rays(kind, origin, kind == RT_RAYS_FIBONACCI ? n : param, tmin, tmax, rays_dev, n,
                              (cudaStream_t)stream),
          "generate rays");
  return RT_OK;
}

int rt_reflect(rt_scene s, const rt_ray* rays_dev, const rt_hit* hits_dev, int64_t n, rt_ray* out_rays_dev,
               int32_t* out_skip_dev, int32_t* out_src_dev, int32_t* out_count_dev, void* stream) {
  g_err[0] = 0;
  if (!s) return fail(RT_EINVAL, "scene is NULL");
  if (n < 0 || n > INT_MAX) return fail(RT_EINVAL, "n out of range");
  if (!out_count_dev || (n > 0 && (!rays_dev || !hits_dev || !out_rays_dev || !out_skip_dev)))
    return fail(RT_EINVAL, "NULL buffer");
  if (((uintptr_t)rays_dev & 15) || ((uintptr_t)hits_dev & 15) || ((uintptr_t)out_rays_dev & 15))
    return fail(RT_EINVAL, "rays/hits must be 16-byte aligned");
  const int64_t nb = (n + 255) / 256 + 1;
  if (s->reflect_blocks_cap < nb) {
    RT_CUDA(dev_alloc(&s->reflect_blocks, nb), "alloc reflect scratch");
    s->reflect_blocks_cap = nb;
  }
  RT_CUDA(rt::launch_reflect(s, rays_dev, hits_dev, n, nullptr, out_rays_dev, out_skip_dev, out_src_dev,
                             out_count_dev, s->reflect_blocks, n, (cudaStream_t)stream),
          "reflect");
  return RT_OK;
}

int rt_trace_closest_host(rt_scene s, const rt_ray* rays_host, int64_t n, rt_hit* hits_host,
                          const rt_trace_params* params, void* stream) {
  g_err[0] = 0;
  if (!s) return fail(RT_EINVAL, "scene is NULL");
  if (n < 0) return fail(RT_EINVAL, "n out of range");
  if (n > 0 && (!rays_host || !hits_host)) return fail(RT_EINVAL, "NULL buffer");
  if (!s->built) return fail(RT_ENOTBUILT, "BVH not built");
  if (params && (params->skip_tri_dev || params->stats_dev))
    return fail(RT_EINVAL, "per-ray device arrays are not supported with host buffers");
  if (params && params->block != 0 && params->block != 64 && params->block != 128 && params->block != 256)
    return fail(RT_EINVAL, "block must be 0, 64, 128 or 256");
  if (params && ((params->stack != 0 && params->stack != 16 && params->stack != 32 && params->stack != 64)))
    return fail(RT_EINVAL, "stack must be 0, 16, 32 or 64");
  if (params && (params->flags & RT_QUANTIZED_NODES) && !s->q_built)
    return fail(RT_EINVAL, "RT_QUANTIZED_NODES needs a build with quantize = 1");
  if (n == 0) return RT_OK;
  // two chunks when they fit in 2 x 2^20 rays (both ray copies can then go
  // under whatever the caller's stream is still doing), else chunks of 2^20
  int64_t chunk = (n + 1) / 2;
  if (chunk > (int64_t(1) << 20)) chunk = int64_t(1) << 20;
  if (s->stage_cap < chunk) {
    for (int k = 0; k < 2; ++k) {
      RT_CUDA(dev_alloc(&s->stage_rays[k], chunk), "alloc staging");
      RT_CUDA(dev_alloc(&s->stage_hits[k], chunk), "alloc staging");
    }
    s->stage_cap = chunk;
  }
  for (int k = 0; k < 2; ++k) {
    if (!s->host_streams[k]) RT_CUDA(cudaStreamCreateWithFlags(&s->host_streams[k], cudaStreamNonBlocking), "create stream");
    int r = ensure_scratch(s->host_scr[k], chunk);
    if (r) return r;
  }
  // the ray copies start at once (they read only the caller's host buffer);
  // the traces wait for everything already queued on the caller's stream
  // (typically the build)
  if (!s->host_ev) RT_CUDA(cudaEventCreateWithFlags(&s->host_ev, cudaEventDisableTiming), "create event");
  cudaEvent_t ev = s->host_ev;
  RT_CUDA(cudaEventRecord(ev, (cudaStream_t)stream), "record event");
  rt_trace_params tp{};
  if (params) {  // n_flagged_dev counts one call of the device path: not written here
    tp.flags = params->flags;
    tp.block = params->block;
    tp.stack = params->stack;
  }
  // page-locked hits the device can address: the walk and the float64 pass
  // (which only write hit records) store into them directly, so no copy
  // back waits for the last chunk's walk
  rt_hit* hits_mapped = nullptr;
  if (((uintptr_t)hits_host & 15) == 0) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, hits_host) == cudaSuccess) {
      if (pa.type == cudaMemoryTypeHost && pa.devicePointer) hits_mapped = static_cast<rt_hit*>(pa.devicePointer);
    } else {
      cudaGetLastError();  // not a pointer CUDA knows: stage as for pageable memory
    }
  }
  int rc = RT_OK;
  for (int64_t off = 0, c = 0; off < n; off += chunk, ++c) {
    const int k = (int)(c & 1);
    const int64_t cnt = (n - off) < chunk ? (n - off) : chunk;
    cudaStream_t st = s->host_streams[k];
    cudaError_t e = cudaMemcpyAsync(s->stage_rays[k], rays_host + off, cnt * sizeof(rt_ray),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && c < 2) e = cudaStreamWaitEvent(st, ev, 0);
    rt_hit* out = hits_mapped ? hits_mapped + off : s->stage_hits[k];
    if (e == cudaSuccess) e = rt::launch_trace(s, s->stage_rays[k], cnt, out, nullptr, &tp, s->host_scr[k], st);
    if (e == cudaSuccess && !hits_mapped)
      e = cudaMemcpyAsync(hits_host + off, s->stage_hits[k], cnt * sizeof(rt_hit), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "host pipeline");
      break;
    }
  }
  for (int k = 0; k < 2; ++k) {
    cudaError_t e = cudaStreamSynchronize(s->host_streams[k]);
    if (e != cudaSuccess && rc == RT_OK) rc = cuda_fail(e, "synchronize pipeline");
  }
  return rc;
}

}  // extern "C"
