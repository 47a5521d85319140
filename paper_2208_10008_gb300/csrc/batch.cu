// Batched multi-bounce tracing: many transmitters, uneven ray counts,
// reflection orders, and transmitter-receiver visibility in one device
// pipeline (Sec. III: launch -> trace -> bounce until the order limit).
//
// One rt_batch owns every buffer the pipeline needs (sized at creation from
// the transmitters' ray counts), so a run allocates nothing and never waits
// on the host.  A run is two launches: one kernel writes every
// transmitter's launch, and one cooperative, persistent kernel traces every
// reflection order and the visibility segments, its CTAs stepping through
// the orders together (walk, float64 pass, stable compaction into the next
// order) with the counts on the device.  The first run executes directly;
// the second captures the run into a CUDA graph, which every later run
// replays.  With reception on, every order's segments are then tested
// against the receivers' spheres (Sec. III.C, Eq. 4), each ray with the
// angular spacing of its own transmitter's launch.
#include <cuda_runtime.h>

#include <array>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "rt_internal.cuh"

struct rt_batch_s {
  rt_scene scene = nullptr;
  int n_tx = 0, kind = 0, max_order = 0, n_rx = 0;
  float tmax = 0.f;
  bool use_graph = true;
  int ray_tile = 0;  // rays per CTA of every walk (0 = default)
  std::vector<float> tx;
  std::vector<long long> param, count, offset;
  long long n0 = 0, n_seg = 0;
  rt_ray* rays[RT_BATCH_MAX_ORDER + 1] = {};
  rt_hit* hits[RT_BATCH_MAX_ORDER + 1] = {};
  int* skip[RT_BATCH_MAX_ORDER + 1] = {};
  int* src[RT_BATCH_MAX_ORDER + 1] = {};
  int* counts = nullptr;  // device: rays of order k at counts[k] (k >= 1)
  int* blocks = nullptr;  // reflect block counts
  rt_ray* seg = nullptr;  // visibility segments, transmitter-major
  uint8_t* occl = nullptr;
  rt::TraceScratch scr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::array<uintptr_t, 10> graph_scene{};  // scene state the graph was captured with
  int runs = 0;
  long long graph_kernels = 0;  // kernels in the captured graph
  // reception (Eq. 4)
  bool receive = false;
  int max_rx = 0;
  float dmax = 0.f;                             // largest transmitter delta
  rt_rxset rxset = nullptr;
  float* delta[RT_BATCH_MAX_ORDER + 1] = {};    // per ray: its transmitter's delta
  rt_rx_record* rec[RT_BATCH_MAX_ORDER + 1] = {};
  int* rx_count = nullptr;                      // device: pairs of order k at rx_count[k]
  long long* tx_off = nullptr;                  // device: first order-0 ray of each transmitter (n_tx + 1)
  float* tx_delta = nullptr;                    // device: each transmitter's delta
  // the one-launch pipeline
  float* tx_dev = nullptr;                      // device: transmitter positions
  long long* param_dev = nullptr;               // device: launch parameters
  int* chunk = nullptr;                         // per 32-ray chunk of order-k rays
  int* cta_total = nullptr;
  int cta_cap = 0;
  unsigned* bar = nullptr;                      // grid barrier words + status
  int* take = nullptr;                          // rays handed out per walk phase
};

namespace rt {
int set_error(int code, const char* msg);
}

namespace {

// Order-0 rays of transmitter t occupy [off[t], off[t + 1]): each gets
// that transmitter's delta.
__global__ void k_delta_fill(const long long* __restrict__ off, const float* __restrict__ dtx, int n_tx, int n,
                             float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = n_tx - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  out[i] = dtx[lo];
}

// What a captured pipeline takes from the scene as launch arguments: the
// arrays the walk and the bounce read and the size of the current tree.  A
// re-upload that grows the scene, the first quantised build or a rebuild
// over another range changes it; the graph is then captured again.
std::array<uintptr_t, 10> scene_key(const rt_scene_s* s) {
  return {(uintptr_t)s->tri_in, (uintptr_t)s->node2,  (uintptr_t)s->wide, (uintptr_t)s->qwide,
          (uintptr_t)s->link2,  (uintptr_t)s->tri_leaf, (uintptr_t)s->ctl, (uintptr_t)s->n_built,
          (uintptr_t)s->wide8,  (uintptr_t)s->params.width};
}

void drop_graph(rt_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void free_batch(rt_batch_s* b) {
  if (b->rxset) rt_rxset_destroy(b->rxset);
  for (int k = 0; k <= RT_BATCH_MAX_ORDER; ++k) {
    if (b->delta[k]) cudaFree(b->delta[k]);
    if (b->rec[k]) cudaFree(b->rec[k]);
  }
  if (b->rx_count) cudaFree(b->rx_count);
  if (b->tx_off) cudaFree(b->tx_off);
  if (b->tx_delta) cudaFree(b->tx_delta);
  if (b->tx_dev) cudaFree(b->tx_dev);
  if (b->param_dev) cudaFree(b->param_dev);
  if (b->chunk) cudaFree(b->chunk);
  if (b->cta_total) cudaFree(b->cta_total);
  if (b->bar) cudaFree(b->bar);
  if (b->take) cudaFree(b->take);
  for (int k = 0; k <= RT_BATCH_MAX_ORDER; ++k) {
    if (b->rays[k]) cudaFree(b->rays[k]);
    if (b->hits[k]) cudaFree(b->hits[k]);
    if (b->skip[k]) cudaFree(b->skip[k]);
    if (b->src[k]) cudaFree(b->src[k]);
  }
  void* p[] = {b->counts, b->blocks, b->seg, b->occl, b->scr.counter, b->scr.queue, b->scr.cand};
  for (void* q : p)
    if (q) cudaFree(q);
  drop_graph(b);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->st) cudaStreamDestroy(b->st);
}

constexpr long long kBarrierTimeoutNs = 10ll * 1000 * 1000 * 1000;  // 10 s per barrier

cudaError_t enqueue(rt_batch_s* b) {
  cudaError_t e;
  cudaStream_t st = b->st;
  if ((e = rt::launch_gen_batch(b->kind, b->tx_dev, b->tx_off, b->param_dev, b->n_tx, b->n0, 0.f, b->tmax,
                                b->rays[0], st)))
    return e;
  rt::BatchLaunch L;
  L.max_order = b->max_order;
  L.n0 = b->n0;
  L.n_seg = b->n_seg;
  for (int k = 0; k <= RT_BATCH_MAX_ORDER; ++k) {
    L.rays[k] = b->rays[k];
    L.hits[k] = b->hits[k];
    L.skip[k] = b->skip[k];
    L.src[k] = b->src[k];
  }
  L.counts = b->counts;
  L.chunk = b->chunk;
  L.cta_total = b->cta_total;
  L.cta_cap = b->cta_cap;
  L.seg = b->seg;
  L.occl = b->occl;
  L.bar = b->bar;
  L.status = reinterpret_cast<int*>(b->bar + 2);
  L.take = b->take;
  L.timeout_ns = kBarrierTimeoutNs;
  L.scr = &b->scr;
  L.receive = b->receive ? 1 : 0;
  for (int k = 0; k <= RT_BATCH_MAX_ORDER; ++k) L.delta[k] = b->delta[k];
  if ((e = rt::launch_batch_persistent(b->scene, L, st))) return e;
  // the receiving spheres of every order (Sec. III.C, Eq. 4), each ray with
  // its own transmitter's delta; one launch per order
  if (b->receive)
    for (int k = 0; k <= b->max_order; ++k) {
      rt_receive_params p{};
      p.delta = b->dmax;
      p.range0 = b->tmax;
      p.max_records = b->max_rx;
      p.delta_ray_dev = b->delta[k];
      if (rt_receive(b->rxset, b->rays[k], b->hits[k], b->n0, k ? b->counts + k : nullptr, &p, b->rec[k],
                     b->rx_count + k, st) != RT_OK)
        return cudaErrorInvalidValue;
    }
  return cudaSuccess;
}

template <class T>
cudaError_t alloc(T** p, long long n) {
  return cudaMalloc((void**)p, (size_t)(n < 1 ? 1 : n) * sizeof(T));
}

}  // namespace

extern "C" {

static int rt_batch_create_body(rt_scene scene, const rt_batch_desc* d, rt_batch* out) {
  if (!out || !scene || !d) return rt::set_error(RT_EINVAL, "NULL argument");
  *out = nullptr;
  if (d->n_tx < 1 || !d->tx_pos || !d->tx_param) return rt::set_error(RT_EINVAL, "need at least one transmitter");
  if (d->dir_kind != RT_RAYS_FIBONACCI && d->dir_kind != RT_RAYS_ICOSPHERE)
    return rt::set_error(RT_EINVAL, "bad dir_kind");
  if (d->max_order < 0 || d->max_order > RT_BATCH_MAX_ORDER) return rt::set_error(RT_EINVAL, "max_order out of range");
  if (!(d->tmax > 0.f)) return rt::set_error(RT_EINVAL, "tmax must be > 0");
  if (d->n_rx < 0 || (d->n_rx > 0 && !d->rx_pos)) return rt::set_error(RT_EINVAL, "bad receivers");
  if (d->receive && (d->n_rx < 1 || d->max_rx_records < 1))
    return rt::set_error(RT_EINVAL, "reception needs receivers and max_rx_records >= 1");
  rt_batch_s* b = new (std::nothrow) rt_batch_s();
  if (!b) return rt::set_error(RT_ENOMEM, "host allocation failed");
  struct Undo {  // frees the half-made batch on every early return or exception
    rt_batch_s* b;
    ~Undo() {
      if (b) {
        free_batch(b);
        delete b;
      }
    }
  } undo{b};
  b->scene = scene;
  b->n_tx = d->n_tx;
  b->kind = d->dir_kind;
  b->max_order = d->max_order;
  b->n_rx = d->n_rx;
  b->tmax = d->tmax;
  b->use_graph = d->use_graph != 0;
  if (d->ray_tile != 0 && d->ray_tile != 64 && d->ray_tile != 128 && d->ray_tile != 256)
    return rt::set_error(RT_EINVAL, "ray_tile must be 0, 64, 128 or 256");
  b->ray_tile = d->ray_tile;
  b->tx.assign(d->tx_pos, d->tx_pos + 3 * d->n_tx);
  long long total = 0;
  for (int t = 0; t < d->n_tx; ++t) {
    const long long c = rt_ray_count(d->dir_kind, d->tx_param[t]);
    if (c < 0) return rt::set_error(RT_EINVAL, "bad ray count for a transmitter");
    b->param.push_back(d->tx_param[t]);
    b->count.push_back(c);
    b->offset.push_back(total);
    total += c;
  }
  if (total < 1 || total > INT_MAX) return rt::set_error(RT_EINVAL, "total ray count out of range");
  b->n0 = total;
  b->n_seg = (long long)d->n_tx * d->n_rx;
  // every upload and initialisation below is ordered on the batch's own
  // stream: creating a batch never waits for other streams' work
  cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  for (int k = 0; k <= b->max_order && e == cudaSuccess; ++k) {
    if (e == cudaSuccess) e = alloc(&b->rays[k], total);
    if (e == cudaSuccess) e = alloc(&b->hits[k], total);
    if (e == cudaSuccess && k > 0) e = alloc(&b->skip[k], total);
    if (e == cudaSuccess && k > 0) e = alloc(&b->src[k], total);
  }
  if (e == cudaSuccess) e = alloc(&b->counts, RT_BATCH_MAX_ORDER + 1);
  if (e == cudaSuccess) e = alloc(&b->chunk, total / 32 + 2);
  b->cta_cap = rt::persistent_batch_ctas();
  if (e == cudaSuccess) e = alloc(&b->cta_total, b->cta_cap);
  if (e == cudaSuccess) e = alloc(&b->bar, 4);
  if (e == cudaSuccess) e = alloc(&b->take, RT_BATCH_MAX_ORDER + 2);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->bar, 0, 4 * sizeof(unsigned), b->st);
  if (e == cudaSuccess) e = alloc(&b->tx_dev, 3 * b->n_tx);
  if (e == cudaSuccess) e = alloc(&b->param_dev, b->n_tx);
  if (e == cudaSuccess) e = alloc(&b->tx_off, b->n_tx + 1);
  if (e == cudaSuccess) {
    std::vector<long long> off(b->offset);
    off.push_back(total);
    // the generator's parameters: the level, or a Fibonacci launch's band
    // width and step packed as w << 32 | c
    std::vector<long long> gp(b->param);
    if (b->kind == RT_RAYS_FIBONACCI)
      for (int t = 0; t < b->n_tx; ++t) {
        long long w = 1, c = 1;
        rt::fib_launch_order(b->count[t], &w, &c);
        gp[t] = (long long)(((unsigned long long)w << 32) | (unsigned long long)c);
      }
    e = cudaMemcpyAsync(b->tx_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->tx_dev, b->tx.data(), 3 * b->n_tx * sizeof(float), cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->param_dev, gp.data(), b->n_tx * sizeof(long long), cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);  // off and gp are host temporaries
  }
  if (e == cudaSuccess) e = alloc(&b->blocks, total / 256 + 2);
  const long long qcap = total > b->n_seg ? total : b->n_seg;
  if (e == cudaSuccess) e = alloc(&b->scr.counter, 4);
  if (e == cudaSuccess) e = alloc(&b->scr.queue, qcap);
  if (e == cudaSuccess) e = alloc(&b->scr.cand, qcap * (rt::kTraceCand + 1));
  b->scr.cap = qcap;
  if (e == cudaSuccess && b->n_seg > 0) {
    e = alloc(&b->seg, b->n_seg);
    if (e == cudaSuccess) e = alloc(&b->occl, b->n_seg);
    if (e == cudaSuccess) {
      std::vector<rt_ray> h((size_t)b->n_seg);
      for (int t = 0; t < b->n_tx; ++t)
        for (int r = 0; r < b->n_rx; ++r) {
          rt_ray& s = h[(size_t)t * b->n_rx + r];
          const float* a = &b->tx[3 * t];
          const float* c = d->rx_pos + 3 * r;
          s = rt_ray{a[0], a[1], a[2], 0.f, c[0] - a[0], c[1] - a[1], c[2] - a[2], 1.f};
        }
      e = cudaMemcpyAsync(b->seg, h.data(), h.size() * sizeof(rt_ray), cudaMemcpyHostToDevice, b->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);  // h is a host temporary
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b->counts, 0, (RT_BATCH_MAX_ORDER + 1) * sizeof(int), b->st);
  if (e == cudaSuccess && d->receive) {
    // each transmitter's delta: the caller's, or the spacing of its launch
    std::vector<float> dtx(b->n_tx);
    for (int t = 0; t < b->n_tx; ++t) {
      double v = d->rx_delta ? (double)d->rx_delta[t]
                             : (b->kind == RT_RAYS_ICOSPHERE ? std::atan(2.0) / std::ldexp(1.0, (int)b->param[t])
                                                              : std::sqrt(4.0 * M_PI / (double)b->count[t]));
      if (!(v > 0.0) || !std::isfinite(v)) return rt::set_error(RT_EINVAL, "bad delta for a transmitter");
      dtx[t] = (float)v;
      b->dmax = std::max(b->dmax, dtx[t]);
    }
    b->receive = true;
    b->max_rx = d->max_rx_records;
    const int rc = rt_rxset_create(d->rx_pos, d->n_rx, (float)(b->tmax * (double)b->dmax / std::sqrt(3.0)) * 1.0001f,
                                   &b->rxset);
    if (rc != RT_OK) return rc;  // the set's own message stays in rt_last_error

    for (int k = 0; k <= b->max_order && e == cudaSuccess; ++k) {
      e = alloc(&b->delta[k], total);
      if (e == cudaSuccess) e = alloc(&b->rec[k], b->max_rx);
    }
    if (e == cudaSuccess) e = alloc(&b->rx_count, RT_BATCH_MAX_ORDER + 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->rx_count, 0, (RT_BATCH_MAX_ORDER + 1) * sizeof(int), b->st);
    if (e == cudaSuccess) e = alloc(&b->tx_delta, b->n_tx);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->tx_delta, dtx.data(), b->n_tx * sizeof(float), cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) {
      k_delta_fill<<<(int)((total + 255) / 256), 256, 0, b->st>>>(b->tx_off, b->tx_delta, b->n_tx, (int)total,
                                                                  b->delta[0]);
      rt::count_launches(1);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);  // dtx is a host temporary
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return rt::set_error(e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA, cudaGetErrorString(e));
  }
  undo.b = nullptr;
  *out = b;
  return RT_OK;
}

int rt_batch_create(rt_scene scene, const rt_batch_desc* d, rt_batch* out) {
  return rt::abi_guard([&] { return rt_batch_create_body(scene, d, out); });
}

int rt_batch_run(rt_batch b, void* stream) {
  if (!b) return rt::set_error(RT_EINVAL, "batch is NULL");
  if (!b->scene->built) return rt::set_error(RT_ENOTBUILT, "BVH not built");
  cudaError_t e = cudaEventRecord(b->ev_in, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->ev_in, 0);
  if (e == cudaSuccess) {
    if (!b->use_graph || b->runs == 0) {
      e = enqueue(b);  // the first run also initialises lazily loaded tables
    } else {
      if (b->exec && b->graph_scene != scene_key(b->scene)) {
        e = cudaStreamSynchronize(b->st);  // the last replay may still run
        drop_graph(b);
      }
      if (e == cudaSuccess && !b->exec) {
        e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          const unsigned long long c0 = rt_launch_count();
          cudaError_t e2 = enqueue(b);
          b->graph_kernels = (long long)(rt_launch_count() - c0);
          rt::count_launches(-(int)b->graph_kernels);  // captured, not launched
          e = cudaStreamEndCapture(b->st, &b->graph);
          if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e == cudaSuccess) {
          b->graph_scene = scene_key(b->scene);
        } else {
          // no graph of this pipeline on this device (a cooperative launch
          // that cannot be captured): run it directly from now on; a run is
          // two launches either way
          drop_graph(b);
          cudaGetLastError();
          b->use_graph = false;
          e = enqueue(b);
        }
      }
      if (e == cudaSuccess && b->exec) {
        e = cudaGraphLaunch(b->exec, b->st);
        rt::count_launches((int)b->graph_kernels);
      }
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, b->ev_out, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return rt::set_error(RT_ECUDA, cudaGetErrorString(e));
  }
  ++b->runs;
  return RT_OK;
}

static int rt_batch_stats_get_body(rt_batch b, void* stream, rt_batch_stats* s) {
  if (!b || !s) return rt::set_error(RT_EINVAL, "NULL argument");
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess || cudaStreamSynchronize(b->st) != cudaSuccess)
    return rt::set_error(RT_ECUDA, "synchronize");
  int c[RT_BATCH_MAX_ORDER + 1];
  if (cudaMemcpy(c, b->counts, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
    return rt::set_error(RT_ECUDA, "read counts");
  memset(s, 0, sizeof(*s));
  s->n_orders = b->max_order + 1;
  s->rays[0] = b->n0;
  s->total_rays = b->n0 + b->n_seg;
  for (int k = 1; k <= b->max_order; ++k) {
    s->rays[k] = c[k];
    s->total_rays += c[k];
  }
  if (b->n_seg > 0) {
    std::vector<uint8_t> o((size_t)b->n_seg);
    if (cudaMemcpy(o.data(), b->occl, o.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return rt::set_error(RT_ECUDA, "read visibility");
    for (uint8_t v : o) s->visible += v == 0;
  }
  if (b->receive) {
    int rc[RT_BATCH_MAX_ORDER + 1];
    if (cudaMemcpy(rc, b->rx_count, sizeof(rc), cudaMemcpyDeviceToHost) != cudaSuccess)
      return rt::set_error(RT_ECUDA, "read reception counts");
    for (int k = 0; k <= b->max_order; ++k) s->received[k] = rc[k];
  }
  int fl = 0;
  cudaMemcpy(&fl, b->scr.counter, sizeof(int), cudaMemcpyDeviceToHost);
  s->flagged = fl;
  s->segments = b->n_seg;
  unsigned w[4] = {0, 0, 0, 0};
  if (cudaMemcpy(w, b->bar, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess)
    return rt::set_error(RT_ECUDA, "read batch status");
  if (w[2] != 0) return rt::set_error(RT_ETIMEOUT, "a grid barrier of the batch kernel ran out of time");
  return RT_OK;
}

int rt_batch_stats_get(rt_batch b, void* stream, rt_batch_stats* s) {
  return rt::abi_guard([&] { return rt_batch_stats_get_body(b, stream, s); });
}

int rt_batch_order(rt_batch b, int order, const rt_ray** rays, const rt_hit** hits, const int32_t** src,
                   const int32_t** count) {
  if (!b || order < 0 || order > b->max_order) return rt::set_error(RT_EINVAL, "bad batch or order");
  if (rays) *rays = b->rays[order];
  if (hits) *hits = b->hits[order];
  if (src) *src = order ? b->src[order] : nullptr;
  if (count) *count = order ? b->counts + order : nullptr;
  return RT_OK;
}

int rt_batch_received(rt_batch b, int order, const rt_rx_record** records, const int32_t** count) {
  if (!b || order < 0 || order > b->max_order) return rt::set_error(RT_EINVAL, "bad batch or order");
  if (!b->receive) return rt::set_error(RT_EINVAL, "the batch was created without reception");
  if (records) *records = b->rec[order];
  if (count) *count = b->rx_count + order;
  return RT_OK;
}

int rt_batch_visibility(rt_batch b, const uint8_t** occluded) {
  if (!b || !occluded) return rt::set_error(RT_EINVAL, "NULL argument");
  *occluded = b->occl;
  return RT_OK;
}

int rt_batch_destroy(rt_batch b) {
  if (!b) return rt::set_error(RT_EINVAL, "batch is NULL");
  cudaStreamSynchronize(b->st);
  free_batch(b);
  delete b;
  return RT_OK;
}

}  // extern "C"
