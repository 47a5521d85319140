// Serving: resident scenes, memory-admitted requests, continuous batching.
//
// A session owns one device pool (allocated once) and `max_slots` CUDA
// streams.  Requests (a scene, a transmitter, a launch, a reflection order
// limit, a range) queue in arrival order; a worker thread admits the head of
// the queue as soon as a slot is free and the pool can hold all of the
// request's buffers, so requests that arrive while others run start at once
// and their kernels overlap on the device.  Each request runs the Sec. III
// path on its slot's stream -- launch (Sec. III.A), closest hit, then up to
// max_order rounds of reflect + compact + trace -- writes its results to the
// caller's host buffers and frees its pool memory.  A request's result
// depends only on its own rays and scene, never on what else is running.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "rt_internal.cuh"

namespace rt {
int set_error(int code, const char* msg);
}

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over the session pool (offsets, 256-byte granules).
class Pool {
 public:
  void reset(size_t bytes) {
    free_.clear();
    free_[0] = bytes;
    cap_ = bytes;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t cap() const { return cap_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t cap_ = 0, used_ = 0, peak_ = 0;
};

struct Req {
  uint64_t ticket;
  rt_request r;
  long long n = 0;
  size_t bytes = 0, off = 0;
  int slot = -1;
  Clock::time_point t_submit, t_start, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  // device buffers inside the pool
  rt_ray* rays[RT_BATCH_MAX_ORDER + 1] = {};
  rt_hit* hits[RT_BATCH_MAX_ORDER + 1] = {};
  int* skip[RT_BATCH_MAX_ORDER + 1] = {};
  int* src[RT_BATCH_MAX_ORDER + 1] = {};
  int* counts = nullptr;
  int* blocks = nullptr;
  rt::TraceScratch scr;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  rt_hit* pinned_hits = nullptr;  // staging for the order-0 hits
  long long pinned_cap = 0;
  int* pinned_counts = nullptr;
  Req* req = nullptr;
};

size_t request_bytes(long long n, int orders) {
  const size_t per_order = (size_t)n * (sizeof(rt_ray) + sizeof(rt_hit) + 2 * sizeof(int));
  size_t b = per_order * (size_t)(orders + 1);
  b += 64 + (size_t)(RT_BATCH_MAX_ORDER + 1) * sizeof(int);      // counts
  b += ((size_t)n / 256 + 2) * sizeof(int);                       // reflect blocks
  b += 64 + (size_t)n * sizeof(int) * (1 + rt::kTraceCand + 1);    // trace counter, queue, candidates
  return b + 64 * 256;                                            // alignment slack (<= 48 arrays)
}

}  // namespace

// Latency percentiles cover this many of the most recent completed requests.
constexpr size_t kLatencyWindow = size_t(1) << 20;

struct rt_session_s {
  int device = 0;
  unsigned char* pool_mem = nullptr;
  Pool pool;
  std::vector<Slot> slots;
  std::vector<rt_scene> scenes;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::map<uint64_t, Req*> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  // statistics: rings of the last kLatencyWindow latencies (submit to done),
  // queue waits (submit to admission) and run times (admission to done)
  std::vector<double> lat_ms, wait_ms, run_ms;
  size_t lat_next = 0;
  long long submitted = 0, completed = 0, failed = 0, rays = 0;
  int running = 0, peak_running = 0;
  Clock::time_point t_first, t_last;
  bool any_done = false;
};

namespace {

template <class T>
T* carve(unsigned char* base, size_t* at, size_t count) {
  *at = (*at + 255) & ~size_t(255);
  T* p = reinterpret_cast<T*>(base + *at);
  *at += count * sizeof(T);
  return p;
}

cudaError_t start(rt_session_s* S, Req* q, Slot& sl) {
  rt_scene scene = S->scenes[q->r.scene_id];
  unsigned char* base = S->pool_mem + q->off;
  size_t at = 0;
  const int orders = q->r.max_order;
  for (int k = 0; k <= orders; ++k) {
    q->rays[k] = carve<rt_ray>(base, &at, q->n);
    q->hits[k] = carve<rt_hit>(base, &at, q->n);
    q->skip[k] = carve<int>(base, &at, q->n);
    q->src[k] = carve<int>(base, &at, q->n);
  }
  q->counts = carve<int>(base, &at, RT_BATCH_MAX_ORDER + 1);
  q->blocks = carve<int>(base, &at, q->n / 256 + 2);
  q->scr.counter = carve<int>(base, &at, 16);
  q->scr.queue = carve<int>(base, &at, q->n);
  q->scr.cand = carve<int>(base, &at, (size_t)q->n * (rt::kTraceCand + 1));
  q->scr.cap = q->n;
  cudaError_t e;
  cudaStream_t st = sl.st;
  if ((e = cudaMemsetAsync(q->counts, 0, (RT_BATCH_MAX_ORDER + 1) * sizeof(int), st))) return e;
  if ((e = rt::launch_gen_rays(q->r.dir_kind, q->r.tx, q->r.param, 0.f, q->r.tmax, q->rays[0], q->n, st)))
    return e;
  rt_trace_params tp{};
  if ((e = rt::launch_trace_dev(scene, q->rays[0], q->n, nullptr, q->hits[0], nullptr, &tp, q->scr, st))) return e;
  for (int k = 1; k <= orders; ++k) {
    const int* prev = k == 1 ? nullptr : q->counts + (k - 1);
    if ((e = rt::launch_reflect(scene, q->rays[k - 1], q->hits[k - 1], q->n, prev, q->rays[k], q->skip[k], q->src[k],
                                q->counts + k, q->blocks, q->n, st)))
      return e;
    rt_trace_params tk{};
    tk.skip_tri_dev = q->skip[k];
    if ((e = rt::launch_trace_dev(scene, q->rays[k], q->n, q->counts + k, q->hits[k], nullptr, &tk, q->scr, st)))
      return e;
  }
  if (q->r.hits_host) {
    if (sl.pinned_cap < q->n) {
      if (sl.pinned_hits) cudaFreeHost(sl.pinned_hits);
      sl.pinned_hits = nullptr;
      if ((e = cudaMallocHost((void**)&sl.pinned_hits, (size_t)q->n * sizeof(rt_hit)))) return e;
      sl.pinned_cap = q->n;
    }
    if ((e = cudaMemcpyAsync(sl.pinned_hits, q->hits[0], (size_t)q->n * sizeof(rt_hit), cudaMemcpyDeviceToHost, st)))
      return e;
  }
  if ((e = cudaMemcpyAsync(sl.pinned_counts, q->counts, (RT_BATCH_MAX_ORDER + 1) * sizeof(int),
                           cudaMemcpyDeviceToHost, st)))
    return e;
  return cudaEventRecord(sl.done, st);
}

// The hits (and parent indices) of every reflection order the request asked
// for: exactly the order's count, known once its work is done, copied from
// the request's pool memory before that memory is released.
cudaError_t copy_orders(Req* q, Slot& sl) {
  cudaError_t e = cudaSuccess;
  for (int k = 1; k <= q->r.max_order && e == cudaSuccess; ++k) {
    const long long c = sl.pinned_counts[k];
    if (c <= 0 || c > q->n) continue;
    if (q->r.order_hits_host && q->r.order_hits_host[k])
      e = cudaMemcpyAsync(q->r.order_hits_host[k], q->hits[k], (size_t)c * sizeof(rt_hit), cudaMemcpyDeviceToHost,
                          sl.st);
    if (e == cudaSuccess && q->r.order_src_host && q->r.order_src_host[k])
      e = cudaMemcpyAsync(q->r.order_src_host[k], q->src[k], (size_t)c * sizeof(int), cudaMemcpyDeviceToHost, sl.st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(sl.st);
  return e;
}

void finish(rt_session_s* S, Slot& sl, bool ok) {
  Req* q = sl.req;
  if (ok && q->r.hits_host) memcpy(q->r.hits_host, sl.pinned_hits, (size_t)q->n * sizeof(rt_hit));
  if (ok && (q->r.order_hits_host || q->r.order_src_host) && copy_orders(q, sl) != cudaSuccess) {
    cudaGetLastError();
    ok = false;
  }
  long long rays = q->n;
  if (ok) {
    for (int k = 1; k <= q->r.max_order; ++k) rays += sl.pinned_counts[k];
    if (q->r.order_counts_host) {
      q->r.order_counts_host[0] = q->n;
      for (int k = 1; k <= q->r.max_order; ++k) q->r.order_counts_host[k] = sl.pinned_counts[k];
    }
  }
  std::lock_guard<std::mutex> lk(S->mu);
  q->t_done = Clock::now();
  q->state = ok ? 2 : 3;
  S->pool.release(q->off, q->bytes);
  sl.req = nullptr;
  --S->running;
  if (ok) {
    ++S->completed;
    S->rays += rays;
    const double ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    const double wait = std::chrono::duration<double, std::milli>(q->t_start - q->t_submit).count();
    if (S->lat_ms.size() < kLatencyWindow) {
      S->lat_ms.push_back(ms);
      S->wait_ms.push_back(wait);
      S->run_ms.push_back(ms - wait);
    } else {
      S->lat_ms[S->lat_next] = ms;
      S->wait_ms[S->lat_next] = wait;
      S->run_ms[S->lat_next] = ms - wait;
      S->lat_next = (S->lat_next + 1) % kLatencyWindow;
    }
    S->t_last = q->t_done;
  } else {
    ++S->failed;
  }
  S->cv_done.notify_all();
}

void worker_loop(rt_session_s* S) {
  cudaSetDevice(S->device);
  for (;;) {
    // 1. admit from the head of the queue while a slot and memory are free
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop && S->queue.empty() && S->running == 0) return;
      for (;;) {
        if (S->queue.empty()) break;
        int free_slot = -1;
        for (size_t i = 0; i < S->slots.size(); ++i)
          if (!S->slots[i].req) {
            free_slot = (int)i;
            break;
          }
        if (free_slot < 0) break;
        Req* q = S->queue.front();
        size_t off;
        if (!S->pool.alloc(q->bytes, &off)) break;  // head waits for memory
        S->queue.pop_front();
        q->off = off;
        q->slot = free_slot;
        q->state = 1;
        q->t_start = Clock::now();
        Slot& sl = S->slots[free_slot];
        sl.req = q;
        ++S->running;
        S->peak_running = std::max(S->peak_running, S->running);
        lk.unlock();
        const bool ok = start(S, q, sl) == cudaSuccess;
        if (!ok) {
          // work queued before the failing call may still use the request's
          // pool memory: let the stream drain before the memory is reused
          cudaStreamSynchronize(sl.st);
          cudaGetLastError();
          finish(S, sl, false);
        }
        lk.lock();
      }
      if (S->running == 0) {
        if (S->stop && S->queue.empty()) return;
        S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
    }
    // 2. retire finished requests
    bool any = false;
    for (Slot& sl : S->slots) {
      if (!sl.req) continue;
      cudaError_t e = cudaEventQuery(sl.done);
      if (e == cudaSuccess) {
        finish(S, sl, true);
        any = true;
      } else if (e != cudaErrorNotReady) {
        cudaGetLastError();
        finish(S, sl, false);
        any = true;
      }
    }
    if (!any) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

static int rt_session_create_body(size_t pool_bytes, int max_slots, rt_session* out) {
  if (!out) return rt::set_error(RT_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_slots < 1 || max_slots > 64) return rt::set_error(RT_EINVAL, "max_slots must be 1..64");
  if (pool_bytes < (1u << 20)) return rt::set_error(RT_EINVAL, "pool_bytes must be at least 1 MiB");
  rt_session_s* S = new (std::nothrow) rt_session_s();
  if (!S) return rt::set_error(RT_ENOMEM, "host allocation failed");
  cudaError_t e = cudaMalloc((void**)&S->pool_mem, pool_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return rt::set_error(e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA, "pool allocation failed");
  }
  cudaGetDevice(&S->device);
  try {
    S->pool.reset(pool_bytes);
    S->lat_ms.reserve(kLatencyWindow);  // the worker thread never reallocates them
    S->wait_ms.reserve(kLatencyWindow);
    S->run_ms.reserve(kLatencyWindow);
    S->slots.resize(max_slots);
    for (Slot& sl : S->slots) {
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.pinned_counts, (RT_BATCH_MAX_ORDER + 1) * sizeof(int));
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      rt_session_destroy(S);
      return rt::set_error(RT_ECUDA, "session streams");
    }
    S->worker = std::thread(worker_loop, S);
  } catch (...) {  // no worker is running: free what was made
    rt_session_destroy(S);
    throw;
  }
  *out = S;
  return RT_OK;
}

int rt_session_create(size_t pool_bytes, int max_slots, rt_session* out) {
  return rt::abi_guard([&] { return rt_session_create_body(pool_bytes, max_slots, out); });
}

static int rt_session_add_scene_body(rt_session S, rt_scene scene, int32_t* scene_id) {
  if (!S || !scene || !scene_id) return rt::set_error(RT_EINVAL, "NULL argument");
  if (!scene->built) return rt::set_error(RT_ENOTBUILT, "build the scene's BVH before adding it");
  std::lock_guard<std::mutex> lk(S->mu);
  *scene_id = (int32_t)S->scenes.size();
  S->scenes.push_back(scene);
  return RT_OK;
}

int rt_session_add_scene(rt_session S, rt_scene scene, int32_t* scene_id) {
  return rt::abi_guard([&] { return rt_session_add_scene_body(S, scene, scene_id); });
}

static int rt_session_submit_body(rt_session S, const rt_request* r, uint64_t* ticket) {
  if (!S || !r || !ticket) return rt::set_error(RT_EINVAL, "NULL argument");
  const long long n = rt_ray_count(r->dir_kind, r->param);
  if (n < 1 || n > (1 << 30)) return rt::set_error(RT_EINVAL, "bad launch");
  if (r->max_order < 0 || r->max_order > RT_BATCH_MAX_ORDER) return rt::set_error(RT_EINVAL, "max_order out of range");
  if (!(r->tmax > 0.f)) return rt::set_error(RT_EINVAL, "tmax must be > 0");
  Req* q = new (std::nothrow) Req();
  if (!q) return rt::set_error(RT_ENOMEM, "host allocation failed");
  q->r = *r;
  q->n = n;
  q->bytes = request_bytes(n, r->max_order);
  std::lock_guard<std::mutex> lk(S->mu);
  if (r->scene_id < 0 || r->scene_id >= (int)S->scenes.size()) {
    delete q;
    return rt::set_error(RT_EINVAL, "unknown scene_id");
  }
  if (q->bytes > S->pool.cap()) {
    delete q;
    return rt::set_error(RT_ENOMEM, "request larger than the session pool");
  }
  q->ticket = S->next_ticket;
  q->t_submit = Clock::now();
  try {
    S->reqs[q->ticket] = q;
    S->queue.push_back(q);
  } catch (...) {  // neither queued nor known: as if never submitted
    S->reqs.erase(q->ticket);
    delete q;
    throw;
  }
  ++S->next_ticket;
  if (!S->submitted) S->t_first = q->t_submit;
  ++S->submitted;
  *ticket = q->ticket;
  S->cv_work.notify_one();
  return RT_OK;
}

int rt_session_submit(rt_session S, const rt_request* r, uint64_t* ticket) {
  return rt::abi_guard([&] { return rt_session_submit_body(S, r, ticket); });
}

int rt_session_poll(rt_session S, uint64_t ticket, int* done) {
  if (!S || !done) return rt::set_error(RT_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return rt::set_error(RT_EINVAL, "unknown ticket");
  *done = it->second->state >= 2 ? 1 : 0;
  return it->second->state == 3 ? rt::set_error(RT_ECUDA, "request failed") : RT_OK;
}

int rt_session_wait(rt_session S, uint64_t ticket, int64_t timeout_ns) {
  if (!S) return rt::set_error(RT_EINVAL, "session is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return rt::set_error(RT_EINVAL, "unknown ticket");
  Req* q = it->second;
  auto pred = [&] { return q->state >= 2; };
  if (timeout_ns < 0) {
    S->cv_done.wait(lk, pred);
  } else if (!S->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), pred)) {
    return rt::set_error(RT_ETIMEOUT, "request not finished within the timeout");
  }
  return q->state == 3 ? rt::set_error(RT_ECUDA, "request failed") : RT_OK;
}

int rt_session_release(rt_session S, uint64_t ticket) {
  if (!S) return rt::set_error(RT_EINVAL, "session is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return rt::set_error(RT_EINVAL, "unknown ticket");
  if (it->second->state < 2) return rt::set_error(RT_EBUSY, "request still queued or running");
  delete it->second;
  S->reqs.erase(it);
  return RT_OK;
}

static int rt_session_stats_get_body(rt_session S, rt_session_stats* st) {
  if (!S || !st) return rt::set_error(RT_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  memset(st, 0, sizeof(*st));
  st->submitted = S->submitted;
  st->completed = S->completed;
  st->failed = S->failed;
  st->queued = (int64_t)S->queue.size();
  st->running = S->running;
  st->peak_running = S->peak_running;
  st->rays = S->rays;
  st->pool_bytes = (int64_t)S->pool.cap();
  st->peak_pool_bytes = (int64_t)S->pool.peak();
  if (!S->lat_ms.empty()) {
    // percentiles (linear interpolation) of one sorted copy
    auto pct = [](std::vector<double> v, double p) {
      std::sort(v.begin(), v.end());
      const double x = p * (double)(v.size() - 1);
      const size_t i = (size_t)x;
      const double f = x - (double)i;
      return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
    };
    st->p50_ms = pct(S->lat_ms, 0.50);
    st->p99_ms = pct(S->lat_ms, 0.99);
    st->wait_p50_ms = pct(S->wait_ms, 0.50);
    st->wait_p99_ms = pct(S->wait_ms, 0.99);
    st->run_p50_ms = pct(S->run_ms, 0.50);
    st->run_p99_ms = pct(S->run_ms, 0.99);
    double s = 0;
    for (double x : S->lat_ms) s += x;
    st->mean_ms = s / (double)S->lat_ms.size();
    st->span_s = std::chrono::duration<double>(S->t_last - S->t_first).count();
  }
  return RT_OK;
}

int rt_session_stats_get(rt_session S, rt_session_stats* st) {
  return rt::abi_guard([&] { return rt_session_stats_get_body(S, st); });
}

int rt_session_destroy(rt_session S) {
  if (!S) return rt::set_error(RT_EINVAL, "session is NULL");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  for (Slot& sl : S->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.pinned_hits) cudaFreeHost(sl.pinned_hits);
    if (sl.pinned_counts) cudaFreeHost(sl.pinned_counts);
  }
  for (auto& kv : S->reqs) delete kv.second;
  if (S->pool_mem) cudaFree(S->pool_mem);
  delete S;
  return RT_OK;
}

}  // extern "C"
