// rd_serve.cu -- a continuous-batching request server around rd_detect.
//
// The paper runs frames through a multiprocessing producer-consumer pool
// (Methods, "Algorithm implementation"; Performance assessment).  Here one
// process serves a stream of single-frame requests of several sizes on one
// GPU:
//   * each size class (frame size, method parameters) runs its batches on up
//     to `slots` detector contexts ("slots"), each with its own stream;
//   * device memory is admitted against a budget: a slot holds its context's
//     workspaces and the device copy of its frames, and a new slot is created
//     only when its bytes fit beside the slots alive; idle slots of other
//     classes are destroyed (least recently used first) to make room, so a
//     request of a large class waits until batches in flight finish and free
//     their memory, while requests of classes that still have an idle slot
//     keep running;
//   * rd_serve_submit copies the request's frame into a host queue;
//   * a scheduler thread admits queued requests, oldest class first, into a
//     free slot, up to max_batch frames per launch (continuous batching:
//     requests that arrive while others are on the GPU join the next free
//     slot, and the slots' launches overlap on their streams);
//   * the detector writes each batch's rings, counts and offsets straight
//     into mapped pinned host memory (coherent over the CPU-GPU link), so
//     only the rings found leave the device;
//   * a host function enqueued after each batch moves the results to the
//     completion queue and frees the slot (it makes no CUDA call and does
//     not allocate beyond the per-request ring vectors, whose failure is that
//     request's RD_E_NOMEM);
//   * rd_serve_poll hands completed results back with their latency.
// A frame's result does not depend on what it is batched with: rd_detect
// processes the frames of a batch independently.
#include "rd_internal.cuh"
#include "rd_abi_guard.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

struct rd_serve_slot;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long id;
  std::vector<unsigned char> frame;
  Clock::time_point t_submit;
};

struct Result {
  long long id = 0;
  int cls = 0;
  int status = RD_OK;
  std::vector<rd_ring> rings;
  double latency_us = 0.0;
};

constexpr int MAX_CLASSES = 64;

struct ServeClass {
  rd_serve_class cfg;
  size_t frame_bytes = 0;
  long long slot_bytes = 0;  // device bytes of one slot (measured when the first is created)
  std::deque<Request> queue;
  std::vector<rd_serve_slot*> slots;  // alive (reserved to cfg.slots: pushes do not allocate)
};

}  // namespace

struct rd_serve_slot {
  rd_server* server = nullptr;
  int cls = 0;
  rd_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  unsigned char* h_frames = nullptr;  // pinned
  unsigned char* d_frames = nullptr;
  rd_ring* h_rings = nullptr;  // pinned and mapped: the detector writes the rings here
  int* h_counts = nullptr;     // pinned and mapped
  int* h_offsets = nullptr;    // pinned and mapped
  rd_ring* m_rings = nullptr;  // their device addresses
  int* m_counts = nullptr;
  int* m_offsets = nullptr;
  int ring_cap = 0;
  long long bytes = 0;  // device bytes the slot holds
  bool busy = false;
  int status = RD_OK;
  Clock::time_point last_used;
  std::vector<Request> batch;  // reserved to max_batch at creation
};

struct rd_server {
  std::vector<ServeClass> classes;
  int device = 0;
  int queue_cap = 0;
  long long budget = 0;       // device bytes the slots may hold together (0: no limit)
  long long mem_used = 0;     // device bytes the alive slots hold
  long long mem_peak = 0;
  std::mutex m;
  std::condition_variable cv_work, cv_done;
  // completed results: a ring of fixed capacity (every admitted request has a place)
  std::vector<Result> done;
  size_t done_head = 0, done_n = 0;
  bool stop = false;
  std::thread worker;
  long long submitted = 0, completed = 0, batches = 0, queued = 0, outstanding = 0;
  long long created = 0, evicted = 0, memory_waits = 0, failed = 0;
  std::atomic<int> inject_result_fail{0}, inject_create_fail{0};
  std::string err;
};

namespace {

thread_local std::string g_serve_error;

rd_status serve_fail(rd_status s, const std::string& m) {
  g_serve_error = m;
  return s;
}

void free_slot(rd_serve_slot* s) {
  if (s->ctx) rd_destroy(s->ctx);
  if (s->stream) cudaStreamDestroy(s->stream);
  cudaFreeHost(s->h_frames);
  cudaFreeHost(s->h_rings);
  cudaFreeHost(s->h_counts);
  cudaFreeHost(s->h_offsets);
  cudaFree(s->d_frames);
  delete s;
}

// A new slot of class ci: its context, stream, device frames and mapped host
// outputs.  Returns nullptr (and the status) on failure; nothing is kept.
rd_serve_slot* make_slot(rd_server* sv, int ci, rd_status* st_out) {
  ServeClass& c = sv->classes[ci];
  if (sv->inject_create_fail.load() > 0) {
    --sv->inject_create_fail;
    *st_out = RD_E_NOMEM;
    return nullptr;
  }
  rd_serve_slot* s = new (std::nothrow) rd_serve_slot();
  if (!s) {
    *st_out = RD_E_NOMEM;
    return nullptr;
  }
  try {
    s->batch.reserve((size_t)c.cfg.max_batch);
  } catch (...) {
    delete s;
    *st_out = RD_E_NOMEM;
    return nullptr;
  }
  s->server = sv;
  s->cls = ci;
  s->ring_cap = c.cfg.max_batch * 4096;
  rd_status st = rd_create(&c.cfg.params, c.cfg.H, c.cfg.W, c.cfg.max_batch, &s->ctx);
  if (st != RD_OK) {
    free_slot(s);
    *st_out = st;
    return nullptr;
  }
  long long ctx_bytes = 0;
  rd_get_device_bytes(s->ctx, &ctx_bytes);
  void *dr = nullptr, *dc = nullptr, *dof = nullptr;
  bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMallocHost((void**)&s->h_frames, (size_t)c.cfg.max_batch * c.frame_bytes) == cudaSuccess &&
            cudaHostAlloc((void**)&s->h_rings, sizeof(rd_ring) * s->ring_cap, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void**)&s->h_counts, sizeof(int) * c.cfg.max_batch, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostAlloc((void**)&s->h_offsets, sizeof(int) * c.cfg.max_batch, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer(&dr, s->h_rings, 0) == cudaSuccess &&
            cudaHostGetDevicePointer(&dc, s->h_counts, 0) == cudaSuccess &&
            cudaHostGetDevicePointer(&dof, s->h_offsets, 0) == cudaSuccess &&
            cudaMalloc((void**)&s->d_frames, (size_t)c.cfg.max_batch * c.frame_bytes) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_slot(s);
    *st_out = RD_E_NOMEM;
    return nullptr;
  }
  s->m_rings = static_cast<rd_ring*>(dr);
  s->m_counts = static_cast<int*>(dc);
  s->m_offsets = static_cast<int*>(dof);
  s->bytes = ctx_bytes + (long long)c.cfg.max_batch * (long long)c.frame_bytes;
  s->last_used = Clock::now();
  *st_out = RD_OK;
  return s;
}

// Append a result to the completion ring (capacity covers every admitted
// request).  Caller holds sv->m.
void push_done(rd_server* sv, Result&& r) {
  const size_t cap = sv->done.size();
  if (r.status != RD_OK) ++sv->failed;
  sv->done[(sv->done_head + sv->done_n) % cap] = std::move(r);
  ++sv->done_n;
  ++sv->completed;
  --sv->outstanding;
}

// Runs on the CUDA callback thread once the slot's device work is done.  The
// rings are in mapped host memory already: only the counted ones are copied.
void CUDART_CB on_slot_done(void* p) {
  rd_serve_slot* s = static_cast<rd_serve_slot*>(p);
  rd_server* sv = s->server;
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> lock(sv->m);
  for (size_t i = 0; i < s->batch.size(); ++i) {
    Result r;
    r.id = s->batch[i].id;
    r.cls = s->cls;
    r.status = s->status;
    if (s->status == RD_OK) {
      const int off = std::max(0, std::min(s->h_offsets[i], s->ring_cap));
      const int cnt = std::max(0, std::min(s->h_counts[i], s->ring_cap - off));
      try {
        if (sv->inject_result_fail.load() > 0) {
          --sv->inject_result_fail;
          throw std::bad_alloc();
        }
        r.rings.assign(s->h_rings + off, s->h_rings + off + cnt);
      } catch (const std::bad_alloc&) {
        r.status = RD_E_NOMEM;  // this request fails; the server carries on
        r.rings = std::vector<rd_ring>();
      }
    }
    r.latency_us = std::chrono::duration<double, std::micro>(now - s->batch[i].t_submit).count();
    push_done(sv, std::move(r));
  }
  s->batch.clear();
  s->busy = false;
  s->last_used = now;
  sv->cv_done.notify_all();
  sv->cv_work.notify_all();
}

// Launch one batch on a free slot (called by the scheduler, lock not held).
void launch_batch(rd_server* sv, rd_serve_slot* s) {
  rd::NvtxScope trace("rd_serve:batch");
  const ServeClass& c = sv->classes[s->cls];
  const int n = (int)s->batch.size();
  for (int i = 0; i < n; ++i) std::memcpy(s->h_frames + (size_t)i * c.frame_bytes, s->batch[i].frame.data(), c.frame_bytes);
  cudaError_t e = cudaMemcpyAsync(s->d_frames, s->h_frames, (size_t)n * c.frame_bytes, cudaMemcpyHostToDevice, s->stream);
  rd_status st = e == cudaSuccess ? RD_OK : RD_E_CUDA;
  if (st == RD_OK)
    st = rd_detect(s->ctx, s->d_frames, n, c.cfg.H, c.cfg.W, c.cfg.dtype, s->stream, s->m_rings, s->ring_cap,
                   s->m_counts, s->m_offsets);
  s->status = st;
  if (cudaLaunchHostFunc(s->stream, on_slot_done, s) != cudaSuccess) {
    s->status = RD_E_CUDA;
    on_slot_done(s);  // deliver the failure without the device
  }
}

// Fail every queued request of class ci with status st (no slot can be made
// for the class).  Caller holds sv->m.
void fail_queue(rd_server* sv, int ci, rd_status st) {
  ServeClass& c = sv->classes[ci];
  const Clock::time_point now = Clock::now();
  while (!c.queue.empty()) {
    Result r;
    r.id = c.queue.front().id;
    r.cls = ci;
    r.status = st;
    r.latency_us = std::chrono::duration<double, std::micro>(now - c.queue.front().t_submit).count();
    c.queue.pop_front();
    --sv->queued;
    push_done(sv, std::move(r));
  }
  sv->cv_done.notify_all();
}

constexpr int MAX_SLOTS_TOTAL = MAX_CLASSES * 16;

// Unlink idle slots of classes other than `keep`, least recently used first,
// until `need` more bytes fit the budget; the caller frees the victims after
// releasing sv->m (freeing device memory may wait for the device, whose
// completion callbacks take sv->m).  Caller holds sv->m.
bool make_room(rd_server* sv, int keep, long long need, rd_serve_slot** victims, int* n_victims) {
  if (sv->budget <= 0 || sv->mem_used + need <= sv->budget) return true;
  long long freeable = 0;  // evict nothing unless evicting every idle slot would make the room
  for (int ci = 0; ci < (int)sv->classes.size(); ++ci)
    if (ci != keep)
      for (rd_serve_slot* x : sv->classes[ci].slots)
        if (!x->busy) freeable += x->bytes;
  if (sv->mem_used - freeable + need > sv->budget) return false;
  while (sv->mem_used + need > sv->budget) {
    rd_serve_slot* victim = nullptr;
    int vc = -1;
    size_t vi = 0;
    for (int ci = 0; ci < (int)sv->classes.size(); ++ci) {
      if (ci == keep) continue;
      auto& sl = sv->classes[ci].slots;
      for (size_t k = 0; k < sl.size(); ++k)
        if (!sl[k]->busy && (!victim || sl[k]->last_used < victim->last_used)) {
          victim = sl[k];
          vc = ci;
          vi = k;
        }
    }
    if (!victim) return false;
    auto& sl = sv->classes[vc].slots;
    sl.erase(sl.begin() + (std::ptrdiff_t)vi);
    sv->mem_used -= victim->bytes;
    ++sv->evicted;
    victims[(*n_victims)++] = victim;
  }
  return true;
}

// Free unlinked slots with sv->m released, then take it again.
void free_victims(std::unique_lock<std::mutex>& lock, rd_serve_slot** victims, int* n_victims) {
  if (*n_victims == 0) return;
  lock.unlock();
  for (int i = 0; i < *n_victims; ++i) free_slot(victims[i]);
  *n_victims = 0;
  lock.lock();
}

void scheduler(rd_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lock(sv->m);
  int order[MAX_CLASSES];
  rd_serve_slot* victims[MAX_SLOTS_TOTAL];
  int n_victims = 0;
  while (!sv->stop) {
    bool launched = false;
    // classes with queued requests, oldest request first
    int n_order = 0;
    for (int ci = 0; ci < (int)sv->classes.size(); ++ci)
      if (!sv->classes[ci].queue.empty()) order[n_order++] = ci;
    std::sort(order, order + n_order, [&](int a, int b) {
      return sv->classes[a].queue.front().t_submit < sv->classes[b].queue.front().t_submit;
    });
    bool memory_blocked = false;  // an older class waits for memory: newer ones take no new memory
    for (int oi = 0; oi < n_order && !sv->stop; ++oi) {
      const int ci = order[oi];
      ServeClass& c = sv->classes[ci];
      while (!c.queue.empty()) {
        rd_serve_slot* s = nullptr;
        for (rd_serve_slot* x : c.slots)
          if (!x->busy) {
            s = x;
            break;
          }
        if (!s) {
          if ((int)c.slots.size() >= c.cfg.slots || memory_blocked) break;
          const bool room = make_room(sv, ci, c.slot_bytes, victims, &n_victims);
          free_victims(lock, victims, &n_victims);
          if (!room) {  // batches in flight hold the memory: wait for them
            memory_blocked = true;
            ++sv->memory_waits;
            break;
          }
          rd_status st = RD_OK;
          lock.unlock();
          rd_serve_slot* ns = make_slot(sv, ci, &st);
          lock.lock();
          if (!ns) {
            if (c.slots.empty()) fail_queue(sv, ci, st == RD_OK ? RD_E_NOMEM : st);
            break;
          }
          if (sv->budget > 0 && sv->mem_used + ns->bytes > sv->budget &&
              !make_room(sv, ci, ns->bytes, victims, &n_victims)) {
            victims[n_victims++] = ns;  // larger than measured before, and no room now
            free_victims(lock, victims, &n_victims);
            memory_blocked = true;
            ++sv->memory_waits;
            break;
          }
          free_victims(lock, victims, &n_victims);
          c.slot_bytes = std::max(c.slot_bytes, ns->bytes);
          c.slots.push_back(ns);
          sv->mem_used += ns->bytes;
          sv->mem_peak = std::max(sv->mem_peak, sv->mem_used);
          ++sv->created;
          s = ns;
        }
        const int take = std::min<int>((int)c.queue.size(), c.cfg.max_batch);
        s->batch.clear();
        for (int i = 0; i < take; ++i) {
          s->batch.push_back(std::move(c.queue.front()));
          c.queue.pop_front();
        }
        sv->queued -= take;
        s->busy = true;
        ++sv->batches;
        lock.unlock();
        launch_batch(sv, s);
        lock.lock();
        launched = true;
      }
    }
    if (!launched) sv->cv_work.wait_for(lock, std::chrono::milliseconds(50));
  }
}

}  // namespace

extern "C" const char* rd_serve_last_error(void) { return g_serve_error.c_str(); }

extern "C" rd_status rd_serve_create(const rd_serve_class* classes, int n_classes, long long mem_budget,
                                     int queue_cap, rd_server** out) {
  return rd_abi::guard(&g_serve_error, [&]() -> rd_status {
    if (!out || !classes || n_classes < 1 || n_classes > MAX_CLASSES || queue_cap < 1 || mem_budget < 0)
      return serve_fail(RD_E_INVAL, "NULL argument, n_classes outside [1, 64], queue_cap < 1 or mem_budget < 0");
    *out = nullptr;
    long long in_flight = 0;
    for (int i = 0; i < n_classes; ++i) {
      const rd_serve_class& c = classes[i];
      if (c.slots < 1 || c.slots > 16 || c.max_batch < 1 || c.max_batch > 65535 ||
          (c.dtype != RD_U8 && c.dtype != RD_U16))
        return serve_fail(RD_E_INVAL,
                          "class " + std::to_string(i) + ": slots in [1, 16], max_batch in [1, 65535], dtype u8/u16");
      in_flight += (long long)c.slots * c.max_batch;
    }
    // Until the server is handed out, every exit (an error return or an
    // exception) releases its slots and the server itself.
    struct Owner {
      rd_server* sv;
      ~Owner() {
        if (!sv) return;
        for (auto& c : sv->classes)
          for (rd_serve_slot* s : c.slots) free_slot(s);
        delete sv;
      }
    } own{new rd_server()};
    rd_server* sv = own.sv;
    if (cudaGetDevice(&sv->device) != cudaSuccess) return serve_fail(RD_E_CUDA, "no CUDA device");
    sv->queue_cap = queue_cap;
    sv->budget = mem_budget;
    sv->done.resize((size_t)queue_cap + (size_t)in_flight);
    sv->classes.resize(n_classes);
    // One slot per class up front: it measures the class's slot size, and a
    // class whose single slot exceeds the budget can never run.  Slots that
    // do not fit together are destroyed again as later classes need room.
    for (int ci = 0; ci < n_classes; ++ci) {
      ServeClass& c = sv->classes[ci];
      c.cfg = classes[ci];
      c.frame_bytes = (size_t)c.cfg.H * c.cfg.W * (c.cfg.dtype == RD_U8 ? 1 : 2);
      c.slots.reserve((size_t)c.cfg.slots);
      rd_status st = RD_OK;
      rd_serve_slot* s = make_slot(sv, ci, &st);
      if (!s) {
        const char* why = st == RD_E_NOMEM ? "device or host allocation failed" : rd_last_error(nullptr);
        return serve_fail(st, "class " + std::to_string(ci) + ": " + why);
      }
      c.slot_bytes = s->bytes;
      if (mem_budget > 0 && s->bytes > mem_budget) {
        const long long b = s->bytes;
        free_slot(s);
        return serve_fail(RD_E_NOMEM, "class " + std::to_string(ci) + ": one slot needs " + std::to_string(b) +
                                          " bytes of device memory, above the budget of " +
                                          std::to_string(mem_budget));
      }
      rd_serve_slot* victims[MAX_SLOTS_TOTAL];  // all idle: nothing runs before the server is handed out
      int n_victims = 0;
      make_room(sv, ci, s->bytes, victims, &n_victims);
      for (int i = 0; i < n_victims; ++i) free_slot(victims[i]);
      c.slots.push_back(s);
      sv->mem_used += s->bytes;
      sv->mem_peak = std::max(sv->mem_peak, sv->mem_used);
      ++sv->created;
    }
    sv->worker = std::thread(scheduler, sv);
    own.sv = nullptr;
    *out = sv;
    return RD_OK;
  });
}

extern "C" rd_status rd_serve_submit(rd_server* sv, int cls, const void* frame_host, long long request_id) {
  return rd_abi::guard(&g_serve_error, [&]() -> rd_status {
    if (!sv || !frame_host) return serve_fail(RD_E_INVAL, "NULL argument");
    if (cls < 0 || cls >= (int)sv->classes.size()) return serve_fail(RD_E_INVAL, "no such class");
    ServeClass& c = sv->classes[cls];
    Request r;
    r.id = request_id;
    r.frame.assign(static_cast<const unsigned char*>(frame_host), static_cast<const unsigned char*>(frame_host) + c.frame_bytes);
    {
      std::lock_guard<std::mutex> lock(sv->m);
      if (sv->queued >= sv->queue_cap) return serve_fail(RD_E_BUSY, "request queue full");
      if (sv->outstanding + (long long)sv->done_n >= (long long)sv->done.size())
        return serve_fail(RD_E_BUSY, "completed results not polled");
      r.t_submit = Clock::now();
      c.queue.push_back(std::move(r));
      ++sv->queued;
      ++sv->outstanding;
      ++sv->submitted;
    }
    sv->cv_work.notify_one();
    return RD_OK;
  });
}

extern "C" int rd_serve_poll(rd_server* sv, long long* ids, int* classes, int* status, int* n_rings, rd_ring* rings,
                             int rings_cap, double* latency_us, int max_results, int wait_ms) {
  return rd_abi::guard_count(&g_serve_error, [&]() -> int {
    if (!sv || !ids || max_results < 1 || rings_cap < 0 || (rings_cap > 0 && !rings)) return -1;
    std::unique_lock<std::mutex> lock(sv->m);
    if (sv->done_n == 0 && wait_ms > 0)
      sv->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return sv->done_n > 0; });
    int k = 0, used = 0;
    while (k < max_results && sv->done_n > 0) {
      Result& r = sv->done[sv->done_head];
      const int nr = (int)r.rings.size();
      if (used + nr > rings_cap && k > 0) break;  // the next poll returns it
      const int keep = std::min(nr, rings_cap - used);
      ids[k] = r.id;
      if (classes) classes[k] = r.cls;
      if (status) status[k] = r.status;
      if (n_rings) n_rings[k] = keep;
      if (latency_us) latency_us[k] = r.latency_us;
      if (keep > 0) std::memcpy(rings + used, r.rings.data(), sizeof(rd_ring) * keep);
      used += keep;
      r.rings = std::vector<rd_ring>();
      sv->done_head = (sv->done_head + 1) % sv->done.size();
      --sv->done_n;
      ++k;
    }
    return k;
  });
}

extern "C" rd_status rd_serve_stats(rd_server* sv, long long* out4) {
  if (!sv || !out4) return RD_E_INVAL;
  std::lock_guard<std::mutex> lock(sv->m);
  out4[0] = sv->submitted;
  out4[1] = sv->completed;
  out4[2] = sv->batches;
  out4[3] = sv->mem_used;
  return RD_OK;
}

extern "C" int rd_serve_stats_ex(rd_server* sv, long long* out, int cap) {
  if (!sv || !out || cap < 0) return -1;
  std::lock_guard<std::mutex> lock(sv->m);
  const long long v[RD_SERVE_N_STATS] = {sv->submitted, sv->completed, sv->batches,      sv->mem_used,
                                         sv->mem_peak,  sv->created,   sv->evicted,      sv->memory_waits,
                                         sv->failed,    sv->budget};
  const int n = std::min(cap, (int)RD_SERVE_N_STATS);
  for (int i = 0; i < n; ++i) out[i] = v[i];
  return n;
}

extern "C" rd_status rd_serve_debug_inject(rd_server* sv, int kind, int count) {
  if (!sv || count < 0 || (kind != RD_SERVE_FAIL_RESULT && kind != RD_SERVE_FAIL_SLOT)) return RD_E_INVAL;
  if (kind == RD_SERVE_FAIL_RESULT)
    sv->inject_result_fail.store(count);
  else
    sv->inject_create_fail.store(count);
  return RD_OK;
}

extern "C" rd_status rd_serve_destroy(rd_server* sv) {
  if (!sv) return RD_E_INVAL;
  {
    std::lock_guard<std::mutex> lock(sv->m);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& c : sv->classes)
    for (rd_serve_slot* s : c.slots)
      if (s->stream) cudaStreamSynchronize(s->stream);  // in-flight batches finish; their callbacks run
  for (auto& c : sv->classes)
    for (rd_serve_slot* s : c.slots) free_slot(s);
  delete sv;
  return RD_OK;
}
