// rd_serve.cu -- a continuous-batching request server around rd_detect.
//
// The paper runs frames through a multiprocessing producer-consumer pool
// (Methods, "Algorithm implementation"; Performance assessment).  Here one
// process serves a stream of single-frame requests of several sizes on one
// GPU:
//   * each size class (frame size, method parameters) owns `slots` detector
//     contexts, each with its own stream and pinned staging buffers, created
//     up front; their device workspaces must fit the server's memory budget;
//   * rd_serve_submit copies the request's frame into a host queue;
//   * a scheduler thread admits queued requests into free slots, up to
//     max_batch frames per launch (continuous batching: requests that arrive
//     while others are on the GPU join the next free slot, and the slots'
//     launches overlap on their streams);
//   * a host function enqueued after each slot's device work moves the
//     results to the completion queue and frees the slot (it makes no CUDA
//     call);
//   * rd_serve_poll hands completed results back with their latency.
// A frame's result does not depend on what it is batched with: rd_detect
// processes the frames of a batch independently.
#include "rd_internal.cuh"
#include "rd_abi_guard.h"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
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
  long long id;
  int cls;
  int status;
  std::vector<rd_ring> rings;
  double latency_us;
};

struct ServeClass {
  rd_serve_class cfg;
  size_t frame_bytes = 0;
  std::deque<Request> queue;
  std::vector<rd_serve_slot*> slots;
};

}  // namespace

struct rd_serve_slot {
  rd_server* server = nullptr;
  int cls = 0;
  rd_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  unsigned char* h_frames = nullptr;  // pinned
  unsigned char* d_frames = nullptr;
  rd_ring* d_rings = nullptr;
  int* d_counts = nullptr;
  int* d_offsets = nullptr;
  rd_ring* h_rings = nullptr;  // pinned
  int* h_counts = nullptr;
  int* h_offsets = nullptr;
  int ring_cap = 0;
  bool busy = false;
  int status = RD_OK;
  std::vector<Request> batch;
};

struct rd_server {
  std::vector<ServeClass> classes;
  std::vector<rd_serve_slot*> all_slots;
  int device = 0;
  int queue_cap = 0;
  long long mem_used = 0;
  std::mutex m;
  std::condition_variable cv_work, cv_done;
  std::deque<Result> done;
  bool stop = false;
  std::thread worker;
  long long submitted = 0, completed = 0, batches = 0, queued = 0;
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
  cudaFree(s->d_rings);
  cudaFree(s->d_counts);
  cudaFree(s->d_offsets);
  delete s;
}

// Runs on the CUDA callback thread once the slot's copies back have landed.
void CUDART_CB on_slot_done(void* p) {
  rd_serve_slot* s = static_cast<rd_serve_slot*>(p);
  rd_server* sv = s->server;
  const Clock::time_point now = Clock::now();
  std::vector<Result> out;
  out.reserve(s->batch.size());
  for (size_t i = 0; i < s->batch.size(); ++i) {
    Result r;
    r.id = s->batch[i].id;
    r.cls = s->cls;
    r.status = s->status;
    if (s->status == RD_OK) {
      const int off = s->h_offsets[i];
      const int cnt = std::max(0, std::min(s->h_counts[i], s->ring_cap - off));
      r.rings.assign(s->h_rings + off, s->h_rings + off + cnt);
    }
    r.latency_us = std::chrono::duration<double, std::micro>(now - s->batch[i].t_submit).count();
    out.push_back(std::move(r));
  }
  {
    std::lock_guard<std::mutex> lock(sv->m);
    for (auto& r : out) sv->done.push_back(std::move(r));
    sv->completed += (long long)out.size();
    s->batch.clear();
    s->busy = false;
  }
  sv->cv_done.notify_all();
  sv->cv_work.notify_all();
}

// Launch one batch on a free slot (called by the scheduler, lock not held).
void launch_batch(rd_server* sv, rd_serve_slot* s) {
  const ServeClass& c = sv->classes[s->cls];
  const int n = (int)s->batch.size();
  for (int i = 0; i < n; ++i) std::memcpy(s->h_frames + (size_t)i * c.frame_bytes, s->batch[i].frame.data(), c.frame_bytes);
  cudaError_t e = cudaMemcpyAsync(s->d_frames, s->h_frames, (size_t)n * c.frame_bytes, cudaMemcpyHostToDevice, s->stream);
  rd_status st = e == cudaSuccess ? RD_OK : RD_E_CUDA;
  if (st == RD_OK)
    st = rd_detect(s->ctx, s->d_frames, n, c.cfg.H, c.cfg.W, c.cfg.dtype, s->stream, s->d_rings, s->ring_cap,
                   s->d_counts, s->d_offsets);
  if (st == RD_OK) {
    e = cudaMemcpyAsync(s->h_counts, s->d_counts, sizeof(int) * n, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_offsets, s->d_offsets, sizeof(int) * n, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->h_rings, s->d_rings, sizeof(rd_ring) * s->ring_cap, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) st = RD_E_CUDA;
  }
  s->status = st;
  if (cudaLaunchHostFunc(s->stream, on_slot_done, s) != cudaSuccess) {
    s->status = RD_E_CUDA;
    on_slot_done(s);  // deliver the failure without the device
  }
}

void scheduler(rd_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lock(sv->m);
  while (!sv->stop) {
    bool launched = false;
    for (size_t ci = 0; ci < sv->classes.size(); ++ci) {
      ServeClass& c = sv->classes[ci];
      for (rd_serve_slot* s : c.slots) {
        if (c.queue.empty()) break;
        if (s->busy) continue;
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
    if (!out || !classes || n_classes < 1 || n_classes > 64 || queue_cap < 1)
      return serve_fail(RD_E_INVAL, "NULL argument, n_classes outside [1, 64] or queue_cap < 1");
    *out = nullptr;
    for (int i = 0; i < n_classes; ++i) {
      const rd_serve_class& c = classes[i];
      if (c.slots < 1 || c.slots > 16 || c.max_batch < 1 || c.max_batch > 65535 ||
          (c.dtype != RD_U8 && c.dtype != RD_U16))
        return serve_fail(RD_E_INVAL,
                          "class " + std::to_string(i) + ": slots in [1, 16], max_batch in [1, 65535], dtype u8/u16");
    }
    // Until the server is handed out, every exit (an error return or an
    // exception) releases its slots and the server itself.
    struct Owner {
      rd_server* sv;
      ~Owner() {
        if (!sv) return;
        for (rd_serve_slot* s : sv->all_slots) free_slot(s);
        delete sv;
      }
    } own{new rd_server()};
    rd_server* sv = own.sv;
    if (cudaGetDevice(&sv->device) != cudaSuccess) return serve_fail(RD_E_CUDA, "no CUDA device");
    sv->queue_cap = queue_cap;
    sv->classes.resize(n_classes);
    for (int ci = 0; ci < n_classes; ++ci) {
      ServeClass& c = sv->classes[ci];
      c.cfg = classes[ci];
      c.frame_bytes = (size_t)c.cfg.H * c.cfg.W * (c.cfg.dtype == RD_U8 ? 1 : 2);
      for (int k = 0; k < c.cfg.slots; ++k) {
        size_t free0 = 0, free1 = 0, total = 0;
        cudaMemGetInfo(&free0, &total);
        sv->all_slots.reserve(sv->all_slots.size() + 1);  // so that the push below cannot fail
        rd_serve_slot* s = new rd_serve_slot();
        sv->all_slots.push_back(s);
        s->server = sv;
        s->cls = ci;
        s->ring_cap = c.cfg.max_batch * 4096;
        const rd_status st = rd_create(&c.cfg.params, c.cfg.H, c.cfg.W, c.cfg.max_batch, &s->ctx);
        if (st != RD_OK) return serve_fail(st, "class " + std::to_string(ci) + ": " + rd_last_error(nullptr));
        bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaMallocHost((void**)&s->h_frames, (size_t)c.cfg.max_batch * c.frame_bytes) == cudaSuccess &&
                  cudaMallocHost((void**)&s->h_rings, sizeof(rd_ring) * s->ring_cap) == cudaSuccess &&
                  cudaMallocHost((void**)&s->h_counts, sizeof(int) * c.cfg.max_batch) == cudaSuccess &&
                  cudaMallocHost((void**)&s->h_offsets, sizeof(int) * c.cfg.max_batch) == cudaSuccess &&
                  cudaMalloc((void**)&s->d_frames, (size_t)c.cfg.max_batch * c.frame_bytes) == cudaSuccess &&
                  cudaMalloc((void**)&s->d_rings, sizeof(rd_ring) * s->ring_cap) == cudaSuccess &&
                  cudaMalloc((void**)&s->d_counts, sizeof(int) * c.cfg.max_batch) == cudaSuccess &&
                  cudaMalloc((void**)&s->d_offsets, sizeof(int) * c.cfg.max_batch) == cudaSuccess;
        if (!ok) {
          cudaGetLastError();
          return serve_fail(RD_E_NOMEM, "class " + std::to_string(ci) + ": slot buffers");
        }
        cudaMemGetInfo(&free1, &total);
        sv->mem_used += (long long)free0 - (long long)free1;
        c.slots.push_back(s);
        if (mem_budget > 0 && sv->mem_used > mem_budget)
          return serve_fail(RD_E_NOMEM, "the classes' slots need " + std::to_string(sv->mem_used) +
                                            " bytes of device memory, above the budget of " + std::to_string(mem_budget));
      }
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
      r.t_submit = Clock::now();
      c.queue.push_back(std::move(r));
      ++sv->queued;
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
    if (sv->done.empty() && wait_ms > 0)
      sv->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return !sv->done.empty(); });
    int k = 0, used = 0;
    while (k < max_results && !sv->done.empty()) {
      Result& r = sv->done.front();
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
      sv->done.pop_front();
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

extern "C" rd_status rd_serve_destroy(rd_server* sv) {
  if (!sv) return RD_E_INVAL;
  {
    std::lock_guard<std::mutex> lock(sv->m);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (rd_serve_slot* s : sv->all_slots)
    if (s->stream) cudaStreamSynchronize(s->stream);  // in-flight batches finish; their callbacks run
  for (rd_serve_slot* s : sv->all_slots) free_slot(s);
  delete sv;
  return RD_OK;
}
