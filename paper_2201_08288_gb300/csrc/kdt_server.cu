// kdt_server.cu -- continuous batching of build requests on one GPU.
//
// The server owns one device arena (allocated once, at creation) holding the
// engine's shared tables and the per-tree working memory of the requests in
// flight. A worker thread loops: it admits queued requests (first in, first
// out) as long as a slot, arena memory and table capacity are free, runs one
// engine tick (one level step over every tree in flight, each at its own
// level, then the subtree kernel), and retires the trees that finished. A
// request that arrives while others are on the GPU therefore joins the next
// level step and its work overlaps theirs on the device. Because no
// reduction crosses trees, every result is the same alone or in a mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "kdt.h"
#include "kdt_engine.h"

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) of the arena's tree region.
class Arena {
 public:
  explicit Arena(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes ? bytes : 1);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct Request {
  uint64_t ticket = 0;
  kdt_tree_desc desc{};
  kdt::TreePlan plan;
  kdt::StepNeeds needs;  // this tree's share of the shared tables
  size_t off = 0;
  uint32_t slot = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  kdt_status status = KDT_OK;
  int32_t levels = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct kdt_server {
  int device = 0;
  size_t budget = 0;
  uint32_t max_slots = 0;
  uint8_t* mem = nullptr;
  size_t tree_base = 0;  // offset of the tree region in mem
  kdt::StepPlan step;
  kdt::Engine* engine = nullptr;
  Arena* arena = nullptr;
  cudaStream_t stream = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> requests;
  std::vector<Request*> slot_req;
  std::vector<uint32_t> free_slots;
  kdt::StepNeeds in_use;  // table capacity used by the trees in flight
  kdt_server_info info{};
  kdt_status fatal = KDT_OK;

  bool fits(const Request& r) const {
    const kdt::StepNeeds& cap = step.needs;
    return in_use.points + r.needs.points <= cap.points && in_use.maxB + r.needs.maxB <= cap.maxB &&
           in_use.cap_small + r.needs.cap_small <= cap.cap_small && in_use.nseg + r.needs.nseg <= cap.nseg &&
           r.needs.max_d <= cap.max_d && r.needs.slice_cells <= cap.slice_cells;
  }
  void take(const kdt::StepNeeds& n, int sign) {
    in_use.points += sign * (int64_t)n.points;
    in_use.maxB += sign * (int64_t)n.maxB;
    in_use.cap_small += sign * (int64_t)n.cap_small;
    in_use.nseg += sign * (int64_t)n.nseg;
  }

  void run() {
    cudaSetDevice(device);
    std::vector<uint32_t> running, done;
    std::vector<kdt_status> st;
    std::vector<int32_t> lv;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        // admit in arrival order while a slot, memory and table capacity are free
        while (!queue.empty() && !free_slots.empty() && fatal == KDT_OK) {
          Request* r = queue.front();
          if (!fits(*r)) break;
          size_t off = 0;
          if (!arena->alloc(r->plan.bytes, &off)) break;
          queue.pop_front();
          r->off = off;
          r->slot = free_slots.back();
          free_slots.pop_back();
          take(r->needs, +1);
          const kdt_params& p = r->desc.params;
          const kdt_status s = engine->admit(r->slot, r->desc.points, p, r->plan, mem + tree_base + off,
                                             r->desc.out_perm, r->desc.out_split_vals, r->desc.out_split_dims,
                                             r->desc.out_node_offsets);
          r->t_admit = now_ms();
          r->state = 1;
          slot_req[r->slot] = r;
          if (s != KDT_OK) fatal = s;
          info.admitted += 1;
        }
        running.clear();
        for (uint32_t k = 0; k < max_slots; ++k)
          if (slot_req[k]) running.push_back(k);
        info.in_flight = (int32_t)running.size();
        info.peak_in_flight = std::max(info.peak_in_flight, info.in_flight);
        info.arena_bytes_in_use = arena->used() + tree_base;
        if (running.empty()) {
          if (stop) return;
          cv_work.wait_for(lk, std::chrono::milliseconds(50));
          continue;
        }
      }
      kdt_status s = kdt::fault_take(KDT_FAULT_SERVER_STEP) ? KDT_ERR_CUDA : engine->tick();
      if (s == KDT_OK) s = engine->done_slots(running, &done);
      if (s == KDT_OK && !done.empty()) s = engine->finalize(done, &st, &lv);
      bool recovered = true;
      if (s != KDT_OK) {
        // The engine's tables no longer describe the trees in flight: clear
        // them (after whatever the failed step left on the stream) so that
        // queued requests can start from scratch.
        recovered = !kdt::fault_take(KDT_FAULT_SERVER_RESET) && engine->reset() == KDT_OK &&
                    cudaStreamSynchronize(stream) == cudaSuccess;
        if (!recovered) (void)cudaGetLastError();
      }
      std::lock_guard<std::mutex> lk(mu);
      info.ticks += 1;
      if (s != KDT_OK) {
        // an engine failure ends every request in flight with that status;
        // if the engine could not be cleared, the queued ones too
        info.engine_failures += 1;
        done = running;
        st.assign(done.size(), s);
        lv.assign(done.size(), 0);
        if (!recovered) {
          fatal = s;
          for (Request* r : queue) {
            r->status = s;
            r->t_done = now_ms();
            r->state = 2;
            info.completed += 1;
          }
          queue.clear();
          cv_done.notify_all();
        }
      }
      for (size_t i = 0; i < done.size(); ++i) {
        Request* r = slot_req[done[i]];
        if (!r) continue;
        r->status = st[i];
        r->levels = r->desc.params.depth > 0 ? r->desc.params.depth : lv[i];
        r->t_done = now_ms();
        r->state = 2;
        slot_req[done[i]] = nullptr;
        free_slots.push_back(done[i]);
        arena->release(r->off, r->plan.bytes);
        take(r->needs, -1);
        info.completed += 1;
      }
      if (!done.empty()) cv_done.notify_all();
    }
  }
};

extern "C" {

kdt_status kdt_server_create(size_t mem_budget_bytes, int32_t max_trees_in_flight, kdt_server** out) {
  if (!out || max_trees_in_flight < 1 || mem_budget_bytes < ((size_t)64 << 20)) return KDT_ERR_INVALID_ARG;
  kdt_server* sv = new kdt_server();
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete sv;
    return KDT_ERR_CUDA;
  }
  sv->budget = mem_budget_bytes;
  sv->max_slots = (uint32_t)max_trees_in_flight;
  // Shared tables sized for the points the budget can hold (a tree needs at
  // least 2*(4d + 4) + 4 >= 20 bytes of working memory per point).
  kdt::StepNeeds cap;
  cap.points = mem_budget_bytes / 24;
  cap.maxB = cap.points / 512 + 2 * (uint64_t)max_trees_in_flight;
  cap.cap_small = cap.points / 16 + 2 * (uint64_t)max_trees_in_flight;
  cap.nseg = cap.maxB * 64;
  cap.max_trees = sv->max_slots;
  cap.slice_cells = 8192;
  cap.widest = true;
  cap.max_d = KDT_MAX_DIMS;
  sv->step = kdt::plan_step(cap);
  sv->tree_base = align_up(sv->step.bytes);
  if (sv->tree_base + ((size_t)16 << 20) > mem_budget_bytes) {
    delete sv;
    return KDT_ERR_CAPACITY;
  }
  if (kdt::dev_malloc((void**)&sv->mem, mem_budget_bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    delete sv;
    return KDT_ERR_OOM;
  }
  if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(sv->mem);
    delete sv;
    return KDT_ERR_CUDA;
  }
  sv->arena = new Arena(mem_budget_bytes - sv->tree_base);
  sv->engine = new kdt::Engine(sv->step, sv->mem, sv->stream);
  kdt_status s = sv->engine->reset();
  if (s == KDT_OK && cudaStreamSynchronize(sv->stream) != cudaSuccess) s = KDT_ERR_CUDA;
  if (s != KDT_OK) {
    delete sv->engine;
    delete sv->arena;
    cudaStreamDestroy(sv->stream);
    cudaFree(sv->mem);
    delete sv;
    return s;
  }
  sv->slot_req.assign(sv->max_slots, nullptr);
  for (uint32_t k = sv->max_slots; k-- > 0;) sv->free_slots.push_back(k);
  sv->worker = std::thread([sv] { sv->run(); });
  *out = sv;
  return KDT_OK;
}

kdt_status kdt_server_submit(kdt_server* sv, const kdt_tree_desc* req, uint64_t* ticket) {
  if (!sv || !req || !ticket) return KDT_ERR_INVALID_ARG;
  const kdt_status v = kdt::validate_params(&req->params);
  if (v != KDT_OK) return v;
  if (req->params.fourier_j != 0) return KDT_ERR_INVALID_ARG;  // plain builds only
  const kdt_params& p = req->params;
  const int L_cap = p.depth > 0 ? p.depth : p.max_levels;
  if ((p.n > 0 && (!req->points || !req->out_perm)) || !req->out_node_offsets ||
      (L_cap > 0 && (!req->out_split_vals || !req->out_split_dims)))
    return KDT_ERR_INVALID_ARG;
  Request* r = new Request();
  r->desc = *req;
  r->plan = kdt::plan_tree(p);
  r->needs.add(p, r->plan);
  r->t_submit = now_ms();
  std::lock_guard<std::mutex> lk(sv->mu);
  // a request that could never fit is refused now
  const kdt::StepNeeds& cap = sv->step.needs;
  if (r->plan.bytes > sv->budget - sv->tree_base || r->needs.points > cap.points || r->needs.maxB > cap.maxB ||
      r->needs.cap_small > cap.cap_small || r->needs.nseg > cap.nseg) {
    delete r;
    return KDT_ERR_CAPACITY;
  }
  if (sv->fatal != KDT_OK) {
    delete r;
    return sv->fatal;
  }
  r->ticket = sv->next_ticket++;
  sv->requests[r->ticket] = r;
  sv->queue.push_back(r);
  sv->info.submitted += 1;
  *ticket = r->ticket;
  sv->cv_work.notify_one();
  return KDT_OK;
}

kdt_status kdt_server_poll(kdt_server* sv, uint64_t ticket, int32_t wait_ms, kdt_status* result,
                           int32_t* levels, double* latency_ms) {
  if (!sv) return KDT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->requests.find(ticket);
  if (it == sv->requests.end()) return KDT_ERR_NOT_FOUND;
  Request* r = it->second;
  if (r->state != 2 && wait_ms != 0) {
    const auto pred = [r] { return r->state == 2; };
    if (wait_ms < 0)
      sv->cv_done.wait(lk, pred);
    else
      sv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), pred);
  }
  if (r->state != 2) return KDT_ERR_BUSY;
  if (result) *result = r->status;
  if (levels) *levels = r->levels;
  if (latency_ms) *latency_ms = r->t_done - r->t_submit;
  sv->requests.erase(it);
  delete r;
  return KDT_OK;
}

kdt_status kdt_server_cancel(kdt_server* sv, uint64_t ticket) {
  if (!sv) return KDT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->requests.find(ticket);
  if (it == sv->requests.end()) return KDT_ERR_NOT_FOUND;
  Request* r = it->second;
  if (r->state != 0) return KDT_ERR_BUSY;  // admitted or finished: poll it
  for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q)
    if (*q == r) {
      sv->queue.erase(q);
      break;
    }
  r->status = KDT_ERR_CANCELLED;
  r->t_done = now_ms();
  r->state = 2;
  sv->info.cancelled += 1;
  sv->info.completed += 1;
  sv->cv_done.notify_all();
  return KDT_OK;
}

kdt_status kdt_server_stats(kdt_server* sv, kdt_server_info* out) {
  if (!sv || !out) return KDT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->info;
  out->arena_bytes = sv->budget;
  return KDT_OK;
}

kdt_status kdt_server_destroy(kdt_server* sv) {
  if (!sv) return KDT_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    // requests still queued are dropped; those in flight finish first
    for (Request* r : sv->queue) {
      sv->requests.erase(r->ticket);
      delete r;
    }
    sv->queue.clear();
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  cudaStreamSynchronize(sv->stream);
  for (auto& kv : sv->requests) delete kv.second;
  delete sv->engine;
  delete sv->arena;
  cudaStreamDestroy(sv->stream);
  cudaFree(sv->mem);
  delete sv;
  return KDT_OK;
}

}  // extern "C"
