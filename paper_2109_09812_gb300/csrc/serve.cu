// Serving runtime: a request loop with continuous batching on top of reindex_meshes.
//
// Clients submit re-indexing requests (device-resident meshes) at any time.  A scheduler thread
// keeps up to `num_streams` batches in flight on separate CUDA streams.  Whenever a stream is
// free, it forms the next batch from the pending requests in arrival order (one stride / arity
// class per batch, at most max_batch_requests), admits it only if its memory fits in the part
// of the HBM budget that is free, gathers the meshes into a contiguous staging region, and
// launches one reindex_meshes sequence.  Requests that arrive while batches run are therefore
// admitted as soon as a stream and memory free up, and their work overlaps on the device.
//
// Memory: one arena of hbm_budget_bytes is allocated at creation; a first-fit allocator with
// coalescing hands out regions.  A batch holds (a) its workspace, returned to the arena when the
// batch finishes, and (b) its staging region, which also holds the outputs (the unique vertices
// and the remapped indices, computed in place): the results are handed to the clients as
// pointers into it, and it returns to the arena when every request of the batch is released.
//
// Faults: a batch whose device run reports an error (e.g. an index out of range in one request)
// is split, and its requests are re-run one per batch, so that only the faulty request fails.
// Completion is signalled by a host callback enqueued after each batch (no CUDA call inside it).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"
#include "reindex.h"

namespace reindex {

static double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing; offsets are 256-byte aligned.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) {
    if (size) free_[0] = size;
  }
  // Returns the offset, or SIZE_MAX if no free range is large enough.
  size_t alloc(size_t bytes) {
    bytes = align_up(std::max<size_t>(bytes, 1), 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        used_[off] = bytes;
        in_use_ += bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t start = off, len = u->second;
    in_use_ -= len;
    used_.erase(u);
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + len) {
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = len;
  }
  size_t in_use() const { return in_use_; }
  size_t size() const { return size_; }
  size_t largest_free() const {
    size_t m = 0;
    for (auto& f : free_) m = std::max(m, f.second);
    return m;
  }
  size_t free_ranges() const { return free_.size(); }

 private:
  size_t size_, in_use_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  std::map<size_t, size_t> used_;  // offset -> length
};

struct Req {
  int64_t id;
  reindex_request r;
  double submit_us = 0, start_us = 0, done_us = 0;
  reindex_status status = REINDEX_OK;
  int64_t nOut = 0;
  const void* out_vtx = nullptr;
  const int32_t* out_idx = nullptr;
  int64_t batch = -1;      // batch holding the outputs
  bool isolated = false;   // re-run alone after its batch failed
};

struct Batch {
  int64_t id;
  std::vector<int64_t> reqs;
  int slot = -1;
  size_t stage_off = SIZE_MAX, ws_off = SIZE_MAX;
  int refs = 0;            // requests whose outputs still point into the staging region
  std::atomic<bool> done{false};   // set by the completion callback
  std::atomic<double> done_us{0};
  bool finished = false;           // completion processed by the scheduler
  int64_t* h_off = nullptr;  // pinned buffer of the stream slot: [voff | eoff | outOff], n+1 each
};

}  // namespace reindex

struct reindex_server {
  reindex::Arena arena{0};
  reindex_server_config cfg{};
  unsigned char* base = nullptr;  // device arena
  std::vector<cudaStream_t> streams;
  std::vector<int64_t> slot_batch;  // batch running on each stream slot, or -1
  std::vector<int64_t*> slot_pinned;  // per slot: 3 * (max_batch_requests + 1) int64, page-locked
  std::mutex mu;
  std::condition_variable cv;       // scheduler wake-up
  std::condition_variable cv_done;  // completions
  std::deque<int64_t> pending;
  std::map<int64_t, std::unique_ptr<reindex::Req>> reqs;
  std::map<int64_t, std::unique_ptr<reindex::Batch>> batches;
  std::deque<int64_t> completed;  // finished, not yet polled
  int64_t next_req = 1, next_batch = 1;
  int64_t outstanding = 0;        // submitted and not yet finished
  bool stop = false;
  std::thread worker;
  reindex_server_stats stats{};
};

namespace reindex {

struct CallbackArg {
  reindex_server* s;
  Batch* b;  // stays alive until the scheduler has processed its completion
};

// Runs on a CUDA driver thread after the batch's last operation.  It takes no lock (the scheduler
// may hold its mutex while it enqueues work, and an enqueue can wait for the stream to drain),
// it only publishes the completion time and wakes the scheduler.
static void CUDART_CB on_batch_done(void* p) {
  CallbackArg* a = static_cast<CallbackArg*>(p);
  a->b->done_us.store(now_us());
  a->b->done.store(true, std::memory_order_release);
  a->s->cv.notify_all();
  delete a;
}

static size_t request_stage_bytes(const reindex_request& r) {
  const int64_t M = r.nElem * r.idxPerElem;
  const int64_t cap = std::min<int64_t>(r.nVtx, M);
  return align_up((size_t)r.nVtx * r.vtxStrideBytes, 256) + align_up((size_t)M * 4, 256) +
         align_up((size_t)cap * r.vtxStrideBytes, 256);
}

// Sizes of a batch made of the given requests (staging incl. outputs and offsets; workspace).
static void batch_bytes(reindex_server* s, const std::vector<int64_t>& ids, size_t* stage, size_t* ws) {
  int64_t N = 0, E = 0, cap = 0;
  int S = 0, k = 0;
  for (int64_t id : ids) {
    const reindex_request& r = s->reqs[id]->r;
    N += r.nVtx;
    E += r.nElem;
    cap += std::min<int64_t>(r.nVtx, r.nElem * r.idxPerElem);
    S = r.vtxStrideBytes;
    k = r.idxPerElem;
  }
  const size_t n = ids.size();
  *stage = align_up((size_t)N * S, 256) + align_up((size_t)E * k * 4, 256) + align_up((size_t)cap * S, 256) +
           3 * align_up((n + 1) * 8, 256);
  *ws = reindex_meshes_workspace_size((int)n, N, S, E, k);
}

// Launch one batch on stream slot `slot` (caller holds the lock).  Returns false if the batch
// does not fit the free arena (nothing is changed then).
static bool launch_batch(reindex_server* s, const std::vector<int64_t>& ids, int slot) {
  size_t stage_b = 0, ws_b = 0;
  batch_bytes(s, ids, &stage_b, &ws_b);
  const size_t stage_off = s->arena.alloc(stage_b);
  if (stage_off == SIZE_MAX) return false;
  const size_t ws_off = s->arena.alloc(ws_b);
  if (ws_off == SIZE_MAX) {
    s->arena.release(stage_off);
    return false;
  }
  auto b = std::make_unique<Batch>();
  b->id = s->next_batch++;
  b->reqs = ids;
  b->slot = slot;
  b->stage_off = stage_off;
  b->ws_off = ws_off;
  b->refs = (int)ids.size();
  const size_t n = ids.size();
  b->h_off = s->slot_pinned[slot];
  int64_t* hv = b->h_off;
  int64_t* he = b->h_off + (n + 1);
  const reindex_request& r0 = s->reqs[ids[0]]->r;
  const int S = r0.vtxStrideBytes, k = r0.idxPerElem;
  int64_t N = 0, E = 0, cap = 0;
  hv[0] = he[0] = 0;
  for (size_t m = 0; m < n; ++m) {
    const reindex_request& r = s->reqs[ids[m]]->r;
    N += r.nVtx;
    E += r.nElem;
    cap += std::min<int64_t>(r.nVtx, r.nElem * r.idxPerElem);
    hv[m + 1] = N;
    he[m + 1] = E;
  }
  unsigned char* st = s->base + stage_off;
  unsigned char* d_vtx = st;
  int32_t* d_idx = reinterpret_cast<int32_t*>(st + align_up((size_t)N * S, 256));
  unsigned char* d_out = reinterpret_cast<unsigned char*>(d_idx) + align_up((size_t)E * k * 4, 256);
  int64_t* d_off = reinterpret_cast<int64_t*>(d_out + align_up((size_t)cap * S, 256));  // voff, eoff, outOff
  const size_t offb = align_up((n + 1) * 8, 256);
  int64_t* d_voff = d_off;
  int64_t* d_eoff = reinterpret_cast<int64_t*>(reinterpret_cast<unsigned char*>(d_off) + offb);
  int64_t* d_oout = reinterpret_cast<int64_t*>(reinterpret_cast<unsigned char*>(d_off) + 2 * offb);
  cudaStream_t stm = s->streams[slot];
  const double t = now_us();
  for (size_t m = 0; m < n; ++m) {
    Req& q = *s->reqs[ids[m]];
    q.start_us = t;
    q.batch = b->id;
    if (q.r.nVtx) cudaMemcpyAsync(d_vtx + (size_t)hv[m] * S, q.r.vtx, (size_t)q.r.nVtx * S, cudaMemcpyDeviceToDevice, stm);
    if (q.r.nElem)
      cudaMemcpyAsync(d_idx + he[m] * k, q.r.idx, (size_t)q.r.nElem * k * 4, cudaMemcpyDeviceToDevice, stm);
  }
  cudaMemcpyAsync(d_voff, hv, (n + 1) * 8, cudaMemcpyHostToDevice, stm);
  cudaMemcpyAsync(d_eoff, he, (n + 1) * 8, cudaMemcpyHostToDevice, stm);
  reindex_status rs = reindex_meshes(d_vtx, d_voff, S, d_idx, d_eoff, k, (int)n, N, E, d_out, d_oout, d_idx,
                                     s->base + ws_off, ws_b, reinterpret_cast<reindex_stream_t>(stm));
  int64_t* hout = b->h_off + 2 * (n + 1);
  if (rs == REINDEX_OK) {
    cudaMemcpyAsync(hout, d_oout, (n + 1) * 8, cudaMemcpyDeviceToHost, stm);
  } else {  // refused on the host: report it as the batch's error
    for (size_t m = 0; m < n; ++m) hout[m] = 0;
    hout[n] = -(int64_t)rs;
  }
  cudaLaunchHostFunc(stm, on_batch_done, new CallbackArg{s, b.get()});
  for (size_t m = 0; m < n; ++m) {  // output pointers (vertex offsets are known after completion)
    Req& q = *s->reqs[ids[m]];
    q.out_idx = d_idx + he[m] * k;
    q.out_vtx = d_out;
  }
  s->slot_batch[slot] = b->id;
  s->stats.batches += 1;
  s->stats.requests_started += (int64_t)n;
  s->batches[b->id] = std::move(b);
  return true;
}

static void release_batch_ref(reindex_server* s, int64_t bid) {
  auto it = s->batches.find(bid);
  if (it == s->batches.end()) return;
  Batch& b = *it->second;
  if (--b.refs > 0) return;
  s->arena.release(b.stage_off);
  s->batches.erase(it);
}

// Finish a completed batch (caller holds the lock).
static void finish_batch(reindex_server* s, Batch& b) {
  const size_t n = b.reqs.size();
  const int64_t* out = b.h_off + 2 * (n + 1);
  s->arena.release(b.ws_off);
  b.ws_off = SIZE_MAX;
  b.finished = true;
  const double done_us = b.done_us.load();
  // Read the pinned offsets now: the slot (and its pinned buffer) is handed to the next batch.
  std::vector<int64_t> offs(out, out + n + 1);
  out = offs.data();
  s->slot_batch[b.slot] = -1;
  const bool failed = out[n] < 0;
  if (failed && n > 1) {  // isolate the faulty request: re-run every request on its own
    for (auto it = b.reqs.rbegin(); it != b.reqs.rend(); ++it) {
      Req& q = *s->reqs[*it];
      q.isolated = true;
      q.status = REINDEX_OK;
      q.batch = -1;
      s->pending.push_front(*it);
    }
    b.refs = 1;
    s->stats.batches_split += 1;
    release_batch_ref(s, b.id);
    return;
  }
  const int S = s->reqs[b.reqs[0]]->r.vtxStrideBytes;
  for (size_t m = 0; m < n; ++m) {
    Req& q = *s->reqs[b.reqs[m]];
    q.done_us = done_us;
    if (failed) {
      q.status = (reindex_status)(-out[n]);
      q.nOut = 0;
    } else if (q.status == REINDEX_OK) {
      q.nOut = out[m + 1] - out[m];
      q.out_vtx = static_cast<const unsigned char*>(q.out_vtx) + (size_t)out[m] * S;
    }
    s->completed.push_back(q.id);
    s->outstanding -= 1;
    s->stats.requests_done += 1;
    if (q.status != REINDEX_OK) s->stats.requests_failed += 1;
  }
}

static void scheduler(reindex_server* s) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool finished_any = false;
    for (auto& kv : s->batches) {
      Batch& b = *kv.second;
      if (!b.finished && b.done.load(std::memory_order_acquire)) {
        finish_batch(s, b);
        finished_any = true;
        break;  // finish_batch may erase batches; restart the scan
      }
    }
    if (finished_any) {
      s->cv_done.notify_all();
      continue;
    }
    if (s->stop && s->outstanding == 0) break;
    bool launched = false;
    for (int slot = 0; slot < (int)s->streams.size() && !s->pending.empty(); ++slot) {
      if (s->slot_batch[slot] >= 0) continue;
      // Continuous batching: everything pending of the head's class, in order, up to the cap and
      // as long as the batch fits the free part of the budget.
      const reindex_request& h = s->reqs[s->pending.front()]->r;
      std::vector<int64_t> ids;
      const bool alone = s->reqs[s->pending.front()]->isolated;
      for (int64_t id : s->pending) {
        const Req& q = *s->reqs[id];
        if (q.r.vtxStrideBytes != h.vtxStrideBytes || q.r.idxPerElem != h.idxPerElem || q.isolated != alone) continue;
        ids.push_back(id);
        size_t st = 0, ws = 0;
        batch_bytes(s, ids, &st, &ws);
        if (st + ws > s->arena.largest_free() || (int)ids.size() > s->cfg.max_batch_requests || (alone && ids.size() > 1)) {
          ids.pop_back();
          break;
        }
      }
      if (ids.empty()) break;  // the head does not fit yet: wait for memory
      if (!launch_batch(s, ids, slot)) {
        if (ids.size() == 1) break;
        ids.resize(ids.size() / 2);  // fragmentation: try a smaller batch once
        if (!launch_batch(s, ids, slot)) break;
      }
      for (int64_t id : ids) s->pending.erase(std::find(s->pending.begin(), s->pending.end(), id));
      launched = true;
    }
    if (launched) continue;
    s->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

}  // namespace reindex

using namespace reindex;

extern "C" {

reindex_status reindex_server_create(const reindex_server_config* cfg, reindex_server** out) {
  if (!cfg || !out || cfg->hbm_budget_bytes < (1u << 20)) return REINDEX_ERR_INVALID_ARG;
  auto s = std::make_unique<reindex_server>();
  s->cfg = *cfg;
  if (s->cfg.max_batch_requests < 1) s->cfg.max_batch_requests = 256;
  if (s->cfg.num_streams < 1) s->cfg.num_streams = 2;
  if (cudaSetDevice(s->cfg.device) != cudaSuccess) return REINDEX_ERR_CUDA;
  const size_t budget = align_up(s->cfg.hbm_budget_bytes, 256);
  if (cudaMalloc(&s->base, budget) != cudaSuccess) return REINDEX_ERR_OOM;
  s->arena = Arena(budget);
  for (int i = 0; i < s->cfg.num_streams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return REINDEX_ERR_CUDA;
    s->streams.push_back(st);
    s->slot_batch.push_back(-1);
    int64_t* pin = nullptr;
    if (cudaMallocHost(&pin, 3 * (size_t)(s->cfg.max_batch_requests + 1) * sizeof(int64_t)) != cudaSuccess)
      return REINDEX_ERR_OOM;
    s->slot_pinned.push_back(pin);
  }
  reindex_server* raw = s.release();
  raw->worker = std::thread(scheduler, raw);
  *out = raw;
  return REINDEX_OK;
}

reindex_status reindex_server_submit(reindex_server* s, const reindex_request* req, int64_t* id_out) {
  if (!s || !req || !id_out) return REINDEX_ERR_INVALID_ARG;
  const int S = req->vtxStrideBytes;
  if (S != 4 && S != 8 && S != 12 && S != 16) return REINDEX_ERR_UNSUPPORTED;
  if (req->nVtx < 0 || req->nElem < 0 || req->idxPerElem < 1) return REINDEX_ERR_INVALID_ARG;
  if ((req->nVtx && !req->vtx) || (req->nElem && !req->idx)) return REINDEX_ERR_INVALID_ARG;
  if (req->nElem > (int64_t)INT32_MAX / req->idxPerElem || req->nVtx > kMaxCount) return REINDEX_ERR_UNSUPPORTED;
  auto q = std::make_unique<Req>();
  q->r = *req;
  q->submit_us = now_us();
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return REINDEX_ERR_INVALID_ARG;
    q->id = s->next_req++;
    // Admission: a request that could never fit the budget, even alone, is refused now.
    std::vector<int64_t> one{q->id};
    s->reqs[q->id] = std::move(q);
    size_t st = 0, ws = 0;
    batch_bytes(s, one, &st, &ws);
    if (st + ws > s->arena.size()) {
      s->reqs.erase(one[0]);
      s->stats.requests_rejected += 1;
      return REINDEX_ERR_OOM;
    }
    *id_out = one[0];
    s->pending.push_back(one[0]);
    s->outstanding += 1;
    s->stats.requests_submitted += 1;
  }
  s->cv.notify_all();
  return REINDEX_OK;
}

int reindex_server_poll(reindex_server* s, reindex_result* out, int max_results, int wait_ms) {
  if (!s || !out || max_results < 1) return -1;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->completed.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->completed.empty(); });
  int n = 0;
  while (n < max_results && !s->completed.empty()) {
    const int64_t id = s->completed.front();
    s->completed.pop_front();
    const Req& q = *s->reqs[id];
    reindex_result& r = out[n++];
    r.id = id;
    r.status = q.status;
    r.nVtxOut = q.nOut;
    r.out_vtx = q.status == REINDEX_OK ? q.out_vtx : nullptr;
    r.out_idx = q.status == REINDEX_OK ? q.out_idx : nullptr;
    r.submit_us = q.submit_us;
    r.start_us = q.start_us;
    r.done_us = q.done_us;
  }
  return n;
}

reindex_status reindex_server_release(reindex_server* s, int64_t id) {
  if (!s) return REINDEX_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second->done_us == 0) return REINDEX_ERR_INVALID_ARG;
  const int64_t bid = it->second->batch;
  s->reqs.erase(it);
  if (bid >= 0) release_batch_ref(s, bid);
  s->cv.notify_all();  // memory may have freed up
  return REINDEX_OK;
}

reindex_status reindex_server_drain(reindex_server* s, int timeout_ms) {
  if (!s) return REINDEX_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return s->outstanding == 0; });
  return ok ? REINDEX_OK : REINDEX_ERR_TIMEOUT;
}

reindex_status reindex_server_get_stats(reindex_server* s, reindex_server_stats* out) {
  if (!s || !out) return REINDEX_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->stats;
  out->arena_bytes_in_use = (int64_t)s->arena.in_use();
  out->pending = (int64_t)s->pending.size();
  return REINDEX_OK;
}

void reindex_server_destroy(reindex_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    s->pending.clear();  // requests not yet started are dropped
  }
  s->cv.notify_all();
  {
    // requests dropped from the queue no longer count as outstanding
    std::lock_guard<std::mutex> g(s->mu);
    int64_t running = 0;
    for (auto& kv : s->batches)
      if (!kv.second->finished) running += (int64_t)kv.second->reqs.size();
    s->outstanding = running;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (int64_t* pin : s->slot_pinned) cudaFreeHost(pin);
  cudaFree(s->base);
  delete s;
}

// Host-only check of the arena allocator against a brute-force model (no CUDA calls): random
// allocations and releases; returns the number of inconsistencies found.
int reindex_debug_arena_check(uint64_t seed, int ops, size_t size) {
  Arena a(size);
  std::vector<std::pair<size_t, size_t>> live;  // (offset, bytes)
  uint64_t x = seed * 0x9E3779B97F4A7C15ull + 1;
  auto rnd = [&]() {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    return x;
  };
  int bad = 0;
  for (int i = 0; i < ops; ++i) {
    if (live.empty() || rnd() % 3) {
      const size_t bytes = 1 + rnd() % (size / 16 + 1);
      const size_t off = a.alloc(bytes);
      const size_t rb = align_up(bytes, 256);
      if (off == SIZE_MAX) {
        // must really be full: no gap of rb bytes between live ranges
        std::vector<std::pair<size_t, size_t>> v = live;
        std::sort(v.begin(), v.end());
        size_t cur = 0, gap = 0;
        for (auto& p : v) {
          gap = std::max(gap, p.first - cur);
          cur = p.first + p.second;
        }
        gap = std::max(gap, size - cur);
        if (gap >= rb) ++bad;
        continue;
      }
      if (off % 256 || off + rb > size) ++bad;
      for (auto& p : live)
        if (off < p.first + p.second && p.first < off + rb) ++bad;  // overlap
      live.push_back({off, rb});
    } else {
      const size_t j = rnd() % live.size();
      a.release(live[j].first);
      live.erase(live.begin() + j);
    }
    size_t sum = 0;
    for (auto& p : live) sum += p.second;
    if (sum != a.in_use()) ++bad;
  }
  for (auto& p : live) a.release(p.first);
  if (a.in_use() != 0 || a.free_ranges() != (size ? 1u : 0u) || a.largest_free() != size) ++bad;
  return bad;
}

}  // extern "C"
