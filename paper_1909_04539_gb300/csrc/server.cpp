// Request server: continuous batching of shared-LHS solves on one GPU.
//
// Requests arrive with host buffers and a resident factorised LHS.  A worker
// thread admits queued requests in arrival order while their device memory
// fits in an arena of fixed size (the HBM budget), gathers every newly
// admitted request into one batch, and runs the batch on one of a few
// streams: host-to-device copies, one replay of a captured CUDA graph (the
// work-list copy and one grouped persistent launch covering all requests of
// the batch), device-to-host copies, an event.  Batches on different streams
// overlap on the device; requests that arrive while batches run are admitted
// as soon as memory and a stream are free.  Completion is observed by polling
// the batch events; latency is host submission to host-observed completion.
// No device-side waits are involved: a batch is a finite work list.
//
// Tail latency: requests are split into two size classes (arena bytes up to
// kSmallBytes, and larger) with a queue each, so a large request waiting for
// memory never holds back small ones, and a batch holds one class only.  With
// two or more streams, stream 0 runs only small-request batches, so small
// requests never queue behind the multi-millisecond copies of a large batch.
// Inside a batch the copies go smallest first and every request has its own
// completion event after its device-to-host copy: it finishes as soon as its
// own results are back, not when the whole batch is.  Copies go in pieces of
// 8 MiB, at most four of a stream in flight (the launcher waits for the piece
// issued four before), so a large batch never queues more than 32 MiB ahead
// of another stream's copies on the copy engines.  Each stream has a
// launcher thread that issues its batches' copies and graph replay, so the
// worker thread, which admits requests and observes completions, never waits
// while the hundreds of copy pieces of a large batch are queued (issuing them
// can block once the stream's command queue is full).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "serve.h"

namespace bs {
namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device allocation; blocks are 256-byte aligned.
class Arena {
 public:
  void init(size_t size) {
    size_ = size;
    free_.clear();
    free_[0] = size;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        if (used_ > peak_) peak_ = used_;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
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
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t size() const { return size_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0, peak_ = 0;
};

enum ReqState { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_CANCELLED = 3, RQ_FAILED = 4 };

// arena bytes up to which a request is "small"
constexpr size_t kSmallBytes = size_t(16) << 20;
// host<->device copies are issued in pieces of at most this many bytes, so
// that the copy engines can interleave other streams' (small) copies with
// a large request's instead of running them after it
constexpr size_t kCopyChunk = size_t(8) << 20;

// Copy pieces of one stream in flight at a time: a piece is issued only after
// the one issued kPaceWindow pieces earlier has finished, so that a large
// batch never has more than kPaceWindow * kCopyChunk bytes queued before
// another stream's copies (a few hundred microseconds of copy-engine work).
constexpr int kPaceWindow = 4;

// Per stream: an event after each piece issued, in a ring.
struct Pacer {
  cudaEvent_t ev[kPaceWindow] = {};
  int64_t issued = 0;
};

// Waits (host side, bounded) for the piece issued kPaceWindow pieces ago.
void pace_wait(Pacer& p) {
  if (p.issued < kPaceWindow) return;
  cudaEvent_t ev = p.ev[p.issued % kPaceWindow];
  const auto t0 = std::chrono::steady_clock::now();
  while (cudaEventQuery(ev) == cudaErrorNotReady) {
    // a wait that long means the device is stuck; stop pacing this piece
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60)) return;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

cudaError_t copy_chunked(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t st,
                         Pacer& p) {
  cudaError_t e = cudaSuccess;
  for (size_t o = 0; o < bytes && e == cudaSuccess; o += kCopyChunk) {
    pace_wait(p);
    e = cudaMemcpyAsync(static_cast<char*>(dst) + o, static_cast<const char*>(src) + o,
                        bytes - o < kCopyChunk ? bytes - o : kCopyChunk, kind, st);
    if (e == cudaSuccess) e = cudaEventRecord(p.ev[p.issued % kPaceWindow], st);
    p.issued++;
  }
  return e;
}

struct Req {
  bs_handle h;
  const void* hB;
  void* hX;
  int mode;
  int64_t M;
  size_t bytes;      // arena bytes
  size_t off;        // arena offset
  double t_submit = 0, t_done = 0;
  int state = RQ_QUEUED;
  bool fail_on_admit = false;
  bool small = true;
};

struct Slot {
  cudaStream_t st = nullptr;
  unsigned char* h_work = nullptr;  // pinned
  unsigned char* d_work = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  bool small_only = false;          // runs small-request batches only
  std::vector<int64_t> reqs;        // the batch's requests, in copy order
  std::vector<cudaEvent_t> ev;      // per request: its device-to-host copy done
  std::vector<char> finished;       // per request: completion recorded
  // launcher thread: busy && !issued while the batch's copies and replay are
  // being queued on the stream (rp: the batch's requests); launch_err is its
  // outcome
  std::thread launcher;
  bool issued = false;
  std::vector<Req*> rp;
  cudaError_t launch_err = cudaSuccess;
  int recorded = 0;  // requests whose completion event is queued (under the server lock)
  Pacer pace;        // the stream's copy pieces in flight
};

}  // namespace
}  // namespace bs

struct bs_server_s {
  int device = 0;
  char* arena_base = nullptr;
  bs::Arena arena;
  std::vector<bs::Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> queue;        // small requests, arrival order
  std::deque<int64_t> queue_large;  // large requests, arrival order
  std::unordered_map<int64_t, bs::Req> reqs;
  int64_t next_id = 1;
  std::thread worker;
  bool stop = false;
  bool paused = false;
  cudaError_t sticky = cudaSuccess;
  // statistics
  int64_t batches = 0, completed = 0, failed = 0, max_batch_reqs = 0, max_concurrent = 0;
};

namespace bs {
namespace {

size_t req_bytes(int width, int64_t N, int mode, int64_t M) {
  (void)width;
  const size_t nm = (size_t)N * (size_t)M;
  return mode == SERVE_F64 ? nm * 8 : nm * 4 + nm * 8;
}

// Admit queued requests of one class (in arrival order) while they fit;
// returns the admitted ids.
std::vector<int64_t> admit(bs_server s, bool small) {
  std::vector<int64_t> out;
  std::deque<int64_t>& queue = small ? s->queue : s->queue_large;
  int tiles = 0;
  while (!queue.empty() && (int)out.size() < kGroupMaxReq) {
    const int64_t id = queue.front();
    Req& r = s->reqs[id];
    if (r.state == RQ_CANCELLED) {
      queue.pop_front();
      continue;
    }
    const int t = (int)((r.M + 31) / 32);
    if (tiles + t > kGroupMaxTiles) break;
    size_t off = 0;
    if (!s->arena.alloc(r.bytes, &off)) break;  // wait for memory (arrival order is kept)
    queue.pop_front();
    r.off = off;
    if (r.fail_on_admit) {  // host-side fault injection for tests
      s->arena.release(off, r.bytes);
      r.state = RQ_FAILED;
      r.t_done = now_s();
      s->failed++;
      handle_unref(r.h);
      continue;
    }
    r.state = RQ_RUNNING;
    tiles += t;
    out.push_back(id);
  }
  // copies smallest first, so that small requests' results come back first
  std::stable_sort(out.begin(), out.end(), [&](int64_t a, int64_t b) { return s->reqs[a].bytes < s->reqs[b].bytes; });
  return out;
}

// Copies in, the grouped launch and copies out of one batch on the slot's
// stream.  Called without the server lock: rp are the batch's requests
// (their entries are not modified by other threads once admitted).
cudaError_t launch_batch(bs_server s, Slot& sl, const std::vector<Req*>& rp) {
  GHeader* hdr = reinterpret_cast<GHeader*>(sl.h_work);
  GReq* greq = reinterpret_cast<GReq*>(sl.h_work + kGroupReqOff);
  GTile* gt = reinterpret_cast<GTile*>(sl.h_work + kGroupTileOff);
  int nt = 0;
  cudaError_t e = cudaSuccess;
  for (size_t q = 0; q < rp.size() && e == cudaSuccess; q++) {
    Req& r = *rp[q];
    const bs_handle h = r.h;
    const size_t nm = (size_t)h->N * (size_t)r.M;
    char* dB = s->arena_base + r.off;
    GReq g{};
    g.c64 = h->plan[0].c64;
    g.c32 = h->plan[0].c32;
    g.lu_hi = h->lu_hi;
    g.lu_lo = h->lu_lo;
    g.dfrec = h->plan[0].dfrec;
    g.pairs = df_eligible(h->plan[0], BS_INTERLEAVED) ? 1 : 0;
    g.M = r.M;
    g.N = (int)h->N;
    g.width = h->width;
    g.mode = r.mode;
    if (r.mode == SERVE_F64) {
      g.B = dB;
      g.X = reinterpret_cast<double*>(dB);
      e = copy_chunked(dB, r.hB, nm * 8, cudaMemcpyHostToDevice, sl.st, sl.pace);
    } else {
      g.X = reinterpret_cast<double*>(dB);                   // nm * 8 bytes
      g.B = dB + nm * 8;                                     // nm * 4 bytes
      e = copy_chunked(g.B, r.hB, nm * 4, cudaMemcpyHostToDevice, sl.st, sl.pace);
    }
    greq[q] = g;
    for (int64_t j0 = 0; j0 < r.M; j0 += 32) gt[nt++] = GTile{(int)q, (int)j0};
  }
  hdr->n_req = (int)rp.size();
  hdr->n_tiles = nt;
  if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec, sl.st);
  while (sl.ev.size() < rp.size() && e == cudaSuccess) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) sl.ev.push_back(ev);
  }
  for (size_t q = 0; q < rp.size() && e == cudaSuccess; q++) {
    Req& r = *rp[q];
    const size_t nm = (size_t)r.h->N * (size_t)r.M;
    e = copy_chunked(r.hX, s->arena_base + r.off, nm * 8, cudaMemcpyDeviceToHost, sl.st, sl.pace);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev[q], sl.st);
    if (e == cudaSuccess) {  // the worker may poll this request from now on
      std::lock_guard<std::mutex> lk(s->mu);
      sl.recorded = (int)q + 1;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.st);
  return e;
}

// Records a request's end: its arena bytes go back, its handle is unpinned.
void finish_request(bs_server s, Req& r, bool ok, double t) {
  s->arena.release(r.off, r.bytes);
  r.t_done = t;
  if (ok) {
    r.state = RQ_DONE;
    s->completed++;
  } else {
    r.state = RQ_FAILED;
    s->failed++;
  }
  handle_unref(r.h);
}

void worker_loop(bs_server s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progressed = false;
    // completions: each request as soon as its own copy back is done; the
    // slot when the whole batch is
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      if (sl.issued && sl.launch_err != cudaSuccess) {  // the rest of this batch cannot be trusted: fail it
        s->sticky = sl.launch_err;
        const double t = now_s();
        for (size_t k = 0; k < sl.reqs.size(); k++)
          if (!sl.finished[k]) finish_request(s, s->reqs[sl.reqs[k]], false, t);
        sl.reqs.clear();
        sl.finished.clear();
        sl.rp.clear();
        sl.busy = false;
        progressed = true;
        continue;
      }
      // requests whose completion event the launcher has queued (it may
      // still be issuing later copies of the batch)
      for (size_t q = 0; q < (size_t)sl.recorded; q++) {
        if (sl.finished[q]) continue;
        const cudaError_t eq = cudaEventQuery(sl.ev[q]);
        if (eq == cudaErrorNotReady) break;  // later copies of the batch are not done either
        if (eq != cudaSuccess) break;        // the batch event reports the failure below
        finish_request(s, s->reqs[sl.reqs[q]], true, now_s());
        sl.finished[q] = 1;
        progressed = true;
      }
      if (!sl.issued) continue;  // the batch event is not queued yet
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      const double t = now_s();
      for (size_t k = 0; k < sl.reqs.size(); k++)
        if (!sl.finished[k]) finish_request(s, s->reqs[sl.reqs[k]], q == cudaSuccess, t);
      if (q != cudaSuccess) s->sticky = q;
      sl.reqs.clear();
      sl.finished.clear();
      sl.rp.clear();
      sl.busy = false;
      progressed = true;
    }
    if (progressed) s->cv.notify_all();
    // admission and launch
    if (!s->paused) {
      for (Slot& sl : s->slots) {
        if (sl.busy) continue;
        // the reserved slot takes small requests; the others the class whose
        // oldest queued request came first (falling back to the other class)
        const bool has_small = !s->queue.empty(), has_large = !s->queue_large.empty();
        if (!has_small && (!has_large || sl.small_only)) continue;
        bool small = has_small;
        if (!sl.small_only && has_large && (!has_small || s->queue_large.front() < s->queue.front())) small = false;
        std::vector<int64_t> ids = admit(s, small);
        if (ids.empty() && !sl.small_only && has_small && has_large) ids = admit(s, !small);
        if (ids.empty()) {
          s->cv.notify_all();  // failures injected at admission are final
          continue;
        }
        // the slot's launcher thread queues the copies and the graph replay
        // without the lock (the slot and the admitted requests belong to it
        // until it sets `issued`: cancel and release refuse admitted
        // requests, and map entries keep their addresses)
        sl.rp.clear();
        for (int64_t id : ids) sl.rp.push_back(&s->reqs.find(id)->second);
        sl.reqs = ids;
        sl.finished.assign(ids.size(), 0);
        sl.issued = false;
        sl.recorded = 0;
        sl.launch_err = cudaSuccess;
        sl.busy = true;
        progressed = true;
        s->batches++;
        s->cv.notify_all();  // wakes the slot's launcher
        if ((int64_t)ids.size() > s->max_batch_reqs) s->max_batch_reqs = (int64_t)ids.size();
      }
      int busy = 0;
      for (Slot& sl : s->slots) busy += sl.busy;
      if (busy > s->max_concurrent) s->max_concurrent = busy;
    }
    bool any_busy = false;
    for (Slot& sl : s->slots) any_busy |= sl.busy;
    if (!progressed) {
      if (any_busy)
        s->cv.wait_for(lk, std::chrono::microseconds(20));
      else
        s->cv.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

// One per slot: queues each batch handed to the slot (busy && !issued).
void launcher_loop(bs_server s, Slot* sl) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv.wait(lk, [&] { return s->stop || (sl->busy && !sl->issued); });
    if (!(sl->busy && !sl->issued)) break;  // stopping, nothing handed over
    const std::vector<Req*> rp = sl->rp;
    lk.unlock();
    cudaError_t e = launch_batch(s, *sl, rp);
    if (e != cudaSuccess) cudaStreamSynchronize(sl->st);
    lk.lock();
    sl->launch_err = e;
    sl->issued = true;
    s->cv.notify_all();
  }
}

void destroy_server(bs_server s) {
  for (Slot& sl : s->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.exec) cudaGraphExecDestroy(sl.exec);
    if (sl.done) cudaEventDestroy(sl.done);
    for (cudaEvent_t ev : sl.ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : sl.pace.ev)
      if (ev) cudaEventDestroy(ev);
    if (sl.h_work) cudaFreeHost(sl.h_work);
    if (sl.d_work) cudaFree(sl.d_work);
    if (sl.st) cudaStreamDestroy(sl.st);
  }
  if (s->arena_base) cudaFree(s->arena_base);
  // requests that never finished (dropped from the queue) unpin their handles
  for (auto& kv : s->reqs)
    if (kv.second.state == RQ_QUEUED || kv.second.state == RQ_RUNNING) handle_unref(kv.second.h);
  delete s;
}

}  // namespace
}  // namespace bs

using namespace bs;

extern "C" {

bs_status bs_server_create(size_t hbm_budget_bytes, int n_streams, bs_server* out) {
  if (!out) return set_error(BS_EINVAL, "bs_server_create: out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes < 4096) return set_error(BS_EINVAL, "bs_server_create: budget too small");
  if (n_streams < 1 || n_streams > 16) return set_error(BS_EINVAL, "bs_server_create: n_streams must be 1..16");
  bs_server s = new bs_server_s();
  cudaGetDevice(&s->device);
  cudaError_t e = cudaMalloc(&s->arena_base, hbm_budget_bytes);
  if (e != cudaSuccess) {
    delete s;
    return set_error(BS_ENOMEM, "bs_server_create: cannot reserve the HBM budget");
  }
  s->arena.init(hbm_budget_bytes);
  s->slots.resize(n_streams);
  if (n_streams >= 2) s->slots[0].small_only = true;
  const int grid = grouped_grid();
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  for (Slot& sl : s->slots) {
    // the small-request stream gets the highest priority: its CTAs are
    // scheduled first when SM resources free up
    if (e == cudaSuccess)
      e = cudaStreamCreateWithPriority(&sl.st, cudaStreamNonBlocking, sl.small_only ? prio_hi : prio_lo);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    for (int k = 0; k < kPaceWindow && e == cudaSuccess; k++)
      e = cudaEventCreateWithFlags(&sl.pace.ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_work, kGroupWorkBytes);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_work, kGroupWorkBytes);
    if (e == cudaSuccess) std::memset(sl.h_work, 0, kGroupWorkBytes);
    // capture: work-list copy + grouped launch, replayed once per batch
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(sl.st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaMemcpyAsync(sl.d_work, sl.h_work, kGroupWorkBytes, cudaMemcpyHostToDevice, sl.st);
      cudaError_t e2 = e1 == cudaSuccess ? launch_grouped(sl.d_work, grid, sl.st) : e1;
      cudaError_t e3 = cudaStreamEndCapture(sl.st, &g);
      e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.exec, g, 0);
    if (g) cudaGraphDestroy(g);
  }
  if (e != cudaSuccess) {
    destroy_server(s);
    return cuda_error(e, "bs_server_create");
  }
  for (Slot& sl : s->slots) sl.launcher = std::thread(launcher_loop, s, &sl);
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return BS_OK;
}

bs_status bs_server_destroy(bs_server s) {
  if (!s) return BS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (Slot& sl : s->slots)
    if (sl.launcher.joinable()) sl.launcher.join();
  destroy_server(s);
  return BS_OK;
}

bs_status bs_server_submit(bs_server s, bs_handle h, const void* host_B, void* host_X, int mode, int64_t M,
                           int64_t* request_id) {
  if (!s || !request_id) return set_error(BS_EINVAL, "bs_server_submit: null argument");
  if (!valid_handle(h)) return set_error(BS_EINVAL, "bs_server_submit: unknown handle");
  if (h->periodic) return set_error(BS_EUNSUPPORTED, "bs_server_submit: not available for a periodic handle");
  if (h->device != s->device) return set_error(BS_EINVAL, "bs_server_submit: handle on another device");
  if (!host_B || !host_X) return set_error(BS_EINVAL, "bs_server_submit: null buffer");
  if (mode != SERVE_F64 && mode != SERVE_F32_REFINE) return set_error(BS_EINVAL, "bs_server_submit: bad mode");
  if (M < 1 || M > (int64_t)kGroupMaxTiles * 32) return set_error(BS_EINVAL, "bs_server_submit: M out of range");
  for (const void* p : {host_B, static_cast<const void*>(host_X)}) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      return set_error(BS_EINVAL, "bs_server_submit: host buffers must be page-locked (pinned) host memory");
    }
  }
  const size_t bytes = req_bytes(h->width, h->N, mode, M);
  std::lock_guard<std::mutex> lk(s->mu);
  if (bytes > s->arena.size())
    return set_error(BS_ENOMEM, "bs_server_submit: request larger than the server's HBM budget");
  if (!handle_ref(h)) return set_error(BS_EINVAL, "bs_server_submit: unknown handle");
  const int64_t id = s->next_id++;
  Req r;
  r.h = h;
  r.hB = host_B;
  r.hX = host_X;
  r.mode = mode;
  r.M = M;
  r.bytes = bytes;
  r.off = 0;
  r.small = bytes <= kSmallBytes;
  r.t_submit = now_s();
  s->reqs[id] = r;
  (r.small ? s->queue : s->queue_large).push_back(id);
  *request_id = id;
  s->cv.notify_all();
  return BS_OK;
}

bs_status bs_server_poll(bs_server s, int64_t id, int* state, double* latency_s) {
  if (!s) return set_error(BS_EINVAL, "bs_server_poll: null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(BS_EINVAL, "bs_server_poll: unknown request");
  if (state) *state = it->second.state;
  if (latency_s) *latency_s = it->second.t_done > 0 ? it->second.t_done - it->second.t_submit : -1.0;
  return BS_OK;
}

bs_status bs_server_wait(bs_server s, int64_t id, double timeout_s, int* state) {
  if (!s) return set_error(BS_EINVAL, "bs_server_wait: null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(BS_EINVAL, "bs_server_wait: unknown request");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (it->second.state == RQ_QUEUED || it->second.state == RQ_RUNNING) {
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout &&
        (it->second.state == RQ_QUEUED || it->second.state == RQ_RUNNING)) {
      if (state) *state = it->second.state;
      return set_error(BS_ETIMEOUT, "bs_server_wait: timed out");
    }
  }
  if (state) *state = it->second.state;
  return BS_OK;
}

bs_status bs_server_cancel(bs_server s, int64_t id) {
  if (!s) return set_error(BS_EINVAL, "bs_server_cancel: null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(BS_EINVAL, "bs_server_cancel: unknown request");
  if (it->second.state != RQ_QUEUED) return set_error(BS_EINVAL, "bs_server_cancel: request already admitted");
  it->second.state = RQ_CANCELLED;
  it->second.t_done = now_s();
  handle_unref(it->second.h);
  s->cv.notify_all();
  return BS_OK;
}

bs_status bs_server_release(bs_server s, int64_t id) {
  if (!s) return set_error(BS_EINVAL, "bs_server_release: null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(BS_EINVAL, "bs_server_release: unknown request");
  if (it->second.state == RQ_QUEUED || it->second.state == RQ_RUNNING)
    return set_error(BS_EINVAL, "bs_server_release: request still pending");
  s->reqs.erase(it);
  return BS_OK;
}

bs_status bs_server_pause(bs_server s, int paused) {
  if (!s) return set_error(BS_EINVAL, "bs_server_pause: null server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->paused = paused != 0;
  s->cv.notify_all();
  return BS_OK;
}

bs_status bs_server_fail_on_admit(bs_server s, int64_t id) {
  if (!s) return set_error(BS_EINVAL, "bs_server_fail_on_admit: null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second.state != RQ_QUEUED)
    return set_error(BS_EINVAL, "bs_server_fail_on_admit: request not queued");
  it->second.fail_on_admit = true;
  return BS_OK;
}

bs_status bs_server_stats(bs_server s, int64_t* out, int n) {
  if (!s || !out || n < 1) return set_error(BS_EINVAL, "bs_server_stats: bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t queued = 0, running = 0;
  for (auto& kv : s->reqs) {
    queued += kv.second.state == RQ_QUEUED;
    running += kv.second.state == RQ_RUNNING;
  }
  const int64_t v[10] = {s->batches, s->completed, s->failed, queued, running, (int64_t)s->arena.used(),
                         (int64_t)s->arena.peak(), (int64_t)s->arena.size(), s->max_batch_reqs, s->max_concurrent};
  for (int q = 0; q < n && q < 10; q++) out[q] = v[q];
  if (s->sticky != cudaSuccess) return cuda_error(s->sticky, "bs_server: a batch failed");
  return BS_OK;
}

}  // extern "C"
