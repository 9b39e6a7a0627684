// server.cu -- a continuous-batching server for bridge queries on one GPU.
//
// Requests (graphs whose edge arrays are already resident on the device) are queued on submit.
// A scheduler thread keeps up to `max_slots` units of work in flight, each on its own stream
// with its own context (workspace), so work from different requests overlaps on the device:
//   - small graphs (V <= 4096) waiting in the queue are gathered into one batched launch
//     (the persistent shared-memory kernel of batched.cu);
//   - a large graph runs the single-graph path (partition forest pass, merge tree, final stage)
//     when its workspace fits in what the memory budget has left.
// Requests that arrive while others run are admitted as soon as a slot and memory free up
// (continuous batching).  Completion is detected with CUDA events; each request's latency is
// measured from submit to the moment its event is seen complete.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/bridges.h"
#include "batched.h"
#include "ctx.h"
#include "internal.h"

using namespace bridges;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SrvReq {
  bridges_request r{};
  size_t ws = 0;  // workspace the single-graph path needs (0 for batched requests)
  bool small = false;
  int state = 0;  // 0 queued, 1 running, 2 done
  int64_t count = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
};

struct SrvSlot {
  bridges_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  std::vector<uint64_t> tickets;
  int64_t* d_counts = nullptr;
  int64_t* h_counts = nullptr;
  size_t reserved = 0;
};

}  // namespace

struct bridges_server {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;
  int32_t max_batch = 4096;
  std::vector<SrvSlot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, SrvReq> reqs;
  uint64_t next_ticket = 1;
  std::thread th;
  bool stop = false;
  int64_t stats[6] = {0, 0, 0, 0, 0, 0};  // completed, batches, singles, max in flight, failures, queued now
  int32_t error = BRIDGES_OK;             // sticky scheduler error
};

namespace {

// Launches queued work on free slots.  Caller holds mu.
void admit(bridges_server* S) {
  for (SrvSlot& sl : S->slots) {
    if (S->queue.empty()) return;
    if (sl.busy) continue;
    SrvReq& head = S->reqs[S->queue.front()];
    const bool take_large = !head.small && (S->budget == 0 || S->used + head.ws <= S->budget);
    sl.tickets.clear();
    int64_t rc = BRIDGES_OK;
    if (take_large) {
      const uint64_t t = S->queue.front();
      S->queue.pop_front();
      SrvReq& q = S->reqs[t];
      q.state = 1;
      q.t_start = now_s();
      sl.tickets.push_back(t);
      sl.reserved = q.ws;
      rc = run_single(sl.ctx, sl.stream, q.r.edges_u, q.r.edges_v, q.r.E, q.r.V, q.r.M, q.r.out_bridges, sl.d_counts);
      S->stats[2]++;
    } else {
      // gather the oldest small requests; large ones keep their place in the queue
      std::vector<BatchTask> graphs, tasks;
      int64_t total_e = 0;
      for (auto it = S->queue.begin(); it != S->queue.end() && (int32_t)graphs.size() < S->max_batch;) {
        SrvReq& q = S->reqs[*it];
        if (!q.small) {
          ++it;
          continue;
        }
        BatchTask bt{};
        bt.u = q.r.edges_u;
        bt.v = q.r.edges_v;
        bt.lo = 0;
        bt.hi = q.r.E;
        bt.out = q.r.out_bridges;
        bt.count = sl.d_counts + graphs.size();
        bt.g = (int32_t)graphs.size();
        bt.V = q.r.V;
        graphs.push_back(bt);
        total_e += q.r.E;
        q.state = 1;
        q.t_start = now_s();
        sl.tickets.push_back(*it);
        it = S->queue.erase(it);
      }
      if (graphs.empty()) return;  // only large requests wait, and the head does not fit yet
      sl.reserved = 0;
      const int64_t slot_words = plan_batch_tasks(sl.ctx, graphs, total_e, tasks);
      rc = launch_batch_tasks(sl.ctx, sl.stream, tasks, (int32_t)graphs.size(), slot_words);
      S->stats[1]++;
    }
    if (rc == BRIDGES_OK &&
        cudaMemcpyAsync(sl.h_counts, sl.d_counts, sizeof(int64_t) * sl.tickets.size(), cudaMemcpyDeviceToHost,
                        sl.stream) != cudaSuccess)
      rc = BRIDGES_ECUDA;
    if (rc == BRIDGES_OK && cudaEventRecord(sl.ev, sl.stream) != cudaSuccess) rc = BRIDGES_ECUDA;
    if (rc != BRIDGES_OK) {
      // the requests fail; the slot stays free
      cudaGetLastError();
      for (uint64_t t : sl.tickets) {
        SrvReq& q = S->reqs[t];
        q.state = 2;
        q.count = rc;
        q.t_done = now_s();
        S->stats[4]++;
      }
      sl.tickets.clear();
      S->cv_done.notify_all();
      continue;
    }
    sl.busy = true;
    S->used += sl.reserved;
    int64_t inflight = 0;
    for (const SrvSlot& x : S->slots) inflight += x.busy ? (int64_t)x.tickets.size() : 0;
    S->stats[3] = std::max(S->stats[3], inflight);
  }
}

// Retires slots whose event completed.  Caller holds mu.  Returns true if anything finished.
bool retire(bridges_server* S) {
  bool any = false;
  for (SrvSlot& sl : S->slots) {
    if (!sl.busy) continue;
    const cudaError_t e = cudaEventQuery(sl.ev);
    if (e == cudaErrorNotReady) continue;
    const double t = now_s();
    for (size_t i = 0; i < sl.tickets.size(); i++) {
      SrvReq& q = S->reqs[sl.tickets[i]];
      q.state = 2;
      q.count = e == cudaSuccess ? sl.h_counts[i] : (int64_t)BRIDGES_ECUDA;
      q.t_done = t;
      S->stats[0]++;
    }
    if (e != cudaSuccess) cudaGetLastError();
    sl.tickets.clear();
    sl.busy = false;
    S->used -= sl.reserved;
    sl.reserved = 0;
    any = true;
  }
  return any;
}

void scheduler(bridges_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    const bool finished = retire(S);
    if (finished) S->cv_done.notify_all();
    admit(S);
    bool busy = false;
    for (const SrvSlot& sl : S->slots) busy = busy || sl.busy;
    if (S->stop && !busy && S->queue.empty()) break;
    // short waits while work is in flight (completion is polled), long ones when idle
    if (busy)
      S->cv_work.wait_for(lk, std::chrono::microseconds(20));
    else
      S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
  }
}

}  // namespace

extern "C" {

bridges_server* bridges_server_create(int device, size_t mem_budget_bytes, int32_t max_slots, int32_t max_batch,
                                      const bridges_opts* opts) {
  if (max_slots <= 0) max_slots = 4;
  if (max_batch <= 0) max_batch = 4096;
  bridges_server* S = new (std::nothrow) bridges_server();
  if (!S) return nullptr;
  S->device = device;
  S->budget = mem_budget_bytes;
  S->max_batch = max_batch;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return nullptr;
  }
  S->slots.resize(max_slots);
  // requests run at the device's highest stream priority: when other work of the process shares
  // the GPU (ingest of the next requests, say), the block scheduler starts the requests' blocks
  // first as SMs free up
  int prio_low = 0, prio_high = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
    cudaGetLastError();
    prio_high = 0;
  }
  bool ok = true;
  for (SrvSlot& sl : S->slots) {
    sl.ctx = bridges_ctx_create(device, 0, opts);
    ok = ok && sl.ctx;
    ok = ok && cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, prio_high) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.d_counts, sizeof(int64_t) * (size_t)max_batch) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl.h_counts, sizeof(int64_t) * (size_t)max_batch) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    S->stop = true;
    bridges_server_destroy(S);
    return nullptr;
  }
  S->th = std::thread(scheduler, S);
  return S;
}

int32_t bridges_server_submit(bridges_server* S, const bridges_request* r, uint64_t* ticket) {
  if (!S || !r || !ticket || r->V < 0 || r->E < 0 || r->V > (1 << 30)) return BRIDGES_EINVAL;
  if (r->E > 0 && (!r->edges_u || !r->edges_v)) return BRIDGES_EINVAL;
  if (r->V > 1 && !r->out_bridges) return BRIDGES_EINVAL;
  SrvReq q;
  q.r = *r;
  q.small = r->V <= kBatchVmax;
  q.ws = q.small ? 0 : single_workspace_bytes(S->slots[0].ctx, r->E, r->V);
  if (S->budget && q.ws > S->budget) return BRIDGES_EAGAIN;  // can never fit
  q.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return BRIDGES_EINVAL;
    *ticket = S->next_ticket++;
    S->reqs.emplace(*ticket, q);
    S->queue.push_back(*ticket);
  }
  S->cv_work.notify_one();
  return BRIDGES_OK;
}

int32_t bridges_server_poll(bridges_server* S, uint64_t ticket, int64_t* count, double* latency_ms) {
  if (!S) return BRIDGES_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return BRIDGES_EINVAL;
  if (it->second.state != 2) return BRIDGES_EBUSY;
  if (count) *count = it->second.count;
  if (latency_ms) *latency_ms = (it->second.t_done - it->second.t_submit) * 1e3;
  S->reqs.erase(it);
  return BRIDGES_OK;
}

int32_t bridges_server_wait(bridges_server* S, uint64_t ticket, int64_t timeout_ms, int64_t* count,
                            double* latency_ms) {
  if (!S) return BRIDGES_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max<int64_t>(timeout_ms, 0));
  while (true) {
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return BRIDGES_EINVAL;
    if (it->second.state == 2) {
      if (count) *count = it->second.count;
      if (latency_ms) *latency_ms = (it->second.t_done - it->second.t_submit) * 1e3;
      S->reqs.erase(it);
      return BRIDGES_OK;
    }
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto jt = S->reqs.find(ticket);
      if (jt != S->reqs.end() && jt->second.state == 2) continue;
      return BRIDGES_ETIMEDOUT;
    }
  }
}

int32_t bridges_server_cancel(bridges_server* S, uint64_t ticket) {
  if (!S) return BRIDGES_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return BRIDGES_EINVAL;
    SrvReq& q = it->second;
    if (q.state != 0) return BRIDGES_EBUSY;  // launched (or done): it completes normally
    auto qt = std::find(S->queue.begin(), S->queue.end(), ticket);
    if (qt != S->queue.end()) S->queue.erase(qt);
    q.state = 2;
    q.count = BRIDGES_ECANCELED;
    q.t_done = now_s();
  }
  S->cv_done.notify_all();
  return BRIDGES_OK;
}

int32_t bridges_server_stats(bridges_server* S, int64_t* vals, int32_t n) {
  if (!S || !vals) return 0;
  std::lock_guard<std::mutex> lk(S->mu);
  S->stats[5] = (int64_t)S->queue.size();
  const int32_t k = std::min<int32_t>(n, 6);
  for (int i = 0; i < k; i++) vals[i] = S->stats[i];
  return k;
}

void bridges_server_destroy(bridges_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->th.joinable()) S->th.join();
  cudaSetDevice(S->device);
  for (SrvSlot& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.ctx) bridges_ctx_destroy(sl.ctx);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.d_counts) cudaFree(sl.d_counts);
    if (sl.h_counts) cudaFreeHost(sl.h_counts);
  }
  cudaGetLastError();
  delete S;
}

}  // extern "C"
