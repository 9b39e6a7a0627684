// api.cu -- the C ABI of libbridges (declared in include/bridges.h): contexts, workspace,
// argument checks and the orchestration of the stages on one stream.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/bridges.h"
#include "batched.h"
#include "ctx.h"
#include "common.cuh"
#include "internal.h"

#include <cmath>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

using namespace bridges;

namespace {

constexpr size_t kMiscBytes = 1024;  // status word, device counts of bridges_from_forest, spare output
constexpr size_t kSpareAt = 512;     // the spare output slot: where a call that has no pairs or points
                                     // to write (V <= 1, null output) points the stages

// NVTX range for the duration of a host scope (what the host enqueues; a profiler correlates the
// launches inside it).  Header-only NVTX: without an attached tool a push / pop is a no-op.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

struct Carved {
  int32_t* status;
  int32_t* counts;  // [2]
  int32_t* spare;   // [2] device scratch for outputs the caller did not ask for
  CertBufs cert;
  FinalBufs fin;
};

// The launch context of a call on c: its stream, its launch counter and the final stage's test
// knobs from the options (zero in normal use).
Launch launch_for(bridges_ctx* c, cudaStream_t s) {
  Launch L{s, &c->launches, c->num_sms, c->smem_optin};
  L.bar_polls = c->opts.test_barrier_polls > 0 ? (unsigned)c->opts.test_barrier_polls : 0u;
  L.hold_polls = c->opts.test_hold_polls > 0 ? c->opts.test_hold_polls : 0;
  return L;
}

int64_t cuda_fail(cudaError_t e) {
  (void)e;
  cudaGetLastError();
  return BRIDGES_ECUDA;
}

size_t total_bytes(const CertPlan& p) { return kMiscBytes + align_up(cert_bytes(p), 256) + final_bytes(p.V); }

Carved carve(bridges_ctx* c, const CertPlan& p) {
  Carved k{};
  char* base = static_cast<char*>(c->ws);
  k.status = reinterpret_cast<int32_t*>(base);
  k.counts = reinterpret_cast<int32_t*>(base + 256);
  k.spare = reinterpret_cast<int32_t*>(base + kSpareAt);
  k.cert = carve_cert(base + kMiscBytes, p);
  k.cert.status = k.status;
  k.fin = carve_final(base + kMiscBytes + align_up(cert_bytes(p), 256), p.V, k.status);
  return k;
}

// Whether ensure_ws(c, need) could succeed without exceeding a limit the caller set (a
// workspace of its own, or a memory budget).
bool ws_fits(const bridges_ctx* c, size_t need) {
  if (need <= c->ws_bytes) return true;
  if (c->user_ws) return false;
  return !c->budget || need + c->stage_bytes <= c->budget;
}

// A device allocation of one of the context's own buffers.  With opts.test_fail_alloc = n > 0 the
// n-th of them since the options were set fails as cudaMalloc does on a full device (a test of the
// failure path; never set in normal use).
cudaError_t ctx_malloc(bridges_ctx* c, void** p, size_t bytes) {
  if (++c->allocs == c->opts.test_fail_alloc && c->opts.test_fail_alloc > 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

// Makes the workspace at least `need` bytes.  Waits for the context's previous work before
// freeing an old, smaller workspace.
int64_t ensure_ws(bridges_ctx* c, size_t need, cudaStream_t s) {
  if (need <= c->ws_bytes) return BRIDGES_OK;
  if (c->user_ws) return BRIDGES_ENOMEM;
  if (c->budget && need + c->stage_bytes > c->budget) return BRIDGES_ENOMEM;
  if (c->ws) {
    cudaStreamSynchronize(s);
    cudaDeviceSynchronize();
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
  }
  size_t bytes = align_up(need + need / 8, 1 << 20);
  if (c->budget) bytes = std::min(bytes, c->budget - c->stage_bytes);
  if (ctx_malloc(c, &c->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->ws = nullptr;
    return BRIDGES_ENOMEM;
  }
  c->ws_bytes = bytes;
  return BRIDGES_OK;
}

CertPlan plan_for(const bridges_ctx* c, int64_t E, int32_t V, int32_t M) {
  const bridges_opts& o = c->opts;
  int32_t m = M > 0 ? M : o.M;
  return make_plan(E, V, m, o.fan_in, o.block, o.ctas_per_sm, o.warm_edges < 0 ? -1 : (o.warm_edges == 0 ? 0 : o.warm_edges),
                   c->num_sms, c->smem_optin, o.warm_block);
}

// Reads back the stage times of every issued call up to (not including) call index `upto`.
// [0] warm-up, [1] snapshot, [2] forest pass, [3] merge, [4] final, [5] total
void resolve_timings(bridges_ctx* c, int64_t upto) {
  for (; c->resolved < upto; c->resolved++) {
    const int s = (int)(c->resolved % bridges_ctx::kRing);
    cudaEvent_t* e = c->ev[s];
    cudaEventSynchronize(e[6]);
    for (int i = 0; i < 5; i++) cudaEventElapsedTime(&c->stage_ms[s][i], e[i], e[i + 1]);
    cudaEventElapsedTime(&c->stage_ms[s][5], e[7], e[6]);
  }
}

// The same for the articulation-point block pass: [0] warm-up, [1] snapshot, [2] stream,
// [3] marking and compaction, [4] the whole pass.
void resolve_ap_timings(bridges_ctx* c, int64_t upto) {
  for (; c->ap_resolved < upto; c->ap_resolved++) {
    const int s = (int)(c->ap_resolved % bridges_ctx::kRing);
    cudaEvent_t* e = c->ap_ev[s];
    cudaEventSynchronize(e[4]);
    for (int i = 0; i < 4; i++) cudaEventElapsedTime(&c->ap_ms[s][i], e[i], e[i + 1]);
    cudaEventElapsedTime(&c->ap_ms[s][4], e[0], e[4]);
  }
}

// Before a profiled call reuses a ring slot, the times of the call that last used it are read.
cudaEvent_t* next_event_slot(bridges_ctx* c) {
  if (!c->events) return nullptr;
  resolve_timings(c, c->calls - bridges_ctx::kRing + 1);
  return c->ev[c->calls % bridges_ctx::kRing];
}

int init_ctx(bridges_ctx* c, int device, const bridges_opts* opts) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return -1;
  }
  c->device = device;
  if (opts) c->opts = *opts;
  if (!opts) c->opts.warm_edges = -1;
  if (cudaSetDevice(device) != cudaSuccess) return -1;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->smem_optin = (size_t)optin;
  if (cudaMallocHost(&c->h_pinned, 64) != cudaSuccess) return -1;
  if (c->opts.profile) {
    for (auto& set : c->ev)
      for (auto& e : set)
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
    for (auto& set : c->ap_ev)
      for (auto& e : set)
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
    c->events = true;
  }
  return 0;
}

// The final stage of a call that wants only the sorted bridges and their count (none of the
// rooted forest's arrays): a graph of 2..kBatchVmax vertices runs it on one block in shared
// memory (small_final_launch: block barriers only, against the grid stage's 19 grid barriers),
// a larger one on the grid.  The grid barrier's test knobs keep the grid form.
void final_bridges(const Launch& L, const Carved& k, int32_t V, int32_t* out) {
  if (V >= 2 && V <= kBatchVmax && L.bar_polls == 0 && L.hold_polls == 0) {
    const SmallFinalArgs a{V, k.cert.P1, k.cert.f1u, k.cert.f1v, k.cert.cnt + 0, k.cert.f2u, k.cert.f2v,
                           k.cert.cnt + 1, k.fin.status, k.fin.count, out};
    small_final_launch(L.stream, a);  // a launch error is caught by the caller's error check
    *L.launches += 1;
    return;
  }
  final_stage(L, k.fin, V, k.cert.f1u, k.cert.f1v, k.cert.cnt + 0, V, k.cert.f2u, k.cert.f2v, k.cert.cnt + 1, V,
              k.cert.P1, out);
}

// The whole path on device-resident edges.  Leaves the count on the device (fin.count).  With
// with_final false it stops after the certificate; otherwise the sorted pairs go to out, or to
// the final stage's own dscan array (free by the time it sorts) when out is null.  With
// bridges_only the caller reads nothing of the final stage but the pairs and the count.
int64_t run_path(bridges_ctx* c, cudaStream_t s, const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t M,
                 int32_t* out, Carved* kout, CertPlan* pout, bool with_final = true, bool bridges_only = false) {
  Range range("bridges: certificate + final stage");
  CertPlan p = plan_for(c, E, V, M);
  int64_t rc = ensure_ws(c, total_bytes(p), s);
  if (rc != BRIDGES_OK) return rc;
  Carved k = carve(c, p);
  Launch L = launch_for(c, s);
  c->last_cfg[0] = p.M;
  c->last_cfg[1] = p.f;
  c->last_cfg[2] = p.G;
  c->last_cfg[3] = p.block;
  c->last_cfg[4] = p.cache ? p.warm : -1;
  cudaEvent_t* ev = next_event_slot(c);
  if (ev) cudaEventRecord(ev[7], s);
  cudaMemsetAsync(k.status, 0, sizeof(int32_t), s);
  cert_init(L, p, k.cert);
  cert_leaves(L, p, k.cert, u, v, ev);
  if (ev && E == 0)
    for (int i = 0; i < 4; i++) cudaEventRecord(ev[i], s);
  cert_merge(L, p, k.cert);
  if (ev) cudaEventRecord(ev[4], s);
  if (with_final) {
    // job 0 holds the final certificate: F (tree) and F' (extra); its UF1 roots the trees
    if (bridges_only)
      final_bridges(L, k, V, out ? out : k.fin.dscan);
    else
      final_stage(L, k.fin, V, k.cert.f1u, k.cert.f1v, k.cert.cnt + 0, V, k.cert.f2u, k.cert.f2v, k.cert.cnt + 1,
                  V, k.cert.P1, out ? out : k.fin.dscan);
  }
  if (ev) {
    cudaEventRecord(ev[5], s);
    cudaEventRecord(ev[6], s);
    c->calls++;
  }
  if (cudaGetLastError() != cudaSuccess) return BRIDGES_ECUDA;
  if (kout) *kout = k;
  if (pout) *pout = p;
  return BRIDGES_OK;
}

int64_t check_args(const bridges_ctx* c, const void* u, const void* v, int64_t E, int32_t V, const void* out) {
  if (!c || E < 0 || V < 0) return BRIDGES_EINVAL;
  if (E > 0 && (!u || !v)) return BRIDGES_EINVAL;
  if (V > 1 && !out) return BRIDGES_EINVAL;
  return BRIDGES_OK;
}

// Stages host edges for a call: either the device aliases of pinned, mapped buffers (opts.host_read)
// or copies into the context's device staging area; *dout receives 2*max(V,1) int32 of device
// output space.  Enqueue only.
int64_t stage_host_edges(bridges_ctx* c, cudaStream_t s, const int32_t* hu, const int32_t* hv, int64_t E, int32_t V,
                         const int32_t** ru_out, const int32_t** rv_out, int32_t** dout_out,
                         bool defer_copy = false, bool* copy_deferred = nullptr) {
  Range range("bridges: host edges");
  // pinned, mapped host memory can be streamed by the kernels in place (no device copy of the
  // edges: graphs larger than device memory work this way)
  const int32_t* ru = nullptr;
  const int32_t* rv = nullptr;
  bool in_place = false;
  if (c->opts.host_read && E > 0) {
    cudaPointerAttributes au{}, av{};
    if (cudaPointerGetAttributes(&au, hu) == cudaSuccess && cudaPointerGetAttributes(&av, hv) == cudaSuccess &&
        au.type == cudaMemoryTypeHost && av.type == cudaMemoryTypeHost && au.devicePointer && av.devicePointer) {
      ru = static_cast<const int32_t*>(au.devicePointer);
      rv = static_cast<const int32_t*>(av.devicePointer);
      in_place = true;
    }
    cudaGetLastError();
  }
  // device staging: the output (2V) and, unless read in place, u and v (E each)
  const size_t eb = in_place ? 0 : align_up(sizeof(int32_t) * (size_t)std::max<int64_t>(E, 1), 256);
  const size_t ob = align_up(sizeof(int32_t) * 2 * (size_t)std::max(V, 1), 256);
  const size_t need = 2 * eb + ob;
  if (need > c->stage_bytes) {
    if (c->user_ws) return BRIDGES_ENOMEM;
    if (c->budget && need + c->ws_bytes > c->budget) return BRIDGES_ENOMEM;
    if (c->stage) {
      cudaStreamSynchronize(s);
      cudaFree(c->stage);
      c->stage = nullptr;
      c->stage_bytes = 0;
    }
    if (ctx_malloc(c, reinterpret_cast<void**>(&c->stage), need) != cudaSuccess) {
      cudaGetLastError();
      return BRIDGES_ENOMEM;
    }
    c->stage_bytes = need;
  }
  char* base = reinterpret_cast<char*>(c->stage);
  int32_t* dout = reinterpret_cast<int32_t*>(base + 2 * eb);
  if (!in_place) {
    int32_t* du = reinterpret_cast<int32_t*>(base);
    int32_t* dv = reinterpret_cast<int32_t*>(base + eb);
    ru = du;
    rv = dv;
    if (!defer_copy && E > 0 &&
        (cudaMemcpyAsync(du, hu, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(dv, hv, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, s) != cudaSuccess))
      return cuda_fail(cudaGetLastError());
  }
  if (copy_deferred) *copy_deferred = defer_copy && !in_place;
  *ru_out = ru;
  *rv_out = rv;
  *dout_out = dout;
  return BRIDGES_OK;
}

// Host input with the copy overlapped: the list is copied in chunks on the context's copy stream
// while the forest pass (one pass over the list, Sec. 3 phase 0) streams the chunks already on
// the device.  Single partition with a snapshot only; returns 1 when the plan does not qualify
// (nothing enqueued: the caller copies everything first).
// The chunk schedule of an overlapped host copy for a plan with warm-up prefix `warm`: chunks of
// C edges (16 M or more, at most kMaxChunks, the first holding the prefix); false when the list
// is too short to gain from it.
static bool chunk_plan(int64_t E, int64_t warm, int64_t* C, int* K) {
  *C = std::max<int64_t>({warm, ceil_div(E, bridges_ctx::kMaxChunks), (int64_t)16 << 20});
  *K = (int)ceil_div(E, *C);
  return *K >= 2 && *K <= bridges_ctx::kMaxChunks;
}

// Issues the chunk copies of (hu, hv) into (du, dv) on the context's copy stream, chunk i's
// completion recorded in c->chunk_ev[i]; the copies start once the work already on `s` (which
// may still read the staging) is done.
static int64_t issue_chunks(bridges_ctx* c, cudaStream_t s, const int32_t* hu, const int32_t* hv, int32_t* du,
                            int32_t* dv, int64_t E, int64_t C, int K) {
  if (!c->copy_stream) {
    if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->entry_ev, cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(cudaGetLastError());
    for (auto& e : c->chunk_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return cuda_fail(cudaGetLastError());
  }
  cudaStream_t cs = c->copy_stream;
  if (cudaEventRecord(c->entry_ev, s) != cudaSuccess || cudaStreamWaitEvent(cs, c->entry_ev, 0) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  for (int i = 0; i < K; i++) {
    const int64_t lo = C * i, n = std::min<int64_t>(C, E - lo);
    if (cudaMemcpyAsync(du + lo, hu + lo, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemcpyAsync(dv + lo, hv + lo, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaEventRecord(c->chunk_ev[i], cs) != cudaSuccess)
      return cuda_fail(cudaGetLastError());
  }
  return BRIDGES_OK;
}

int64_t run_path_host(bridges_ctx* c, cudaStream_t s, const int32_t* hu, const int32_t* hv, int32_t* du, int32_t* dv,
                      int64_t E, int32_t V, int32_t M, int32_t* out, Carved* kout, bool bridges_only) {
  Range range("bridges: pipelined host input");
  const CertPlan p = plan_for(c, E, V, M);
  if (p.M != 1 || !p.cache) return 1;
  int64_t C = 0;
  int K = 0;
  if (!chunk_plan(E, p.warm, &C, &K)) return 1;
  int64_t rc = ensure_ws(c, total_bytes(p), s);
  if (rc != BRIDGES_OK) return rc;
  Carved k = carve(c, p);
  Launch L = launch_for(c, s);
  c->last_cfg[0] = p.M;
  c->last_cfg[1] = p.f;
  c->last_cfg[2] = p.G;
  c->last_cfg[3] = p.block;
  c->last_cfg[4] = p.warm;
  rc = issue_chunks(c, s, hu, hv, du, dv, E, C, K);
  if (rc != BRIDGES_OK) return rc;
  cudaEvent_t* ev = next_event_slot(c);
  if (ev) cudaEventRecord(ev[7], s);
  cudaMemsetAsync(k.status, 0, sizeof(int32_t), s);
  cert_init(L, p, k.cert);
  cudaStreamWaitEvent(s, c->chunk_ev[0], 0);  // the first chunk holds the warm-up prefix (C >= warm)
  if (ev) cudaEventRecord(ev[0], s);
  cert_warm(L, p, k.cert, du, dv);
  if (ev) cudaEventRecord(ev[1], s);
  cert_snapshot(L, p, k.cert);
  if (ev) cudaEventRecord(ev[2], s);
  for (int i = 0; i < K; i++) {
    if (i > 0) cudaStreamWaitEvent(s, c->chunk_ev[i], 0);
    cert_stream(L, p, k.cert, du, dv, C * i, std::min<int64_t>(E, C * (i + 1)));
  }
  if (ev) cudaEventRecord(ev[3], s);
  cert_merge(L, p, k.cert);
  if (ev) cudaEventRecord(ev[4], s);
  if (bridges_only)
    final_bridges(L, k, V, out);
  else
    final_stage(L, k.fin, V, k.cert.f1u, k.cert.f1v, k.cert.cnt + 0, V, k.cert.f2u, k.cert.f2v, k.cert.cnt + 1, V,
                k.cert.P1, out);
  if (ev) {
    cudaEventRecord(ev[5], s);
    cudaEventRecord(ev[6], s);
    c->calls++;
  }
  if (cudaGetLastError() != cudaSuccess) return BRIDGES_ECUDA;
  *kout = k;
  return BRIDGES_OK;
}

std::mutex g_default_mu[64];
bridges_ctx* g_default[64];

}  // namespace

extern "C" {

bridges_ctx* bridges_ctx_create(int device, size_t mem_budget_bytes, const bridges_opts* opts) {
  bridges_ctx* c = new (std::nothrow) bridges_ctx();
  if (!c) return nullptr;
  c->budget = mem_budget_bytes;
  if (init_ctx(c, device, opts) != 0) {
    bridges_ctx_destroy(c);
    return nullptr;
  }
  return c;
}

bridges_ctx* bridges_ctx_create_ws(int device, void* ws_device, size_t ws_bytes, const bridges_opts* opts) {
  if (!ws_device || (reinterpret_cast<uintptr_t>(ws_device) & 255)) return nullptr;
  bridges_ctx* c = new (std::nothrow) bridges_ctx();
  if (!c) return nullptr;
  c->user_ws = true;
  c->ws = ws_device;
  c->ws_bytes = ws_bytes;
  if (init_ctx(c, device, opts) != 0) {
    c->ws = nullptr;
    bridges_ctx_destroy(c);
    return nullptr;
  }
  return c;
}

void bridges_ctx_destroy(bridges_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  if (!c->user_ws && c->ws) cudaFree(c->ws);
  if (c->stage) cudaFree(c->stage);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  for (int k = 0; k < 2; k++) {
    if (c->b_exec[k]) cudaGraphExecDestroy(c->b_exec[k]);
    if (c->bstage[k]) cudaFreeHost(c->bstage[k]);
    if (c->b_done_ev[k]) cudaEventDestroy(c->b_done_ev[k]);
  }
  if (c->bws) cudaFree(c->bws);
  if (c->copy_stream) {
    cudaStreamDestroy(c->copy_stream);
    cudaEventDestroy(c->entry_ev);
    for (auto& e : c->chunk_ev) cudaEventDestroy(e);
  }
  if (c->events) {
    for (auto& set : c->ev)
      for (auto& e : set) cudaEventDestroy(e);
    for (auto& set : c->ap_ev)
      for (auto& e : set) cudaEventDestroy(e);
  }
  cudaGetLastError();
  delete c;
}

size_t bridges_workspace_bytes(const bridges_ctx* c, int64_t E, int32_t V, int32_t M) {
  if (!c || E < 0 || V < 0) return 0;
  return total_bytes(plan_for(c, E, V, M));
}

int64_t bridges_find_ctx(bridges_ctx* c, struct CUstream_st* stream, const int32_t* u, const int32_t* v, int64_t E,
                         int32_t V, int32_t M, int32_t* out, int64_t* out_count_device) {
  int64_t rc = check_args(c, u, v, E, V, out);
  if (rc) return rc;
  if (V > (1 << 30)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  Carved k{};
  rc = run_path(c, s, u, v, E, V, M, out, &k, nullptr, true, true);
  if (rc) return rc;
  if (out_count_device) {
    if (cudaMemcpyAsync(out_count_device, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return cuda_fail(cudaGetLastError());
    return BRIDGES_OK;
  }
  if (cudaMemcpyAsync(c->h_pinned, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  return c->h_pinned[0];
}

int64_t bridges_find(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t M, int32_t* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cuda_fail(cudaGetLastError());
  std::lock_guard<std::mutex> lock(g_default_mu[dev]);
  if (!g_default[dev]) {
    bridges_opts o{};
    o.warm_edges = -1;
    g_default[dev] = bridges_ctx_create(dev, 0, &o);
    if (!g_default[dev]) return BRIDGES_ECUDA;
  }
  return bridges_find_ctx(g_default[dev], nullptr, u, v, E, V, M, out, nullptr);
}

int64_t bridges_find_host(bridges_ctx* c, struct CUstream_st* stream, const int32_t* hu, const int32_t* hv, int64_t E,
                          int32_t V, int32_t M, int32_t* hout) {
  int64_t rc = check_args(c, hu, hv, E, V, hout);
  if (rc) return rc;
  if (V > (1 << 30)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  const int32_t* ru = nullptr;
  const int32_t* rv = nullptr;
  int32_t* dout = nullptr;
  bool deferred = false;
  rc = stage_host_edges(c, s, hu, hv, E, V, &ru, &rv, &dout, true, &deferred);
  if (rc) return rc;
  Carved k{};
  rc = 1;
  if (deferred)  // copies not issued yet: overlap them with the forest pass if the plan allows
    rc = run_path_host(c, s, hu, hv, const_cast<int32_t*>(ru), const_cast<int32_t*>(rv), E, V, M, dout, &k, true);
  if (rc < 0) return rc;
  if (rc == 1) {
    if (deferred && E > 0 &&
        (cudaMemcpyAsync(const_cast<int32_t*>(ru), hu, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, s) !=
             cudaSuccess ||
         cudaMemcpyAsync(const_cast<int32_t*>(rv), hv, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, s) !=
             cudaSuccess))
      return cuda_fail(cudaGetLastError());
    rc = run_path(c, s, ru, rv, E, V, M, dout, &k, nullptr, true, true);
    if (rc) return rc;
  }
  if (cudaMemcpyAsync(c->h_pinned, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  const int64_t n = c->h_pinned[0];
  if (n > 0) {
    if (cudaMemcpyAsync(hout, dout, sizeof(int32_t) * 2 * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return cuda_fail(cudaGetLastError());
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  }
  return n;
}

int64_t bridges_certificate(bridges_ctx* c, struct CUstream_st* stream, const int32_t* u, const int32_t* v, int64_t E,
                            int32_t V, int32_t M, int32_t* cu, int32_t* cv, uint8_t* ct) {
  int64_t rc = check_args(c, u, v, E, V, cu);
  if (rc) return rc;
  if (V > 1 && (!cv || !ct)) return BRIDGES_EINVAL;
  if (V > (1 << 30)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  Carved k{};
  CertPlan p{};
  rc = run_path(c, s, u, v, E, V, M, nullptr, &k, &p, false);
  if (rc) return rc;
  if (V > 1) cert_export(launch_for(c, s), p, k.cert, cu, cv, ct);
  // counts and status
  if (cudaMemcpyAsync(c->h_pinned, k.cert.cnt, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(c->h_pinned + 1, k.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  const int32_t* h = reinterpret_cast<const int32_t*>(c->h_pinned);
  const int32_t st = h[2];
  if (st) return st;
  const int64_t n = (int64_t)h[0] + h[1];
  return std::min<int64_t>(n, 2 * (int64_t)std::max(V - 1, 0));
}

int64_t bridges_from_forest(bridges_ctx* c, struct CUstream_st* stream, const int32_t* tu, const int32_t* tv,
                            int64_t n_tree, const int32_t* xu, const int32_t* xv, int64_t n_extra, int32_t V,
                            int32_t* out) {
  if (!c || V < 0 || n_tree < 0 || n_extra < 0) return BRIDGES_EINVAL;
  if (n_tree > std::max(V - 1, 0)) return BRIDGES_EINVAL;
  if ((n_tree > 0 && (!tu || !tv)) || (n_extra > 0 && (!xu || !xv)) || (V > 1 && !out)) return BRIDGES_EINVAL;
  if (n_extra > INT32_MAX || V > (1 << 30)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  CertPlan p = make_plan(0, V, 1, 2, 0, 0, 0, c->num_sms, c->smem_optin);
  int64_t rc = ensure_ws(c, total_bytes(p), s);
  if (rc) return rc;
  Carved k = carve(c, p);
  Launch L = launch_for(c, s);
  int32_t* h = reinterpret_cast<int32_t*>(c->h_pinned);
  // the pinned scratch may still be read by an earlier copy on another stream: wait for it
  cudaStreamSynchronize(s);
  h[0] = (int32_t)n_tree;
  h[1] = (int32_t)n_extra;
  cudaMemsetAsync(k.status, 0, sizeof(int32_t), s);
  cudaMemcpyAsync(k.counts, h, 2 * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  final_stage(L, k.fin, V, tu, tv, k.counts, n_tree, xu, xv, k.counts + 1, n_extra, nullptr, out ? out : k.spare);
  if (cudaGetLastError() != cudaSuccess) return BRIDGES_ECUDA;
  if (cudaMemcpyAsync(c->h_pinned + 1, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  return c->h_pinned[1];
}

int64_t bridges_rooted_forest(bridges_ctx* c, struct CUstream_st* stream, const int32_t* tu, const int32_t* tv,
                              int64_t n_tree, int32_t V, int32_t* out_parent, int32_t* out_pre, int32_t* out_size) {
  if (!c || V < 0 || n_tree < 0 || n_tree > std::max(V - 1, 0) || V > (1 << 30)) return BRIDGES_EINVAL;
  if (n_tree > 0 && (!tu || !tv)) return BRIDGES_EINVAL;
  if (V == 0) return BRIDGES_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  CertPlan p = make_plan(0, V, 1, 2, 0, 0, 0, c->num_sms, c->smem_optin);
  int64_t rc = ensure_ws(c, total_bytes(p), s);
  if (rc) return rc;
  Carved k = carve(c, p);
  Launch L = launch_for(c, s);
  int32_t* h = reinterpret_cast<int32_t*>(c->h_pinned);
  cudaStreamSynchronize(s);  // the pinned scratch may still be read by an earlier copy
  h[0] = (int32_t)n_tree;
  h[1] = 0;
  cudaMemsetAsync(k.status, 0, sizeof(int32_t), s);
  cudaMemcpyAsync(k.counts, h, 2 * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  // with no extra edges every tree edge is a bridge; the sorted list goes to dscan, which the
  // stage no longer reads once it sorts
  final_stage(L, k.fin, V, tu, tv, k.counts, n_tree, nullptr, nullptr, k.counts + 1, 0, nullptr, k.fin.dscan,
              /*ordered=*/true);
  const size_t bytes = sizeof(int32_t) * (size_t)V;
  if ((out_parent && cudaMemcpyAsync(out_parent, k.fin.par, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) ||
      (out_pre && cudaMemcpyAsync(out_pre, k.fin.pre, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) ||
      (out_size && cudaMemcpyAsync(out_size, k.fin.sz, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) ||
      cudaMemcpyAsync(c->h_pinned + 1, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  return c->h_pinned[1] < 0 ? c->h_pinned[1] : (int64_t)BRIDGES_OK;
}

int32_t bridges_ctx_stage_ms(const bridges_ctx* c, float* ms, int32_t n) {
  if (!c || !c->events || !ms || c->calls == 0) return 0;
  bridges_ctx* m = const_cast<bridges_ctx*>(c);
  resolve_timings(m, m->calls);
  const int s = (int)((m->calls - 1) % bridges_ctx::kRing);
  int32_t k = std::min<int32_t>(n, 6);
  for (int i = 0; i < k; i++) ms[i] = m->stage_ms[s][i];
  return k;
}

int32_t bridges_ctx_stage_ms_history(const bridges_ctx* c, float* ms, int32_t max_calls) {
  if (!c || !c->events || !ms || max_calls <= 0) return 0;
  bridges_ctx* m = const_cast<bridges_ctx*>(c);
  resolve_timings(m, m->calls);
  const int64_t n = std::min<int64_t>({(int64_t)max_calls, m->calls, (int64_t)bridges_ctx::kRing});
  for (int64_t i = 0; i < n; i++) {
    const int s = (int)((m->calls - n + i) % bridges_ctx::kRing);
    for (int j = 0; j < 6; j++) ms[6 * i + j] = m->stage_ms[s][j];
  }
  return (int32_t)n;
}

int64_t bridges_ctx_launches(const bridges_ctx* c) { return c ? c->launches : 0; }

int32_t bridges_ctx_last_config(const bridges_ctx* c, int64_t* vals, int32_t n) {
  if (!c || !vals) return 0;
  int32_t k = std::min<int32_t>(n, 8);
  for (int i = 0; i < k; i++) vals[i] = c->last_cfg[i];
  return k;
}

const char* bridges_status_string(int32_t st) {
  switch (st) {
    case BRIDGES_OK: return "ok";
    case BRIDGES_EINVAL: return "invalid argument";
    case BRIDGES_ERANGE: return "vertex id outside [0, V)";
    case BRIDGES_ENOMEM: return "workspace exceeds the memory budget or allocation failed";
    case BRIDGES_ECUDA: return "CUDA runtime error";
    case BRIDGES_ETIMEDOUT: return "bounded device wait gave up";
    case BRIDGES_EAGAIN: return "request can never fit the memory budget";
    case BRIDGES_EBUSY: return "result not ready";
    case BRIDGES_EINTERNAL: return "internal invariant failed";
    case BRIDGES_ECANCELED: return "request canceled";
    default: return "unknown status";
  }
}

}  // extern "C"

namespace {

// Layout of the batched workspace for the given capacities (bytes from the start).
struct BLayout {
  size_t args, ntasks, queue, tasks, corder, gerr, slots, total;
  size_t s_args, s_ntasks, s_tasks, s_corder, s_total;  // pinned staging
};

BLayout blayout(int64_t task_cap, int64_t graph_cap, int64_t slot_cap) {
  // The first s_total bytes of the device area (args, ntasks, tasks) are a byte copy of the
  // pinned staging area, so both use the same offsets for them.
  BLayout L{};
  size_t o = 0;
  L.args = L.s_args = o;
  o += align_up(sizeof(BatchArgs), 256);
  L.ntasks = L.s_ntasks = o;
  o += 256;
  L.tasks = L.s_tasks = o;
  o += align_up(sizeof(BatchTask) * (size_t)task_cap, 256);
  L.corder = L.s_corder = o;
  o += align_up(sizeof(int32_t) * (size_t)task_cap, 256);
  L.s_total = o;
  L.queue = o;
  o += 256;
  L.gerr = o;
  o += align_up(sizeof(int32_t) * (size_t)graph_cap, 256);
  L.slots = o;
  o += align_up(sizeof(uint32_t) * (size_t)std::max<int64_t>(slot_cap, 1), 256);
  L.total = o;
  return L;
}

int64_t next_pow2(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// (Re)creates the batched buffers and the two captured CUDA graphs for these capacities.
int64_t ensure_batched(bridges_ctx* c, cudaStream_t s, int64_t ntasks, int64_t G, int64_t slots) {
  if (ntasks <= c->b_task_cap && G <= c->b_graph_cap && slots <= c->b_slot_cap && c->b_exec[0] && c->b_exec[1])
    return BRIDGES_OK;
  const int64_t tcap = next_pow2(std::max<int64_t>(ntasks, 64)), gcap = next_pow2(std::max<int64_t>(G, 64));
  const int64_t scap = next_pow2(std::max<int64_t>(slots, 1024));
  const BLayout L = blayout(tcap, gcap, scap);
  if (c->user_ws) return BRIDGES_ENOMEM;
  if (c->budget && L.total + c->ws_bytes + c->stage_bytes > c->budget) return BRIDGES_ENOMEM;
  for (int k = 0; k < 2; k++)
    if (c->b_done_ev[k]) cudaEventSynchronize(c->b_done_ev[k]);
  cudaStreamSynchronize(s);
  for (int k = 0; k < 2; k++) {
    if (c->b_exec[k]) cudaGraphExecDestroy(c->b_exec[k]);
    if (c->bstage[k]) cudaFreeHost(c->bstage[k]);
    c->b_exec[k] = nullptr;
    c->bstage[k] = nullptr;
  }
  if (c->bws) cudaFree(c->bws);
  c->bws = nullptr;
  if (ctx_malloc(c, &c->bws, L.total) != cudaSuccess || cudaMallocHost(&c->bstage[0], L.s_total) != cudaSuccess ||
      cudaMallocHost(&c->bstage[1], L.s_total) != cudaSuccess) {
    cudaGetLastError();
    return BRIDGES_ENOMEM;
  }
  for (int k = 0; k < 2; k++)
    if (!c->b_done_ev[k] && cudaEventCreateWithFlags(&c->b_done_ev[k], cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(cudaGetLastError());
  c->b_task_cap = tcap;
  c->b_graph_cap = gcap;
  c->b_slot_cap = scap;
  c->bws_bytes = L.total;
  c->bstage_bytes = L.s_total;
  c->b_next = 0;
  // capture, once per staging copy: reset counters, upload descriptors from that copy, run the
  // kernel
  char* d = static_cast<char*>(c->bws);
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail(cudaGetLastError());
  bool ok = true;
  for (int k = 0; k < 2 && ok; k++) {
    cudaGraph_t graph;
    ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    ok = ok && cudaMemsetAsync(d + L.queue, 0, 256, cs) == cudaSuccess;
    ok = ok && cudaMemsetAsync(d + L.gerr, 0, L.slots - L.gerr, cs) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(d, c->bstage[k], L.s_total, cudaMemcpyHostToDevice, cs) == cudaSuccess;
    ok = ok && batched_launch(cs, reinterpret_cast<const BatchArgs*>(d + L.args), c->num_sms);
    ok = (cudaStreamEndCapture(cs, &graph) == cudaSuccess) && ok;
    if (ok) ok = cudaGraphInstantiate(&c->b_exec[k], graph, 0) == cudaSuccess;
    cudaGraphDestroy(graph);
  }
  cudaStreamDestroy(cs);
  if (!ok) {
    cudaGetLastError();
    for (int k = 0; k < 2; k++) {
      if (c->b_exec[k]) cudaGraphExecDestroy(c->b_exec[k]);
      c->b_exec[k] = nullptr;
    }
    return BRIDGES_ECUDA;
  }
  return BRIDGES_OK;
}

}  // namespace

namespace bridges {

// The bucket of a graph with V vertices under plan P (-1: the automatic plan).
static int batch_bucket(const bridges_batch_plan& P, int32_t V) {
  if (P.n <= 0) return -1;
  for (int b = 0; b < P.n; b++)
    if (V <= P.vmax[b]) return b;
  return P.n - 1;
}

// Applies the context's batched plan (see plan_batch_tasks in ctx.h).
int64_t plan_batch_tasks(const bridges_ctx* c, std::vector<BatchTask>& graphs, int64_t total_e,
                         std::vector<BatchTask>& tasks) {
  const bridges_batch_plan& P = c->bplan;
  const int64_t auto_split = default_split(c, total_e);
  int64_t slot = 0;
  tasks.clear();
  for (const BatchTask& g : graphs) {
    const int b = batch_bucket(P, g.V);
    const int64_t split = b >= 0 && P.split[b] > 0 ? P.split[b] : auto_split;
    const int64_t E = g.hi - g.lo;
    const int32_t np = (int32_t)std::min<int64_t>(64, std::max<int64_t>(1, (E + split - 1) / split));
    // the plan's group, raised to the smallest one the task fits (class 0 is the largest group)
    int cls = batch_min_class(g.V, np);
    if (b >= 0 && P.group[b] > 0) cls = std::min(cls, P.group[b] >= 1024 ? 0 : (P.group[b] >= 512 ? 1 : 2));
    int64_t warm = 4LL * g.V + 2048;  // measured on the batched workload against 2V + 1024, 8V + 2048, 16V + 2048
    if (b >= 0 && (P.warm_per_v[b] > 0 || P.warm_add[b] > 0)) warm = (int64_t)P.warm_per_v[b] * g.V + P.warm_add[b];
    for (int32_t p = 0; p < np; p++) {
      BatchTask t = g;
      t.lo = g.lo + E * p / np;
      t.hi = g.lo + E * (p + 1) / np;
      t.slot = slot + (int64_t)p * batch_slot_words(g.V);  // every task's certificate gets a slot
      t.part = p;
      t.nparts = np;
      t.cls = cls;
      t.warm = warm;
      tasks.push_back(t);
    }
    slot += (int64_t)np * batch_slot_words(g.V);
  }
  // whole-block tasks first, then the ones for half and for quarter blocks; largest first in each
  std::stable_sort(tasks.begin(), tasks.end(), [](const BatchTask& x, const BatchTask& y) {
    const int cx = batch_task_class(x), cy = batch_task_class(y);
    if (cx != cy) return cx < cy;
    return x.hi - x.lo > y.hi - y.lo;
  });
  return slot;
}

// Enqueues the two persistent launches over `tasks` (G graphs: certification, then the bridge
// stages) on stream s, through the context's cached CUDA graph.
int64_t launch_batch_tasks(bridges_ctx* c, cudaStream_t s, const std::vector<BatchTask>& tasks, int32_t G,
                           int64_t slot_words) {
  if (tasks.empty()) return BRIDGES_OK;
  Range range("bridges: batched launch");
  int64_t rc = ensure_batched(c, s, (int64_t)tasks.size(), G, slot_words);
  if (rc) return rc;
  // Two staging copies in turn: the host waits only for the batch before last (the last one to
  // read this copy), so it fills the next batch while the previous one runs.  The device area is
  // shared, so this batch also waits on the device for the previous one, whatever its stream.
  const int k = c->b_next;
  c->b_next ^= 1;
  cudaEventSynchronize(c->b_done_ev[k]);
  const BLayout L = blayout(c->b_task_cap, c->b_graph_cap, c->b_slot_cap);
  char* d = static_cast<char*>(c->bws);
  char* h = static_cast<char*>(c->bstage[k]);
  BatchArgs A{};
  A.tasks = reinterpret_cast<const BatchTask*>(d + L.tasks);
  A.corder = reinterpret_cast<const int32_t*>(d + L.corder);
  A.d_ntasks = reinterpret_cast<const int32_t*>(d + L.ntasks);
  A.queue = reinterpret_cast<int32_t*>(d + L.queue);
  A.gerr = reinterpret_cast<int32_t*>(d + L.gerr);
  A.slots = reinterpret_cast<uint32_t*>(d + L.slots);
  A.G = G;
  // the class boundaries of the ordered list; a list out of class order runs every task on whole
  // blocks (always correct)
  const int32_t n = (int32_t)tasks.size();
  int32_t nbig = 0, nmid = 0;
  while (nbig < n && batch_task_class(tasks[nbig]) == 0) nbig++;
  while (nbig + nmid < n && batch_task_class(tasks[nbig + nmid]) == 1) nmid++;
  for (int32_t i = nbig + nmid; i < n; i++)
    if (batch_task_class(tasks[i]) != 2) {
      nbig = n;
      nmid = 0;
      break;
    }
  A.nbig = nbig;
  A.nmid = nmid;
  // certification order: most edges first
  std::vector<int32_t>& order = c->b_order;
  order.resize(n);
  for (int32_t i = 0; i < n; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    return tasks[x].hi - tasks[x].lo > tasks[y].hi - tasks[y].lo;
  });
  // the tail of small tasks that one group per SM takes from the back
  int32_t nback = 0;
  while (nback < n && tasks[order[n - 1 - nback]].hi - tasks[order[n - 1 - nback]].lo <= c->b_back_edges) nback++;
  A.nback = nback;
  A.slot_words = c->b_slot_cap;
  std::memcpy(h + L.s_args, &A, sizeof(A));
  const int32_t nt = (int32_t)tasks.size();
  std::memcpy(h + L.s_ntasks, &nt, sizeof(nt));
  std::memcpy(h + L.s_tasks, tasks.data(), sizeof(BatchTask) * tasks.size());
  std::memcpy(h + L.s_corder, order.data(), sizeof(int32_t) * tasks.size());
  if (cudaStreamWaitEvent(s, c->b_done_ev[k ^ 1], 0) != cudaSuccess) return cuda_fail(cudaGetLastError());
  if (cudaGraphLaunch(c->b_exec[k], s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  if (cudaEventRecord(c->b_done_ev[k], s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  c->launches += 2;
  return BRIDGES_OK;
}

// The automatic split: the batch's edges over three certification groups per SM (there are
// four), no task above 2^20 edges and none below 2^17 (every task pays its own warm-up prefix).
// A small batch then cuts its large graphs finer, so that the launch does not wait on its one
// longest graph (512 graphs of the batched workload: 0.30 ms against 0.50 with 2^20 alone);
// the 4,096-graph batch keeps 2^20 (0.881 M edges a task with four groups per SM was 2% slower).
int64_t default_split(const bridges_ctx* c, int64_t total_e) {
  if (c->b_split_edges > 0) return c->b_split_edges;
  return std::min<int64_t>(1 << 20, std::max<int64_t>(1 << 17, total_e / std::max(1, c->num_sms * 3)));
}

// The single-graph path on a context, count copied to count_dev (device).
int64_t run_single(bridges_ctx* c, cudaStream_t s, const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t M,
                   int32_t* out, int64_t* count_dev) {
  Carved k{};
  int64_t rc = run_path(c, s, u, v, E, V, M, out, &k, nullptr, true, true);
  if (rc) return rc;
  if (cudaMemcpyAsync(count_dev, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  return BRIDGES_OK;
}

size_t single_workspace_bytes(const bridges_ctx* c, int64_t E, int32_t V) { return total_bytes(plan_for(c, E, V, 0)); }

}  // namespace bridges

extern "C" int64_t bridges_find_batched(bridges_ctx* c, struct CUstream_st* stream, const int32_t* u, const int32_t* v,
                                        const int64_t* edge_off, const int32_t* Vs, int32_t G, int32_t* out,
                                        int64_t* out_counts) {
  if (!c || G < 0 || (G > 0 && (!edge_off || !Vs || !out_counts))) return BRIDGES_EINVAL;
  if (G == 0) return BRIDGES_OK;
  int64_t total_out = 0, total_e = 0;
  for (int32_t g = 0; g < G; g++) {
    if (Vs[g] < 0 || Vs[g] > (1 << 30) || edge_off[g] < 0 || edge_off[g + 1] < edge_off[g]) return BRIDGES_EINVAL;
    total_out += 2 * (int64_t)std::max(Vs[g] - 1, 0);
    total_e += edge_off[g + 1] - edge_off[g];
  }
  if (total_e > 0 && (!u || !v)) return BRIDGES_EINVAL;
  if (total_out > 0 && !out) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  // small graphs become batch tasks; graphs above the shared-memory size take the single-graph
  // path afterwards on the same stream
  std::vector<BatchTask> graphs, tasks;
  std::vector<int32_t> large;
  std::vector<int64_t> out_off(G);
  int64_t o = 0;
  for (int32_t g = 0; g < G; g++) {
    out_off[g] = o;
    o += 2 * (int64_t)std::max(Vs[g] - 1, 0);
    if (Vs[g] > kBatchVmax) {
      large.push_back(g);
      continue;
    }
    BatchTask t{};
    t.u = u;
    t.v = v;
    t.lo = edge_off[g];
    t.hi = edge_off[g + 1];
    t.out = out ? out + out_off[g] : nullptr;
    t.count = out_counts + g;
    t.g = (int32_t)graphs.size();
    t.V = Vs[g];
    graphs.push_back(t);
  }
  const int64_t slots = plan_batch_tasks(c, graphs, total_e, tasks);
  int64_t rc = launch_batch_tasks(c, s, tasks, (int32_t)graphs.size(), slots);
  if (rc) return rc;
  for (int32_t g : large) {
    rc = run_single(c, s, u + edge_off[g], v + edge_off[g], edge_off[g + 1] - edge_off[g], Vs[g], 0, out + out_off[g],
                    out_counts + g);
    if (rc) return rc;
  }
  return BRIDGES_OK;
}

extern "C" int32_t bridges_ctx_set_batch_split(bridges_ctx* c, int64_t split_edges) {
  if (!c || split_edges < 0) return BRIDGES_EINVAL;
  c->b_split_edges = split_edges;
  return BRIDGES_OK;
}

extern "C" int32_t bridges_ctx_set_batch_plan(bridges_ctx* c, const bridges_batch_plan* P) {
  if (!c || !P || P->n < 0 || P->n > BRIDGES_BATCH_BUCKETS) return BRIDGES_EINVAL;
  for (int b = 0; b < P->n; b++) {
    const int32_t g = P->group[b];
    if ((b > 0 && P->vmax[b] <= P->vmax[b - 1]) || P->vmax[b] < 0 || (g != 0 && g != 256 && g != 512 && g != 1024) ||
        P->split[b] < 0 || P->warm_per_v[b] < 0 || P->warm_add[b] < 0)
      return BRIDGES_EINVAL;
  }
  c->bplan = *P;
  return BRIDGES_OK;
}

extern "C" int32_t bridges_ctx_get_batch_plan(const bridges_ctx* c, bridges_batch_plan* P) {
  if (!c || !P) return BRIDGES_EINVAL;
  *P = c->bplan;
  return BRIDGES_OK;
}

// Batched autotuner: coordinate descent over the buckets' group, split and warm-up choices,
// each candidate timed over whole batched calls (a bucket's choices interact with the others'
// only through the shared queue, so one bucket is changed at a time, largest first, twice over).
extern "C" int32_t bridges_batch_autotune(bridges_ctx* c, struct CUstream_st* stream, const int32_t* u,
                                          const int32_t* v, const int64_t* edge_off, const int32_t* Vs, int32_t G,
                                          int32_t reps, bridges_batch_plan* best, double* best_us) {
  if (!c || G <= 0 || !edge_off || !Vs) return BRIDGES_EINVAL;
  int64_t total_out = 0;
  for (int32_t g = 0; g < G; g++) {
    if (Vs[g] < 0 || Vs[g] > (1 << 30) || edge_off[g] < 0 || edge_off[g + 1] < edge_off[g]) return BRIDGES_EINVAL;
    total_out += 2 * (int64_t)std::max(Vs[g] - 1, 0);
  }
  if (edge_off[G] > 0 && (!u || !v)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return (int32_t)cuda_fail(cudaGetLastError());
  if (reps <= 0) reps = 3;
  int32_t* out = nullptr;
  int64_t* cnt = nullptr;
  if (cudaMalloc(&out, sizeof(int32_t) * (size_t)std::max<int64_t>(total_out, 1)) != cudaSuccess ||
      cudaMalloc(&cnt, sizeof(int64_t) * (size_t)G) != cudaSuccess) {
    cudaGetLastError();
    if (out) cudaFree(out);
    return BRIDGES_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bridges_batch_plan saved = c->bplan;
  int32_t rc = BRIDGES_OK;
  // time of one batched call under plan P (ms), or a negative value on error
  auto time_plan = [&](const bridges_batch_plan& P) -> float {
    c->bplan = P;
    int64_t r = bridges_find_batched(c, stream, u, v, edge_off, Vs, G, out, cnt);  // untimed: first use
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps && !r; i++) r = bridges_find_batched(c, stream, u, v, edge_off, Vs, G, out, cnt);
    cudaEventRecord(e1, s);
    if (r || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = r ? (int32_t)r : (int32_t)BRIDGES_ECUDA;
      return -1.0f;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
  };
  bridges_batch_plan cur{};
  const int32_t vmax[5] = {256, 512, 1024, 2048, kBatchVmax};
  cur.n = 5;
  for (int b = 0; b < 5; b++) cur.vmax[b] = vmax[b];
  std::vector<int> present(5, 0);
  for (int32_t g = 0; g < G; g++)
    if (Vs[g] <= kBatchVmax) present[batch_bucket(cur, Vs[g])] = 1;
  const bridges_batch_plan automatic = cur;
  float best_ms = time_plan(cur);
  // a change is kept only when it is faster by more than the timing noise of a few calls: the
  // minimum over many noisy candidates otherwise drifts to a plan that is merely lucky
  constexpr float kMargin = 0.995f;
  for (int pass = 0; pass < 2 && rc == BRIDGES_OK; pass++) {
    for (int b = 4; b >= 0 && rc == BRIDGES_OK; b--) {
      if (!present[b]) continue;
      auto consider = [&](const bridges_batch_plan& P) {
        const float ms = time_plan(P);
        if (ms >= 0 && ms < best_ms * kMargin) {
          best_ms = ms;
          cur = P;
        }
      };
      for (int32_t grp : {1024, 512, 256}) {  // groups the bucket's largest graph fits
        if ((grp == 256 && vmax[b] > kBatchQuarterVmax) || (grp == 512 && vmax[b] > kBatchHalfVmax)) continue;
        bridges_batch_plan P = cur;
        P.group[b] = grp;
        if (P.group[b] != cur.group[b]) consider(P);
      }
      for (int64_t sp : {(int64_t)0, (int64_t)1 << 18, (int64_t)1 << 19, (int64_t)1 << 20, (int64_t)1 << 21,
                         (int64_t)1 << 22}) {
        bridges_batch_plan P = cur;
        P.split[b] = sp;
        if (P.split[b] != cur.split[b]) consider(P);
      }
      const int32_t warms[3][2] = {{4, 2048}, {2, 1024}, {8, 2048}};
      for (const auto& w : warms) {
        bridges_batch_plan P = cur;
        P.warm_per_v[b] = w[0];
        P.warm_add[b] = w[1];
        if (P.warm_per_v[b] != cur.warm_per_v[b] || P.warm_add[b] != cur.warm_add[b]) consider(P);
      }
    }
  }
  // the search's plan against the automatic one, timed in turn over more calls: the automatic
  // plan stays unless the other is faster beyond the margin
  auto same_plan = [](const bridges_batch_plan& x, const bridges_batch_plan& y) {
    if (x.n != y.n) return false;
    for (int b = 0; b < x.n && b < BRIDGES_BATCH_BUCKETS; b++)
      if (x.vmax[b] != y.vmax[b] || x.group[b] != y.group[b] || x.split[b] != y.split[b] ||
          x.warm_per_v[b] != y.warm_per_v[b] || x.warm_add[b] != y.warm_add[b])
        return false;
    return true;
  };
  if (rc == BRIDGES_OK && !same_plan(cur, automatic)) {
    float t_cur = 0, t_auto = 0;
    for (int k = 0; k < 3 && rc == BRIDGES_OK; k++) {
      const float a = time_plan(automatic), b = time_plan(cur);
      t_auto += a;
      t_cur += b;
    }
    if (rc == BRIDGES_OK) {
      if (t_cur < t_auto * kMargin) {
        best_ms = t_cur / 3;
      } else {
        cur = automatic;
        best_ms = t_auto / 3;
      }
    }
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  cudaFree(cnt);
  c->bplan = rc ? saved : cur;
  if (rc) return rc;
  if (best) *best = cur;
  if (best_us) *best_us = (double)best_ms * 1000.0;
  return BRIDGES_OK;
}

// ---------------------------------------------------------------------------------------------
// Autotuner: times candidate plans on the caller's input and keeps the fastest in the context.
extern "C" int32_t bridges_autotune(bridges_ctx* c, struct CUstream_st* stream, const int32_t* u, const int32_t* v,
                                    int64_t E, int32_t V, int32_t reps, int64_t* best) {
  if (!c || E < 0 || V < 0 || (E > 0 && (!u || !v)) || !best) return BRIDGES_EINVAL;
  if (V > (1 << 30)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return (int32_t)cuda_fail(cudaGetLastError());
  if (reps <= 0) reps = 3;
  int32_t* out = nullptr;
  int64_t* cnt = nullptr;
  if (cudaMalloc(&out, sizeof(int32_t) * 2 * (size_t)std::max(V, 1)) != cudaSuccess ||
      cudaMalloc(&cnt, sizeof(int64_t)) != cudaSuccess) {
    cudaGetLastError();
    if (out) cudaFree(out);
    return BRIDGES_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bridges_opts saved = c->opts;
  const double lnv = std::log((double)V + 1.0);
  float best_ms = 1e30f;
  bridges_opts best_o = saved;
  int32_t rc = BRIDGES_OK;
  const int32_t Ms[] = {1, 2, 4, 8, 16, 32};
  const double warms[] = {0.3, 0.45, 0.6, 0.8, 1.2, 2.0};
  const int32_t blocks[] = {1024, 768, 512};
  for (int32_t M : Ms) {
    if (M > 1 && (int64_t)M > std::max<int64_t>(E, 1)) break;
    for (int32_t f : {2, M}) {
      if (M == 1 && f != 2) continue;
      if (M > 1 && f == 2 && M == 2) continue;  // same as f = M
      for (double w : warms) {
        for (int32_t blk : blocks) {
          bridges_opts o = saved;
          o.M = M;
          o.fan_in = f;
          o.block = blk;
          o.warm_edges = (int64_t)std::ceil(w * V * lnv) + 4096;
          o.profile = 0;
          c->opts = o;
          // one untimed run (workspace growth, first-touch), then reps timed runs
          int64_t r = BRIDGES_OK;
          Carved k{};
          r = run_path(c, s, u, v, E, V, 0, out, &k, nullptr, true, true);
          if (r) {
            rc = (int32_t)r;
            break;
          }
          cudaEventRecord(e0, s);
          for (int i = 0; i < reps && !r; i++) r = run_path(c, s, u, v, E, V, 0, out, &k, nullptr, true, true);
          cudaEventRecord(e1, s);
          if (r || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = r ? (int32_t)r : (int32_t)BRIDGES_ECUDA;
            break;
          }
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          ms /= reps;
          if (ms < best_ms) {
            best_ms = ms;
            best_o = o;
          }
        }
        if (rc) break;
      }
      if (rc) break;
    }
    if (rc) break;
  }
  // refinement: the warm-up launch's block size for the chosen plan
  for (int32_t wb : {128, 256, 512, 1024}) {
    if (rc) break;
    bridges_opts o = best_o;
    o.warm_block = wb;
    o.profile = 0;
    c->opts = o;
    Carved k{};
    int64_t r = run_path(c, s, u, v, E, V, 0, out, &k, nullptr, true, true);
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps && !r; i++) r = run_path(c, s, u, v, E, V, 0, out, &k, nullptr, true, true);
    cudaEventRecord(e1, s);
    if (r || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = r ? (int32_t)r : (int32_t)BRIDGES_ECUDA;
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms < best_ms) {
      best_ms = ms;
      best_o = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  cudaFree(cnt);
  best_o.profile = saved.profile;
  best_o.host_read = saved.host_read;
  c->opts = rc ? saved : best_o;
  best[0] = best_o.M;
  best[1] = best_o.fan_in;
  best[2] = best_o.warm_edges;
  best[3] = best_o.block;
  best[4] = (int64_t)(best_ms * 1000.0f);  // microseconds per call
  return rc;
}

extern "C" int32_t bridges_ctx_get_opts(const bridges_ctx* c, bridges_opts* o) {
  if (!c || !o) return BRIDGES_EINVAL;
  *o = c->opts;
  return BRIDGES_OK;
}

// Sets the tuning options of a context (e.g. from a cache of autotune results).
extern "C" int32_t bridges_ctx_set_opts(bridges_ctx* c, const bridges_opts* o) {
  if (!c || !o) return BRIDGES_EINVAL;
  const int32_t prof = c->opts.profile;
  c->opts = *o;
  c->opts.profile = prof;  // event slots exist only if created with profiling
  c->allocs = 0;           // opts.test_fail_alloc counts from here
  return BRIDGES_OK;
}

// ---------------------------------------------------------------------------------------------
// A bounded device-side wait on a flag (the primitive behind the library's barriers).
namespace {
__global__ void wait_value_kernel(const int32_t* flag, int32_t value, unsigned long long max_polls, int32_t* status) {
  const bool ok = bounded_poll([&] { return ld_acquire_s32(flag) == value; }, max_polls);
  *status = ok ? BRIDGES_OK : BRIDGES_ETIMEDOUT;
}
}  // namespace

extern "C" int32_t bridges_wait_value(bridges_ctx* c, struct CUstream_st* stream, const int32_t* flag, int32_t value,
                                      int64_t max_polls) {
  if (!c || !flag || max_polls < 0) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return (int32_t)cuda_fail(cudaGetLastError());
  int64_t rc = ensure_ws(c, kMiscBytes, s);
  if (rc) return (int32_t)rc;
  int32_t* st = static_cast<int32_t*>(c->ws);
  wait_value_kernel<<<1, 1, 0, s>>>(flag, value, (unsigned long long)max_polls, st);
  c->launches += 1;
  if (cudaMemcpyAsync(c->h_pinned, st, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return (int32_t)cuda_fail(cudaGetLastError());
  return *reinterpret_cast<int32_t*>(c->h_pinned);
}

// ---------------------------------------------------------------------------------------------
// 2-edge-connected components and incremental sessions on a resident certificate.
extern "C" int64_t bridges_two_edge_components(bridges_ctx* c, struct CUstream_st* stream, const int32_t* u,
                                               const int32_t* v, int64_t E, int32_t V, int32_t M, int32_t* labels,
                                               int32_t* out_bridges) {
  int64_t rc = check_args(c, u, v, E, V, labels);
  if (rc) return rc;
  if (V > (1 << 30)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  // the bridges go to the caller's buffer or to the (then unused) workspace key area
  Carved k{};
  CertPlan p{};
  rc = run_path(c, s, u, v, E, V, M, out_bridges, &k, &p);
  if (rc) return rc;
  Launch L = launch_for(c, s);
  two_edge_components(L, k.fin, V, k.cert.f2u, k.cert.f2v, k.cert.cnt + 1, V, labels, k.fin.count);
  if (cudaMemcpyAsync(c->h_pinned, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  return c->h_pinned[0];
}

// ---------------------------------------------------------------------------------------------
// Articulation points: the bridge path, then the block pass over the same edges.
// Edges of the list offered to the block pass before its snapshot (after the certificate's).
static int64_t ap_warm_edges(const bridges_ctx* c, int64_t E, int32_t V) {
  const int32_t w = c->opts.ap_warm_edges;
  if (w < 0) return 0;
  if (w > 0) return std::min<int64_t>(w, E);
  return std::min<int64_t>(E, 2 * (int64_t)V + 4096);
}

// The plan of the two-pass block pass: the whole list as one
// partition, its own prefix before the snapshot.
static CertPlan block_pass_plan(const bridges_ctx* c, int64_t E, int32_t V) {
  CertPlan q = plan_for(c, E, V, 1);
  q.warm = ap_warm_edges(c, E, V);
  // The plan's snapshot form: 16-bit labels when 2V bytes fit in shared memory, else a bitmap of
  // the largest class, taken only when it reaches every vertex (R-MAT, 2^21 vertices, 1.85 M in
  // reach: 0.71 ms for the block pass with it, 0.66 without).  With the bitmap the automatic
  // prefix is none: the certificate's blocks already seed the classes (R-MAT 2^18 / 2^20: 0.12 /
  // 0.22 ms without a prefix, 0.16 / 0.31 ms with 2V + 4096 edges, 0.21 / 0.59 ms with no snapshot).
  if (q.mode == 2 && c->opts.ap_warm_edges == 0) q.warm = 0;
  q.cache = (q.mode == 1 || (q.mode == 2 && q.Vb >= V)) && q.warm < E;
  return q;
}

// One read of the list for both passes: one partition with a 16-bit label snapshot.
static bool fused_eligible(const bridges_ctx* c, const CertPlan& p, int64_t E, int32_t V) {
  return c->opts.ap_fused >= 0 && p.M == 1 && p.cache && p.mode == 1 && V >= 2 && E > p.warm;
}

// Workspace of the fused form: the bridge path's, two sets of class buffers (T_0's, the final
// T's) and one mark per edge.
static size_t fused_ws_bytes(const CertPlan& p, int32_t V) {
  return align_up(total_bytes(p), 256) + 2 * align_up(ap_bytes(V), 256) + fused_bytes(p.E);
}

// The fused form.  With host edges (hu, hv) not yet on the device, (u, v) is their device
// staging: the copy runs in chunks and the stream follows it chunk by chunk.
static int64_t articulation_fused_run(bridges_ctx* c, cudaStream_t s, const Launch& L, const CertPlan& p,
                                      const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t* out_points,
                                      int32_t* out_bridges, int64_t* out_counts_device, const int32_t* hu,
                                      const int32_t* hv) {
  Range range("bridges: articulation points, fused");
  const size_t ap_at = align_up(total_bytes(p), 256);
  const size_t apb = align_up(ap_bytes(V), 256);
  int64_t rc = ensure_ws(c, fused_ws_bytes(p, V), s);
  if (rc) return rc;
  Carved k = carve(c, p);
  if (!out_points) out_points = k.spare;  // V <= 1: no point is written
  char* ws = static_cast<char*>(c->ws);
  const ApBufs b0 = carve_ap(ws + ap_at, V);
  const ApBufs b1 = carve_ap(ws + ap_at + apb, V);
  const FusedBufs fb = carve_fused(ws + ap_at + 2 * apb, E);
  c->last_cfg[0] = p.M;
  c->last_cfg[1] = p.f;
  c->last_cfg[2] = p.G;
  c->last_cfg[3] = p.block;
  c->last_cfg[4] = p.warm;
  c->last_cfg[5] = p.warm;
  c->last_cfg[6] = p.G;
  c->last_cfg[7] = 1;
  cudaEvent_t* bev = next_event_slot(c);
  if (bev) cudaEventRecord(bev[7], s);
  cudaEvent_t* aev = nullptr;
  if (c->events) {
    resolve_ap_timings(c, c->ap_calls - bridges_ctx::kRing + 1);  // the slot's previous call
    aev = c->ap_ev[c->ap_calls % bridges_ctx::kRing];
  }
  ChunkSchedule chunks{};
  if (hu) {
    int64_t C = 0;
    int K = 0;
    if (chunk_plan(E, p.warm, &C, &K)) {
      rc = issue_chunks(c, s, hu, hv, const_cast<int32_t*>(u), const_cast<int32_t*>(v), E, C, K);
      if (rc) return rc;
      chunks = ChunkSchedule{c->chunk_ev, C, K};
    } else if (E > 0 &&
               (cudaMemcpyAsync(const_cast<int32_t*>(u), hu, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess ||
                cudaMemcpyAsync(const_cast<int32_t*>(v), hv, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess)) {
      return cuda_fail(cudaGetLastError());
    }
  }
  cudaMemsetAsync(k.status, 0, sizeof(int32_t), s);
  cert_init(L, p, k.cert);
  articulation_fused(L, p, k.cert, k.fin, b0, b1, fb, u, v, out_points, out_bridges, b1.count, bev, aev, chunks);
  if (bev) c->calls++;
  if (aev) c->ap_calls++;
  if (cudaGetLastError() != cudaSuccess) return BRIDGES_ECUDA;
  if (out_counts_device) {
    if (cudaMemcpyAsync(out_counts_device, b1.count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(out_counts_device + 1, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
      return cuda_fail(cudaGetLastError());
    return BRIDGES_OK;
  }
  if (cudaMemcpyAsync(c->h_pinned, b1.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  return c->h_pinned[0];
}

// The articulation-point path on device edges (u, v).  When hu / hv are given (and the edges
// were not copied yet), the bridge path's forest pass runs behind a chunked copy of them into
// (u, v) (run_path_host); the block pass then streams (u, v) from the device.
static int64_t articulation_run(bridges_ctx* c, cudaStream_t s, const int32_t* u, const int32_t* v, int64_t E, int32_t V,
                         int32_t M, int32_t* out_points, int32_t* out_bridges, int64_t* out_counts_device,
                         const int32_t* hu, const int32_t* hv) {
  const CertPlan p0 = plan_for(c, E, V, M);
  const size_t ap_at = align_up(total_bytes(p0), 256);
  Launch L = launch_for(c, s);
  // the fused form when it applies and its larger workspace fits the caller's limits, else two passes
  if (fused_eligible(c, p0, E, V) && ws_fits(c, fused_ws_bytes(p0, V)))
    return articulation_fused_run(c, s, L, p0, u, v, E, V, out_points, out_bridges, out_counts_device, hu, hv);
  int64_t rc = ensure_ws(c, ap_at + ap_bytes(V), s);
  if (rc) return rc;
  Carved k{};
  c->last_cfg[7] = 0;
  rc = 1;
  if (hu) {
    // the rooted forest is needed either way; without a bridge buffer the bridges go to dscan,
    // free by the time the final stage sorts
    const Carved k0 = carve(c, p0);
    rc = run_path_host(c, s, hu, hv, const_cast<int32_t*>(u), const_cast<int32_t*>(v), E, V, M,
                       out_bridges ? out_bridges : k0.fin.dscan, &k, false);
    if (rc < 0) return rc;
    if (rc == 1 && E > 0 &&
        (cudaMemcpyAsync(const_cast<int32_t*>(u), hu, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, s) !=
             cudaSuccess ||
         cudaMemcpyAsync(const_cast<int32_t*>(v), hv, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, s) !=
             cudaSuccess))
      return cuda_fail(cudaGetLastError());
  }
  if (rc == 1) {
    rc = run_path(c, s, u, v, E, V, M, out_bridges, &k, nullptr);
    if (rc) return rc;
  }
  if (!out_points) out_points = k.spare;  // V <= 1: no point is written
  Range range("bridges: articulation block pass");
  ApBufs b = carve_ap(static_cast<char*>(c->ws) + ap_at, V);
  // the block pass streams the whole list as one partition, its own warm-up before the snapshot
  const CertPlan q = block_pass_plan(c, E, V);
  c->last_cfg[5] = q.cache ? q.warm : -1;
  c->last_cfg[6] = (int64_t)q.G * q.M;
  cudaEvent_t* ev = nullptr;
  if (c->events) {
    resolve_ap_timings(c, c->ap_calls - bridges_ctx::kRing + 1);  // the slot's previous call
    ev = c->ap_ev[c->ap_calls % bridges_ctx::kRing];
    cudaEventRecord(ev[0], s);
  }
  articulation_stage(L, q, k.fin, b, u, v, k.cert.f2u, k.cert.f2v, k.cert.cnt + 1, out_points, b.count,
                     ev ? ev + 1 : nullptr);
  if (ev) {
    cudaEventRecord(ev[4], s);
    c->ap_calls++;
  }
  if (cudaGetLastError() != cudaSuccess) return BRIDGES_ECUDA;
  if (out_counts_device) {
    if (cudaMemcpyAsync(out_counts_device, b.count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(out_counts_device + 1, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
      return cuda_fail(cudaGetLastError());
    return BRIDGES_OK;
  }
  if (cudaMemcpyAsync(c->h_pinned, b.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  return c->h_pinned[0];
}

extern "C" int64_t bridges_articulation_points(bridges_ctx* c, struct CUstream_st* stream, const int32_t* u,
                                               const int32_t* v, int64_t E, int32_t V, int32_t M,
                                               int32_t* out_points, int32_t* out_bridges,
                                               int64_t* out_counts_device) {
  int64_t rc = check_args(c, u, v, E, V, out_points);
  if (rc) return rc;
  if (V > (1 << 30)) return BRIDGES_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  return articulation_run(c, reinterpret_cast<cudaStream_t>(stream), u, v, E, V, M, out_points, out_bridges,
                          out_counts_device, nullptr, nullptr);
}

extern "C" int64_t bridges_articulation_points_host(bridges_ctx* c, struct CUstream_st* stream, const int32_t* hu,
                                                    const int32_t* hv, int64_t E, int32_t V, int32_t M,
                                                    int32_t* out_points_host) {
  int64_t rc = check_args(c, hu, hv, E, V, out_points_host);
  if (rc) return rc;
  if (V > (1 << 30)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  const int32_t* ru = nullptr;
  const int32_t* rv = nullptr;
  int32_t* dout = nullptr;
  bool deferred = false;
  rc = stage_host_edges(c, s, hu, hv, E, V, &ru, &rv, &dout, true, &deferred);
  if (rc) return rc;
  const int64_t n = articulation_run(c, s, ru, rv, E, V, M, dout, nullptr, nullptr, deferred ? hu : nullptr,
                                     deferred ? hv : nullptr);
  if (n <= 0) return n;
  if (cudaMemcpyAsync(out_points_host, dout, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  return n;
}

extern "C" int64_t bridges_articulation_workspace_bytes(const bridges_ctx* c, int64_t E, int32_t V, int32_t M) {
  if (!c || E < 0 || V < 0) return 0;
  const CertPlan p = plan_for(c, E, V, M);
  const size_t two_pass = align_up(total_bytes(p), 256) + ap_bytes(V);
  if (!fused_eligible(c, p, E, V)) return (int64_t)two_pass;
  return (int64_t)std::max(two_pass, fused_ws_bytes(p, V));
}

extern "C" int32_t bridges_ctx_ap_stage_ms(const bridges_ctx* c, float* ms, int32_t n) {
  if (!c || !c->events || !ms || n <= 0 || c->ap_calls == 0) return 0;
  bridges_ctx* m = const_cast<bridges_ctx*>(c);
  resolve_ap_timings(m, m->ap_calls);
  const int s = (int)((m->ap_calls - 1) % bridges_ctx::kRing);
  const int32_t k = std::min(n, 5);
  for (int i = 0; i < k; i++) ms[i] = m->ap_ms[s][i];
  return k;
}

extern "C" int32_t bridges_ctx_ap_stage_ms_history(const bridges_ctx* c, float* ms, int32_t max_calls) {
  if (!c || !c->events || !ms || max_calls <= 0) return 0;
  bridges_ctx* m = const_cast<bridges_ctx*>(c);
  resolve_ap_timings(m, m->ap_calls);
  const int64_t n = std::min<int64_t>({(int64_t)max_calls, m->ap_calls, (int64_t)bridges_ctx::kRing});
  for (int64_t i = 0; i < n; i++) {
    const int s = (int)((m->ap_calls - n + i) % bridges_ctx::kRing);
    for (int j = 0; j < 5; j++) ms[5 * i + j] = m->ap_ms[s][j];
  }
  return (int32_t)n;
}

struct bridges_inc {
  bridges_ctx* ctx = nullptr;
  bool ready = false;
  int32_t V = 0;
  CertPlan p{};
  Carved k{};
};

extern "C" bridges_inc* bridges_inc_create(int device, const bridges_opts* opts) {
  bridges_inc* I = new (std::nothrow) bridges_inc();
  if (!I) return nullptr;
  I->ctx = bridges_ctx_create(device, 0, opts);
  if (!I->ctx) {
    delete I;
    return nullptr;
  }
  return I;
}

extern "C" void bridges_inc_destroy(bridges_inc* I) {
  if (!I) return;
  bridges_ctx_destroy(I->ctx);
  delete I;
}

extern "C" int64_t bridges_inc_reset(bridges_inc* I, struct CUstream_st* stream, const int32_t* u, const int32_t* v,
                                     int64_t E, int32_t V, int32_t M, int32_t* out_bridges) {
  if (!I) return BRIDGES_EINVAL;
  I->ready = false;
  int64_t rc = check_args(I->ctx, u, v, E, V, out_bridges);
  if (rc) return rc;
  if (V > (1 << 30)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(I->ctx->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  rc = run_path(I->ctx, s, u, v, E, V, M, out_bridges, &I->k, &I->p);
  if (rc) return rc;
  if (cudaMemcpyAsync(I->ctx->h_pinned, I->k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  const int64_t n = I->ctx->h_pinned[0];
  I->V = V;
  I->ready = n >= 0;
  return n;
}

extern "C" int64_t bridges_inc_add(bridges_inc* I, struct CUstream_st* stream, const int32_t* yu, const int32_t* yv,
                                   int64_t n, int32_t* out_bridges) {
  if (!I || !I->ready || n < 0 || (n > 0 && (!yu || !yv)) || (I->V > 1 && !out_bridges)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  bridges_ctx* c = I->ctx;
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  Launch L = launch_for(c, s);
  const Carved& k = I->k;
  const int32_t V = I->V;
  if (cudaMemsetAsync(k.status, 0, sizeof(int32_t), s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  cert_offer(L, I->p, k.cert, yu, yv, n);
  final_stage(L, k.fin, V, k.cert.f1u, k.cert.f1v, k.cert.cnt + 0, V, k.cert.f2u, k.cert.f2v, k.cert.cnt + 1, V,
              k.cert.P1, out_bridges ? out_bridges : k.spare);
  if (cudaMemcpyAsync(c->h_pinned, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  return c->h_pinned[0];
}

extern "C" int64_t bridges_inc_two_edge_components(bridges_inc* I, struct CUstream_st* stream, int32_t* labels) {
  if (!I || !I->ready || (I->V > 0 && !labels)) return BRIDGES_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  bridges_ctx* c = I->ctx;
  if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError());
  Launch L = launch_for(c, s);
  const Carved& k = I->k;
  two_edge_components(L, k.fin, I->V, k.cert.f2u, k.cert.f2v, k.cert.cnt + 1, I->V, labels, k.fin.count);
  if (cudaMemcpyAsync(c->h_pinned, k.fin.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  return c->h_pinned[0];
}

extern "C" int64_t bridges_inc_certificate_size(const bridges_inc* I) {
  if (!I || !I->ready) return BRIDGES_EINVAL;
  int32_t h[2] = {0, 0};
  if (cudaMemcpy(h, I->k.cert.cnt, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  return (int64_t)h[0] + h[1];
}
