// ctx.h -- the context object behind bridges_ctx* and the host helpers the server shares with
// the plain and batched entry points.  Nothing here is part of the C ABI.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bridges.h"
#include "batched.h"

struct bridges_ctx {
  int device = 0;
  size_t budget = 0;  // 0: unlimited
  bool user_ws = false;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // device staging for bridges_find_host
  int32_t* stage = nullptr;
  size_t stage_bytes = 0;
  int64_t* h_pinned = nullptr;  // pinned host scratch (counts)
  bridges_opts opts{};
  int num_sms = 0;
  size_t smem_optin = 0;
  int64_t launches = 0;
  int64_t allocs = 0;  // device allocations of the context's own buffers since its options were set
  // profiling: a ring of kRing event sets, one per call; slot = call index % kRing
  static constexpr int kRing = 32;
  cudaEvent_t ev[kRing][8]{};
  bool events = false;
  int64_t calls = 0;         // profiled calls issued
  int64_t resolved = 0;      // calls whose times have been read back
  float stage_ms[kRing][6]{};
  int64_t last_cfg[8]{};  // [5], [6]: block pass prefix edges (-1: no snapshot) and blocks; [7] fused
  // profiling of the articulation-point block pass, a ring like the above; per call the events
  // are start, after warm-up, after snapshot, after stream, end
  cudaEvent_t ap_ev[kRing][5]{};
  int64_t ap_calls = 0;
  int64_t ap_resolved = 0;
  float ap_ms[kRing][5]{};
  // batched path: device descriptors; two pinned staging copies used in turn, each with the CUDA
  // graph that uploads from it and the event of the last batch that read it
  void* bws = nullptr;          // device: BatchArgs | ntasks | tasks[cap] | corder[cap] | queue | gerr[gcap] | slots
  size_t bws_bytes = 0;
  void* bstage[2]{};             // pinned: BatchArgs | ntasks | tasks[cap] | corder[cap]
  size_t bstage_bytes = 0;
  int64_t b_task_cap = 0, b_graph_cap = 0, b_slot_cap = 0;
  std::vector<int32_t> b_order;  // the last batch's certification order (host scratch)
  cudaGraphExec_t b_exec[2]{};
  cudaEvent_t b_done_ev[2]{};
  int b_next = 0;                // the staging copy the next batch fills
  int64_t b_split_edges = 0;     // partition graphs with more edges than this (0: automatic)
  int64_t b_back_edges = 16384;  // certification: tasks of at most this many edges may be taken from the back
  bridges_batch_plan bplan{};    // per-bucket plan of the batched form (n = 0: automatic)
  // pipelined host input: a copy stream and one event per chunk copied
  static constexpr int kMaxChunks = 64;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t entry_ev = nullptr;
  cudaEvent_t chunk_ev[kMaxChunks]{};
};

namespace bridges {

// Applies the context's batched plan to whole-graph tasks: splits graphs with many edges into
// partitions (certificate slots filled in), picks each task's group and warm-up prefix, and
// orders the tasks by group, largest first; returns the slot words needed.  total_e: the edges
// of every graph of the batch (the automatic split depends on it).
int64_t plan_batch_tasks(const bridges_ctx* c, std::vector<BatchTask>& graphs, int64_t total_e,
                         std::vector<BatchTask>& tasks);
// One persistent launch over `tasks` (G graphs) on stream s, through the context's CUDA graph.
int64_t launch_batch_tasks(bridges_ctx* c, cudaStream_t s, const std::vector<BatchTask>& tasks, int32_t G,
                           int64_t slot_words);
// Edge count above which a batched graph is partitioned.
int64_t default_split(const bridges_ctx* c, int64_t total_e);
// The single-graph path, count copied to count_dev (device); enqueue only.
int64_t run_single(bridges_ctx* c, cudaStream_t s, const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t M,
                   int32_t* out, int64_t* count_dev);
// Workspace bytes of the single-graph path for (E, V) with automatic M.
size_t single_workspace_bytes(const bridges_ctx* c, int64_t E, int32_t V);

}  // namespace bridges
