// batched.h -- device-side descriptors of the batched (many small graphs) kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bridges {

constexpr int kBatchVmax = 4096;  // graphs up to this many vertices are handled in shared memory
constexpr int kBatchHalfVmax = kBatchVmax / 2;     // ... up to this many, two per block
constexpr int kBatchQuarterVmax = kBatchVmax / 4;  // ... up to this many, four per block

// One unit of work: a whole graph (nparts == 1) or partition `part` of it.
struct BatchTask {
  const int32_t* u;  // the graph's edge arrays
  const int32_t* v;
  int64_t lo, hi;    // edge range of this task in u / v
  int32_t* out;      // the graph's output pairs
  int64_t* count;    // the graph's count (or negative status)
  int64_t slot;      // u32 offset of this partition's certificate slot (nparts > 1)
  int32_t g;         // graph index within the launch (done / gerr counters)
  int32_t part;      // partition index within the graph
  int32_t nparts;    // partitions of the graph
  int32_t V;         // vertices of the graph
};

// Everything the kernel reads, in device memory so a captured CUDA graph stays valid when the
// caller's pointers change between calls.
struct BatchArgs {
  const BatchTask* tasks;
  const int32_t* d_ntasks;
  int32_t* queue;    // next task (atomic)
  int32_t* done;     // per graph: partitions finished
  int32_t* gerr;     // per graph: first error of any partition
  uint32_t* slots;   // certificates of partitions
  int32_t G;           // graphs (bounds the graph index of every task)
  int32_t nbig;        // tasks [0, nbig) run on whole blocks,
  int32_t nmid;        // [nbig, nbig + nmid) on half-block groups, the rest on quarter-block groups
  int64_t slot_words;  // capacity of slots (u32)
};

// Which group a task needs: 0 a whole block (more than kBatchHalfVmax vertices, or a partition of
// a graph: partitions merge through the slots), 1 a half block, 2 a quarter block.
inline int batch_task_class(const BatchTask& t) {
  if (t.V > kBatchHalfVmax || t.nparts > 1) return 0;
  return t.V > kBatchQuarterVmax ? 1 : 2;
}

size_t batched_smem_bytes();
// Launches the persistent kernel (one block per SM) reading its arguments from *dev_args.
bool batched_launch(cudaStream_t s, const BatchArgs* dev_args, int num_sms);

}  // namespace bridges
