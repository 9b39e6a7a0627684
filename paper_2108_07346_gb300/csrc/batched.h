// batched.h -- device-side descriptors of the batched (many small graphs) kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bridges {

constexpr int kBatchVmax = 4096;  // graphs up to this many vertices are handled in shared memory
// ... up to this many, two per block: the largest size whose bridge-stage layout fits twice in a
// block's shared memory (2 x 115,200 bytes)
constexpr int kBatchHalfVmax = 3008;
constexpr int kBatchQuarterVmax = kBatchVmax / 4;  // ... up to this many, by a certification group

// One unit of work: a whole graph (nparts == 1) or partition `part` of it.
struct BatchTask {
  const int32_t* u;  // the graph's edge arrays
  const int32_t* v;
  int64_t lo, hi;    // edge range of this task in u / v
  int32_t* out;      // the graph's output pairs
  int64_t* count;    // the graph's count (or negative status)
  int64_t slot;      // u32 offset of this task's certificate slot (batch_slot_words(V); a graph's are consecutive)
  int32_t g;         // graph index within the launch (its gerr word)
  int32_t part;      // partition index within the graph
  int32_t nparts;    // partitions of the graph
  int32_t V;         // vertices of the graph
  int32_t cls;       // group that runs its bridge stage: 0 a whole block, 1 a half block, 2 the
                     // quarter-block group that certified it (in certify_kernel)
  int32_t pad;
  int64_t warm;      // edges certified one by one before the union-finds are flattened
};

// Everything the kernel reads, in device memory so a captured CUDA graph stays valid when the
// caller's pointers change between calls.
struct BatchArgs {
  const BatchTask* tasks;
  const int32_t* corder;  // certification order: task indices, most edges first
  const int32_t* d_ntasks;
  int32_t* queue;    // next task (atomic): [0..1] bridge stages by group size; words [4, 5] the
                     // certification claims (front count low, back count high, one 64-bit word)
  int32_t* gerr;     // per graph: first error of any partition
  uint32_t* slots;   // the tasks' certificates
  int32_t G;           // graphs (bounds the graph index of every task)
  int32_t nbig;        // bridge stages: tasks [0, nbig) run on whole blocks,
  int32_t nmid;        // [nbig, nbig + nmid) on half-block groups; the rest were finished by certify_kernel
  int32_t nback;       // certification: the last nback tasks of corder may be claimed from the back
  int32_t pad;
  int64_t slot_words;  // capacity of slots (u32)
};

// The smallest group a task fits: 0 a whole block (more than kBatchHalfVmax vertices, or a
// partition of a graph: partitions merge from the slots), 1 a half block, 2 the certification
// group (a quarter block).
inline int batch_min_class(int32_t V, int32_t nparts) {
  if (V > kBatchHalfVmax || nparts > 1) return 0;
  return V > kBatchQuarterVmax ? 1 : 2;
}

// The group a planned task runs on (its cls, which the plan may set to a larger group than the
// smallest it fits; never a smaller one).
inline int batch_task_class(const BatchTask& t) { return t.cls; }

// Words of a task's certificate slot: [nF, nF', F (V words), F' (V words), the root of each
// vertex's F tree (V u16, padded to a word), the root of each vertex's F' tree (likewise)]; the
// roots are written by a graph's first task (the F' roots only when more tasks follow).  A
// graph's slots are consecutive.
__host__ __device__ inline int64_t batch_slot_words(int32_t V) { return 2 + 2 * (int64_t)V + 2 * (((int64_t)V + 1) / 2); }

// One graph's final stage on one block (small_final_launch): the final certificate as the forest
// pass and the merge tree leave it in global memory, for a graph of 2..kBatchVmax vertices.
struct SmallFinalArgs {
  int32_t V;
  const int32_t* P;     // F's union-find (P[x] <= x; a root is its set's minimum vertex)
  const int32_t* tu;    // F: tree edges, *d_nt of them
  const int32_t* tv;
  const int32_t* d_nt;
  const int32_t* xu;    // F': the other certificate edges, *d_nx of them
  const int32_t* xv;
  const int32_t* d_nx;
  const int32_t* status;  // the call's status word (0, or the first error of an earlier stage)
  int64_t* count;       // receives the bridge count, or the status when it is set
  int32_t* out;         // receives the sorted (a, b) pairs, capacity 2 (V - 1)
};

size_t batched_smem_bytes();
// Launches the one-block final stage (bridges and count only) on stream s.
bool small_final_launch(cudaStream_t s, const SmallFinalArgs& a);
// Launches the two persistent kernels (one block per SM each: certification, then the bridge
// stages) reading their arguments from *dev_args.
bool batched_launch(cudaStream_t s, const BatchArgs* dev_args, int num_sms);

}  // namespace bridges
