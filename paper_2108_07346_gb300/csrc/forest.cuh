// forest.cuh -- one certificate job's two union-finds (Alg. 2's F and F') as the streaming
// kernels see them: the forest pass of certify.cu and the fused pass of blocks.cu offer edges
// through the same code.  Nothing here is visible through the C ABI.
#pragma once

#include "common.cuh"

namespace bridges {

// Job j's slices of the certificate buffers: UF1 (F) and UF2 (F') parents and the two edge lists.
struct Job {
  int32_t* P1;
  int32_t* P2;
  int32_t* f1u;
  int32_t* f1v;
  int32_t* f2u;
  int32_t* f2v;
  int32_t* cnt;  // [2]
};

__device__ __forceinline__ Job job_of(const CertBufs& b, int32_t V, int64_t j) {
  Job J;
  int64_t o = j * (int64_t)V;
  J.P1 = b.P1 + o;
  J.P2 = b.P2 + o;
  J.f1u = b.f1u + o;
  J.f1v = b.f1v + o;
  J.f2u = b.f2u + o;
  J.f2v = b.f2v + o;
  J.cnt = b.cnt + 2 * j;
  return J;
}

// Offers edge (a, b) to F then F'.  Returns 0 (dropped), 1 (joined F) or 2 (joined F').
__device__ __forceinline__ int offer(const Job& J, int32_t a, int32_t b) {
  if (uf_link(J.P1, a, b)) return 1;
  if (uf_link(J.P2, a, b)) return 2;
  return 0;
}

}  // namespace bridges
