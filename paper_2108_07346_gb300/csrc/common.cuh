// common.cuh -- device helpers shared by the kernels of libbridges (union-find, status word,
// warp compaction).  Nothing here is visible through the C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace bridges {

constexpr unsigned kFull = 0xffffffffu;

// First error wins; later errors leave the status unchanged.
__device__ __forceinline__ void set_status(int32_t* status, int32_t code) { atomicCAS(status, 0, code); }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Relaxed, device-scope accesses to union-find parents that other blocks update concurrently.
__device__ __forceinline__ int32_t ld_relaxed(const int32_t* p) {
  int32_t v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(int32_t* p, int32_t v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Read-only streaming loads of the edge list (never written during a call).
__device__ __forceinline__ int4 ld_stream4(const int4* p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_stream1(const int32_t* p) { return __ldcs(p); }

// ---------------------------------------------------------------------------------------------
// Concurrent union-find on a parent array P[0..V) in global memory (Alg. 2's union-find,
// Sec. 4.B, made concurrent as Sec. 7 suggests).
//
// Invariant: P[x] <= x for every x, i.e. a root is hooked only under a SMALLER root.  Hence the
// parent graph is acyclic whatever the interleaving, the root of a set is its minimum vertex,
// and a successful CAS P[a]: a -> b (a > b both roots when read) always joins two different
// sets: if b were already in a's set its chain would lead to a, yet chains only descend.
// Each successful link therefore adds one forest edge, so a forest gets at most V-1 links and
// every CAS failure means another thread's link succeeded: the loops below terminate.
// Path halving writes only ancestors into non-roots, which is safe under races.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int32_t uf_find(int32_t* P, int32_t x) {
  while (true) {
    int32_t p = ld_relaxed(P + x);
    if (p == x) return x;
    int32_t g = ld_relaxed(P + p);
    if (g == p) return p;
    st_relaxed(P + x, g);
    x = g;
  }
}

// Root of x when no link can happen concurrently (snapshots, the final stage): roots are then
// immutable, so their entries may come from L1 (ld.ca) and the many readers of one giant root
// are served by each SM's L1 instead of queueing on one L2 slice.  Non-root entries read stale
// are still ancestors, so the walk still ends at the root; halving uses plain stores.
__device__ __forceinline__ int32_t uf_find_static(int32_t* P, int32_t x) {
  int32_t p = __ldca(P + x);
  while (p != x) {
    const int32_t g = __ldca(P + p);
    if (g == p) return p;
    P[x] = g;
    x = g;
    p = __ldca(P + x);
  }
  return x;
}

// Joins the sets of a and b.  Returns true iff they were different (the edge is a forest edge).
//
// Walks up from both ends comparing PARENTS, not roots: equal parents prove a common set, so in
// the dense phase, where nearly every vertex points straight at its root, a rejection costs two
// loads and never touches the root's own entry (which every block would otherwise hammer).  The
// end with the larger parent moves up (path halving); a grandparent equal to the other end's
// parent also proves a common set.  When the end with the larger parent is a root x (or its
// parent px is one), it is hooked under the other end's parent py < x: members of a set are >=
// its root, so py is not in x's set and the CAS joins two different sets.  Hooking under py
// rather than under py's root spares the walk to that root, whose entry every vertex joining
// the giant component would otherwise read -- one L2 line for all blocks while the forests grow
// (large workload, 150 k-edge prefix: 0.136 ms with root-under-root hooking, 0.090 ms so).
__device__ __forceinline__ bool uf_link(int32_t* P, int32_t a, int32_t b) {
  int32_t x = a, y = b;
  while (true) {
    int32_t px = ld_relaxed(P + x), py = ld_relaxed(P + y);
    if (px == py) return false;
    if (px < py) {
      int32_t t = x;
      x = y;
      y = t;
      t = px;
      px = py;
      py = t;
    }
    // now px > py
    if (px == x) {
      if (atomicCAS(P + x, x, py) == x) return true;  // py < x lies in y's set
      continue;  // x was hooked meanwhile: re-read its parent
    }
    const int32_t g = ld_relaxed(P + px);
    if (g == py) {  // x's grandparent is y's parent: one set (halve x's path on the way out)
      st_relaxed(P + x, g);
      return false;
    }
    if (g == px) {              // px is a root: hook it without reading its entry again
      if (atomicCAS(P + px, px, py) == px) return true;
      continue;
    }
    st_relaxed(P + x, g);  // path halving
    x = g;
  }
}

// Bounded poll: calls done() until it returns true or max_polls polls have been made (sleeping
// ~100 ns between polls).  Returns whether done() became true.  Every device-side wait of the
// library goes through this, so no wait can hang a kernel.
template <class Done>
__device__ __forceinline__ bool bounded_poll(Done done, unsigned long long max_polls) {
  for (unsigned long long i = 0; i < max_polls; i++) {
    if (done()) return true;
    if (i >= 32) __nanosleep(100);
  }
  return done();
}

__device__ __forceinline__ int32_t ld_acquire_s32(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Warp-aggregated append of (a, b) to a list with a shared counter: one atomic per warp.
// Every lane of the warp must call it (pred may be false).
__device__ __forceinline__ void warp_append(bool pred, int32_t a, int32_t b, int32_t* cnt, int32_t* ou,
                                            int32_t* ov, int32_t cap, int32_t* status) {
  unsigned m = __ballot_sync(kFull, pred);
  if (!m) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(m) - 1;
  int32_t base = 0;
  if (lane == leader) base = atomicAdd(cnt, __popc(m));
  base = __shfl_sync(kFull, base, leader);
  if (pred) {
    int32_t i = base + __popc(m & lanemask_lt());
    if (i < cap) {
      ou[i] = a;
      ov[i] = b;
    } else {
      set_status(status, BRIDGES_EINTERNAL_CODE);
    }
  }
}

}  // namespace bridges
