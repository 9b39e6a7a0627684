// batched.cu -- many small graphs in one persistent launch.
//
// Each block repeatedly takes a task from an atomic queue.  A task is a whole graph (V <= 4096)
// or one partition of a large one (Sec. 3: the edge list split into contiguous sets).  The block
// certifies the task's edges with two concurrent union-finds in SHARED memory (Alg. 2: F, then F'
// from the edges F rejects), so a graph never touches global memory except to read its edges.
// A single-task graph then runs the whole bridge stage in shared memory; a partitioned graph
// writes its certificate to a global slot, and the block that finishes the graph's LAST
// partition merges all of them (Sec. 3 merge, fan-in = number of partitions) and runs the
// bridge stage.  Nothing waits on another block, so there is no spin anywhere.
//
// The bridge stage is the same Euler-tour / preorder-range test as final.cu, on 16-bit arrays
// with __syncthreads between phases (list ranking four hops per round), then a rank sort of the
// packed (a << 12 | b) keys (bitonic above 1,024 bridges).  A graph's fixed cost is its block
// barriers, so the stage keeps their number low.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/bridges.h"
#include "batched.h"
#include "common.cuh"

namespace bridges {

namespace {

constexpr int kT = 1024;          // threads per block
constexpr int kW = kT / 32;
constexpr int kVmax = kBatchVmax;  // 4096
constexpr int kAmax = 2 * kVmax;  // arcs
constexpr uint16_t kNone16 = 0xffff;

// shared-memory regions (bytes), each a multiple of 16
constexpr int kR0 = 16448;  // P1 (int32[V]); later aoff (u16[V+1]) + vbase (u16[V+1])
constexpr int kR1 = 16448;  // P2 (int32[V]); later root (u16[V]) + cur (u16[V])
constexpr int kR2 = 16384;  // F list (u32[V]); later bridge keys (u32[V])
constexpr int kR3 = 16384;  // F' list (u32[V])
constexpr int kR4 = 8208;   // off (u16[V+1])
constexpr int kR5 = 16384;  // dst (u16[2V]); later lo (int32[V])
constexpr int kR6 = 16384;  // twin (u16[2V]); later hi (int32[V])
constexpr int kR7 = 16400;  // succ (u16[2V]); later dflag / dscan (u16[2V+1])
constexpr int kR8 = 16384;  // rnk (u16[2V])
constexpr int kR9 = 24576;  // pre, sz, par (u16[V] each)
constexpr int kSmem = kR0 + kR1 + kR2 + kR3 + kR4 + kR5 + kR6 + kR7 + kR8 + kR9;

struct Smem {
  int32_t* P1;
  int32_t* P2;
  uint32_t* F1;
  uint32_t* F2;
  uint16_t* aoff;
  uint16_t* vbase;
  uint16_t* root;
  uint16_t* cur;
  uint32_t* keys;
  uint16_t* off;
  uint16_t* dst;
  uint16_t* twin;
  int32_t* lo;
  int32_t* hi;
  uint16_t* succ;
  uint16_t* dflag;
  uint16_t* rnk;
  uint16_t* pre;
  uint16_t* sz;
  uint16_t* par;
};

__device__ Smem carve_smem(char* base) {
  Smem s;
  char* c = base;
  s.P1 = reinterpret_cast<int32_t*>(c);
  s.aoff = reinterpret_cast<uint16_t*>(c);
  s.vbase = reinterpret_cast<uint16_t*>(c + 8224);
  c += kR0;
  s.P2 = reinterpret_cast<int32_t*>(c);
  s.root = reinterpret_cast<uint16_t*>(c);
  s.cur = reinterpret_cast<uint16_t*>(c + 8224);
  c += kR1;
  s.F1 = reinterpret_cast<uint32_t*>(c);
  s.keys = s.F1;
  c += kR2;
  s.F2 = reinterpret_cast<uint32_t*>(c);
  c += kR3;
  s.off = reinterpret_cast<uint16_t*>(c);
  c += kR4;
  s.dst = reinterpret_cast<uint16_t*>(c);
  s.lo = reinterpret_cast<int32_t*>(c);
  c += kR5;
  s.twin = reinterpret_cast<uint16_t*>(c);
  s.hi = reinterpret_cast<int32_t*>(c);
  c += kR6;
  s.succ = reinterpret_cast<uint16_t*>(c);
  s.dflag = s.succ;
  c += kR7;
  s.rnk = reinterpret_cast<uint16_t*>(c);
  c += kR8;
  s.pre = reinterpret_cast<uint16_t*>(c);
  s.sz = s.pre + kVmax;
  s.par = s.sz + kVmax;
  return s;
}

// 16-bit counters packed two to a 32-bit word (shared-memory atomics are 32-bit).
__device__ __forceinline__ uint16_t inc16(uint16_t* a, int i) {
  uint32_t* w = reinterpret_cast<uint32_t*>(a + (i & ~1));
  const int sh = 16 * (i & 1);
  return (uint16_t)(atomicAdd(w, 1u << sh) >> sh);
}

// Concurrent union-find in shared memory: the algorithm of uf_link (common.cuh) -- parents are
// compared first, a root is hooked under a smaller vertex, P[x] <= x always.
__device__ __forceinline__ bool s_link(int32_t* P, int32_t a, int32_t b) {
  volatile int32_t* VP = P;
  int32_t x = a, y = b;
  while (true) {
    int32_t px = VP[x], py = VP[y];
    if (px == py) return false;
    if (px < py) {
      int32_t t = x;
      x = y;
      y = t;
      t = px;
      px = py;
      py = t;
    }
    if (px == x) {
      int32_t r = py, q = VP[r];  // hook under the other side's root (shallow trees)
      while (q != r) {
        r = q;
        q = VP[r];
      }
      if (atomicCAS(P + x, x, r) == x) return true;
      continue;
    }
    const int32_t g = VP[px];
    if (g != px) VP[x] = g;
    x = g;
  }
}

// Block-wide exclusive scan of n (<= 2*kT*... ) u16 values in place; returns the total.
__device__ int32_t block_scan16(uint16_t* a, int32_t n, int32_t* red) {
  const int per = (n + kT - 1) / kT;  // contiguous items per thread
  const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
  int32_t s = 0;
  for (int i = lo; i < hi; i++) s += a[i];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) red[w] = incl;
  __syncthreads();
  int32_t base = 0, tot = 0;
  for (int k = 0; k < kW; k++) {
    if (k < w) base += red[k];
    tot += red[k];
  }
  int32_t run = base + incl - s;
  for (int i = lo; i < hi; i++) {
    const int32_t v = a[i];
    a[i] = (uint16_t)run;
    run += v;
  }
  __syncthreads();
  return tot;
}

// The same for two arrays of equal length at once (one pair of block barriers for both).
__device__ void block_scan16_pair(uint16_t* a, uint16_t* b, int32_t n, int32_t* red) {
  __shared__ int32_t red_b[kW];
  const int per = (n + kT - 1) / kT;
  const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
  int32_t sa = 0, sb = 0;
  for (int i = lo; i < hi; i++) {
    sa += a[i];
    sb += b[i];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t ia = sa, ib = sb;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t ya = __shfl_up_sync(kFull, ia, o), yb = __shfl_up_sync(kFull, ib, o);
    if (lane >= o) {
      ia += ya;
      ib += yb;
    }
  }
  if (lane == 31) {
    red[w] = ia;
    red_b[w] = ib;
  }
  __syncthreads();
  int32_t ba = 0, bb = 0;
  for (int k = 0; k < w; k++) {
    ba += red[k];
    bb += red_b[k];
  }
  int32_t ra = ba + ia - sa, rb = bb + ib - sb;
  for (int i = lo; i < hi; i++) {
    const int32_t va = a[i], vb = b[i];
    a[i] = (uint16_t)ra;
    b[i] = (uint16_t)rb;
    ra += va;
    rb += vb;
  }
  __syncthreads();
}

// Offers edge (a, b) to F, then F'; appends winners (warp-aggregated).  Every lane calls it.
__device__ __forceinline__ void s_settle(const Smem& S, bool need, int32_t a, int32_t b, int32_t* n1, int32_t* n2,
                                         int32_t V) {
  if (!__any_sync(kFull, need)) return;
  int r = 0;
  if (need) r = s_link(S.P1, a, b) ? 1 : (s_link(S.P2, a, b) ? 2 : 0);
  const unsigned m1 = __ballot_sync(kFull, r == 1), m2 = __ballot_sync(kFull, r == 2);
  const int lane = threadIdx.x & 31;
  int32_t b1 = 0, b2 = 0;
  if (m1 && lane == __ffs(m1) - 1) b1 = atomicAdd(n1, __popc(m1));
  if (m2 && lane == __ffs(m2) - 1) b2 = atomicAdd(n2, __popc(m2));
  if (m1) b1 = __shfl_sync(kFull, b1, __ffs(m1) - 1);
  if (m2) b2 = __shfl_sync(kFull, b2, __ffs(m2) - 1);
  const uint32_t packed = (uint32_t)a | ((uint32_t)b << 16);
  if (r == 1) {
    const int32_t i = b1 + __popc(m1 & lanemask_lt());
    if (i < V) S.F1[i] = packed;
  } else if (r == 2) {
    const int32_t i = b2 + __popc(m2 & lanemask_lt());
    if (i < V) S.F2[i] = packed;
  }
}

// Points every vertex straight at its root (no link runs meanwhile), so that afterwards "equal
// parents" recognises every pair that shares a set.
__device__ __forceinline__ void s_flatten(int32_t* P, int32_t V) {
  __syncthreads();
  for (int x = threadIdx.x; x < V; x += kT) {
    int32_t r = x, p = P[x];
    while (p != r) {
      r = p;
      p = P[r];
    }
    P[x] = r;
  }
  __syncthreads();
}

// Scalar certification of edges [lo, hi): every lane takes one edge per step.
__device__ void s_certify_scalar(const Smem& S, const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                 int64_t lo, int64_t hi, int32_t V, int32_t* n1, int32_t* n2, int32_t* err) {
  volatile int32_t* P2 = S.P2;
  for (int64_t t0 = lo; t0 < hi; t0 += kT) {
    const int64_t i = t0 + threadIdx.x;
    const bool valid = i < hi;
    const int32_t a = valid ? __ldcs(u + i) : 0, b = valid ? __ldcs(v + i) : 0;
    bool need = valid;
    if (need && ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V)) {
      *err = BRIDGES_ERANGE;
      need = false;
    }
    if (need && (a == b || P2[a] == P2[b])) need = false;
    s_settle(S, need, a, b, n1, n2, V);
  }
}

// The lanes' flagged edges of one tile go through the union-finds (bit 4k+c of m: element
// 4*(base + k*kT + tid) + c of ub / vb).  Out of line: rare after the flatten.
__device__ __noinline__ void s_offer_misses(const Smem& S, uint32_t m, const int32_t* __restrict__ ub,
                                            const int32_t* __restrict__ vb, int64_t base, int32_t V, int32_t* n1,
                                            int32_t* n2, int32_t* err) {
  while (__any_sync(kFull, m != 0)) {
    int32_t a = 0, b = 0;
    bool go = false;
    if (m) {
      const int bit = __ffs(m) - 1;
      m &= m - 1;
      const int64_t e = 4 * (base + (int64_t)(bit >> 2) * kT + threadIdx.x) + (bit & 3);
      a = ub[e];
      b = vb[e];
      if ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V)
        *err = BRIDGES_ERANGE;
      else
        go = a != b;
    }
    s_settle(S, go, a, b, n1, n2, V);
  }
}

// Certifies edges [lo, hi) of (u, v) with 16-byte loads when u and v share their alignment (a
// scalar head and tail otherwise), four units of four edges per thread in flight, a per-thread
// miss mask (the ends' F' parents differ, or an id is out of range) and one warp vote per tile.
__device__ __forceinline__ void s_certify_vec(const Smem& S, const int32_t* __restrict__ u, const int32_t* __restrict__ v, int64_t lo,
                              int64_t hi, int32_t V, int32_t* n1, int32_t* n2, int32_t* err) {
  constexpr int U = 4;
  if (lo >= hi) return;
  const bool same = ((reinterpret_cast<uintptr_t>(u) ^ reinterpret_cast<uintptr_t>(v)) & 15) == 0;
  int64_t body = lo;
  if (same) {
    while (body < hi && (reinterpret_cast<uintptr_t>(u + body) & 15)) body++;
  } else {
    body = hi;
  }
  s_certify_scalar(S, u, v, lo, body, V, n1, n2, err);
  const int64_t nunits = (hi - body) >> 2;
  const int32_t* ub = u + body;
  const int32_t* vb = v + body;
  const int4* u4 = reinterpret_cast<const int4*>(ub);
  const int4* v4 = reinterpret_cast<const int4*>(vb);
  volatile int32_t* P2 = S.P2;
  const uint32_t cl = (uint32_t)(kVmax - 1);
  for (int64_t base = 0; base < nunits; base += (int64_t)kT * U) {
    int4 ua[U], va[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      const int64_t idx = base + (int64_t)k * kT + threadIdx.x;
      if (idx < nunits) {
        ua[k] = __ldcs(u4 + idx);
        va[k] = __ldcs(v4 + idx);
      } else {
        ua[k] = make_int4(0, 0, 0, 0);
        va[k] = make_int4(0, 0, 0, 0);
      }
    }
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < U; k++) {
      if (base + (int64_t)k * kT + threadIdx.x >= nunits) continue;
      const int32_t as[4] = {ua[k].x, ua[k].y, ua[k].z, ua[k].w};
      const int32_t bs[4] = {va[k].x, va[k].y, va[k].z, va[k].w};
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const uint32_t a = (uint32_t)as[c], b = (uint32_t)bs[c];
        const bool bad = a >= (uint32_t)V || b >= (uint32_t)V;
        const bool same_set = P2[min(a, cl)] == P2[min(b, cl)];
        m |= (uint32_t)(bad || !same_set) << (4 * k + c);
      }
    }
    if (__any_sync(kFull, m != 0)) s_offer_misses(S, m, ub, vb, base, V, n1, n2, err);
  }
  s_certify_scalar(S, u, v, body + 4 * nunits, hi, V, n1, n2, err);
}

// Certifies edges [lo, hi) of (u, v) into S.F1 / S.F2 (appending to *n1 / *n2); ids outside
// [0, V) set *err.  A warm-up prefix goes edge by edge (most of its edges still link; a vector
// tile's miss loop would run as long as its busiest lane), then both union-finds are flattened,
// so that "equal F' parents" afterwards recognises nearly every pair inside one F' component,
// and the rest streams through the vector loop.
__device__ void s_certify_range(const Smem& S, const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                int64_t lo, int64_t hi, int32_t V, int32_t* n1, int32_t* n2, int32_t* err) {
  const int64_t warm = min(hi - lo, (int64_t)8 * V + 2048);
  s_certify_scalar(S, u, v, lo, lo + warm, V, n1, n2, err);
  lo += warm;
  if (lo >= hi) return;
  s_flatten(S.P1, V);
  s_flatten(S.P2, V);
  s_certify_vec(S, u, v, lo, hi, V, n1, n2, err);
}

// Certifies packed edges (a | b << 16) of a global list.
__device__ void s_certify_packed(const Smem& S, const uint32_t* e, int32_t n, int32_t V, int32_t* n1, int32_t* n2) {
  volatile int32_t* P2 = S.P2;
  for (int32_t t0 = 0; t0 < n; t0 += kT) {
    const int32_t i = t0 + threadIdx.x;
    const bool valid = i < n;
    const uint32_t x = valid ? __ldcg(e + i) : 0;
    const int32_t a = (int32_t)(x & 0xffff), b = (int32_t)(x >> 16);
    const bool need = valid && a != b && P2[a] != P2[b];
    s_settle(S, need, a, b, n1, n2, V);
  }
}

// Bridges of the certificate in S (F1 = tree, F2 = extra), written sorted to out; returns count.
__device__ int32_t s_bridges(const Smem& S, int32_t V, int32_t nt, int32_t nx, int32_t* out, int32_t* red,
                             int32_t* sh) {
  const int tid = threadIdx.x;
  // roots (minimum vertex of each tree), degrees
  for (int x = tid; x < V; x += kT) {
    int32_t r = x, p = S.P1[x];
    while (p != r) {
      r = p;
      p = S.P1[r];
    }
    S.root[x] = (uint16_t)r;  // P2 region: F' union-find no longer needed
  }
  for (int x = tid; x <= V + 1; x += kT) S.off[x] = 0;
  for (int x = tid; x < V + 2; x += kT) S.cur[x] = 0;
  __syncthreads();
  for (int e = tid; e < nt; e += kT) {
    const uint32_t p = S.F1[e];
    inc16(S.off, (int)(p & 0xffff));
    inc16(S.off, (int)(p >> 16));
  }
  __syncthreads();
  const int32_t narcs = block_scan16(S.off, V + 1, red);  // off[V] = narcs
  for (int e = tid; e < nt; e += kT) {
    const uint32_t p = S.F1[e];
    const int32_t a = (int32_t)(p & 0xffff), b = (int32_t)(p >> 16);
    const int32_t ia = S.off[a] + inc16(S.cur, a), ib = S.off[b] + inc16(S.cur, b);
    S.dst[ia] = (uint16_t)b;
    S.dst[ib] = (uint16_t)a;
    S.twin[ia] = (uint16_t)ib;
    S.twin[ib] = (uint16_t)ia;
  }
  __syncthreads();
  // Euler-tour successors, cut at each root
  for (int i = tid; i < narcs; i += kT) {
    const int32_t y = S.dst[i], t = S.twin[i];
    uint16_t s;
    if (t + 1 < S.off[y + 1])
      s = (uint16_t)(t + 1);
    else
      s = S.root[y] == y ? kNone16 : S.off[y];
    S.succ[i] = s;
    S.rnk[i] = s == kNone16 ? 0 : 1;
  }
  __syncthreads();
  // list ranking by pointer jumping, four hops per round (shared-memory loads are cheap, the
  // block barriers between rounds are not): ceil(log4 n) rounds, double-buffered in the P1 and F
  // regions (both free now: the roots are known and the adjacency is built)
  {
    int rounds = 0;
    while ((1 << (2 * rounds)) < max(narcs, 1)) rounds++;
    uint16_t* sa = S.succ;
    uint16_t* ra = S.rnk;
    uint16_t* sb = reinterpret_cast<uint16_t*>(S.P1);
    uint16_t* rb = reinterpret_cast<uint16_t*>(S.F1);
    for (int r = 0; r < rounds; r++) {
      for (int i = tid; i < narcs; i += kT) {
        uint16_t s = sa[i], acc = ra[i];
#pragma unroll
        for (int h = 0; h < 3 && s != kNone16; h++) {
          acc = (uint16_t)(acc + ra[s]);
          s = sa[s];
        }
        rb[i] = acc;
        sb[i] = s;
      }
      __syncthreads();
      uint16_t* t = sa;
      sa = sb;
      sb = t;
      t = ra;
      ra = rb;
      rb = t;
    }
    if (ra != S.rnk) {
      for (int i = tid; i < narcs; i += kT) S.rnk[i] = ra[i];
      __syncthreads();
    }
  }
  // per root: tour arcs (aoff) and tree vertices (vbase); P1 region is free now
  for (int x = tid; x <= V; x += kT) {
    uint16_t L = 0, nv = 0;
    if (x < V && S.root[x] == x) {
      L = S.off[x + 1] > S.off[x] ? (uint16_t)(S.rnk[S.off[x]] + 1) : 0;
      nv = (uint16_t)(L / 2 + 1);
    }
    S.aoff[x] = L;
    S.vbase[x] = nv;
  }
  __syncthreads();
  block_scan16_pair(S.aoff, S.vbase, V + 1, red);
  // tour positions; down arcs (dflag reuses succ, free after ranking)
  for (int i = tid; i <= narcs; i += kT) S.dflag[i] = 0;
  __syncthreads();
  for (int i = tid; i < narcs; i += kT) {
    const int32_t x = S.dst[S.twin[i]];
    const int32_t r = S.root[x];
    const int32_t L = S.rnk[S.off[r]] + 1;
    const int32_t ri = S.rnk[i], rt = S.rnk[S.twin[i]];
    const int32_t g = S.aoff[r] + L - 1 - ri;
    if (g < 0 || g >= narcs) continue;
    if (ri > rt) {
      const int32_t y = S.dst[i];
      S.dflag[g] = 1;
      S.par[y] = (uint16_t)x;
      S.pre[y] = (uint16_t)g;
      S.sz[y] = (uint16_t)((ri - rt + 1) / 2);
    }
  }
  __syncthreads();
  block_scan16(S.dflag, narcs, red);  // dscan in place
  // preorder numbers; lo / hi (dst and twin are free now)
  for (int x = tid; x < V; x += kT) {
    const int32_t r = S.root[x];
    int32_t p;
    if (r == x) {
      p = S.vbase[x];
      S.sz[x] = (uint16_t)((S.aoff[x + 1] - S.aoff[x]) / 2 + 1);
      S.par[x] = kNone16;
    } else {
      const int32_t g = S.pre[x], a0 = S.aoff[r];
      p = (g < narcs && a0 < narcs) ? S.vbase[r] + 1 + S.dflag[g] - S.dflag[a0] : 0;
    }
    S.pre[x] = (uint16_t)min(max(p, 0), V - 1);
  }
  __syncthreads();
  for (int x = tid; x < V; x += kT) {
    S.lo[S.pre[x]] = S.pre[x];
    S.hi[S.pre[x]] = S.pre[x];
  }
  __syncthreads();
  for (int e = tid; e < nx; e += kT) {
    const uint32_t p = S.F2[e];
    const int32_t a = (int32_t)(p & 0xffff), b = (int32_t)(p >> 16);
    if (a == b) continue;
    const int32_t pa = S.pre[a], pb = S.pre[b];
    atomicMin(S.lo + pa, pb);
    atomicMin(S.lo + pb, pa);
    atomicMax(S.hi + pa, pb);
    atomicMax(S.hi + pb, pa);
  }
  __syncthreads();
  // chunk (32) minima / maxima kept in the off region, free now
  int32_t* cmin = reinterpret_cast<int32_t*>(S.off);
  int32_t* cmax = cmin + kVmax / 32;
  const int nch = (V + 31) / 32;
  for (int c = tid >> 5; c < nch; c += kW) {
    const int i = c * 32 + (tid & 31);
    int32_t mn = i < V ? S.lo[i] : INT32_MAX, mx = i < V ? S.hi[i] : INT32_MIN;
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(kFull, mn, o));
      mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    }
    if ((tid & 31) == 0) {
      cmin[c] = mn;
      cmax[c] = mx;
    }
  }
  if (tid == 0) *sh = 0;
  __syncthreads();
  // test every tree edge (par(y), y); keys reuse the F region
  for (int y = tid; y < V; y += kT) {
    if (S.par[y] == kNone16) continue;
    const int32_t l = S.pre[y], r = min(V, l + max((int32_t)S.sz[y], 1));
    int32_t mn = INT32_MAX, mx = INT32_MIN;
    const int32_t cl = (l + 31) / 32, cr = r / 32;
    if (cl >= cr) {
      for (int i = l; i < r; i++) mn = min(mn, S.lo[i]), mx = max(mx, S.hi[i]);
    } else {
      for (int i = l; i < cl * 32; i++) mn = min(mn, S.lo[i]), mx = max(mx, S.hi[i]);
      for (int c = cl; c < cr; c++) mn = min(mn, cmin[c]), mx = max(mx, cmax[c]);
      for (int i = cr * 32; i < r; i++) mn = min(mn, S.lo[i]), mx = max(mx, S.hi[i]);
    }
    if (mn >= l && mx < r) {
      const uint32_t a = (uint32_t)min(y, (int)S.par[y]), b = (uint32_t)max(y, (int)S.par[y]);
      const int32_t k = atomicAdd(sh, 1);
      if (k < V) S.keys[k] = (a << 12) | b;
    }
  }
  __syncthreads();
  const int32_t n = min(*sh, max(V - 1, 0));
  if (n <= kT) {
    // rank sort: keys are unique (a bridge has no parallel copy), every thread ranks one key
    // against all n with broadcast reads; one pass, no barrier
    if (tid < n) {
      const uint32_t mine = S.keys[tid];
      int32_t rank = 0;
      for (int j = 0; j < n; j++) rank += S.keys[j] < mine;
      out[2 * rank] = (int32_t)(mine >> 12);
      out[2 * rank + 1] = (int32_t)(mine & 0xfff);
    }
    __syncthreads();
    return n;
  }
  // bitonic sort of n keys (padded to a power of two with ~0)
  int np = 1;
  while (np < n) np <<= 1;
  for (int i = n + tid; i < np; i += kT) S.keys[i] = 0xffffffffu;
  __syncthreads();
  for (int k = 2; k <= np; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < np; i += kT) {
        const int l = i ^ j;
        if (l > i) {
          const uint32_t x = S.keys[i], y = S.keys[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            S.keys[i] = y;
            S.keys[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < n; i += kT) {
    out[2 * i] = (int32_t)(S.keys[i] >> 12);
    out[2 * i + 1] = (int32_t)(S.keys[i] & 0xfff);
  }
  __syncthreads();
  return n;
}

__global__ void __launch_bounds__(kT, 1) batched_kernel(const BatchArgs* __restrict__ dA) {
  const BatchArgs A = *dA;
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ int32_t red[kW];
  __shared__ int32_t task_sh, n1, n2, err, flag, sh;
  const Smem S = carve_smem(smem_raw);
  const int tid = threadIdx.x;
  const int32_t ntasks = *A.d_ntasks;
  while (true) {
    __syncthreads();  // every thread is done with the previous task (and with task_sh)
    if (tid == 0) task_sh = atomicAdd(A.queue, 1);
    __syncthreads();
    const int32_t t = task_sh;
    if (t >= ntasks) break;
    const BatchTask T = A.tasks[t];
    const int32_t V = T.V;
    // a malformed descriptor is skipped, never used to index shared memory
    const int64_t stride = 2 + 2 * (int64_t)V;
    if (V < 0 || V > kVmax || T.lo < 0 || T.hi < T.lo || T.g < 0 || T.g >= A.G || T.nparts < 1 ||
        T.part < 0 || T.part >= T.nparts || !T.count || (V > 1 && !T.out) ||
        (T.nparts > 1 && (T.slot < (int64_t)T.part * stride ||
                          T.slot + (int64_t)(T.nparts - T.part) * stride > A.slot_words))) {
      if (tid == 0 && T.count) *T.count = BRIDGES_EINTERNAL;
      continue;
    }
    for (int x = tid; x < V; x += kT) {
      S.P1[x] = x;
      S.P2[x] = x;
    }
    if (tid == 0) {
      n1 = 0;
      n2 = 0;
      err = 0;
    }
    __syncthreads();
    s_certify_range(S, T.u, T.v, T.lo, T.hi, V, &n1, &n2, &err);
    __syncthreads();
    int32_t nt = min(n1, V), nx = min(n2, V);
    if (T.nparts > 1) {
      // publish this partition's certificate; the last partition of the graph merges
      uint32_t* slot = A.slots + T.slot;
      for (int i = tid; i < nt; i += kT) slot[2 + i] = S.F1[i];
      for (int i = tid; i < nx; i += kT) slot[2 + nt + i] = S.F2[i];
      if (tid == 0) {
        slot[0] = (uint32_t)nt;
        slot[1] = (uint32_t)nx;
        if (err) atomicExch(A.gerr + T.g, err);
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) flag = atomicAdd(A.done + T.g, 1) == T.nparts - 1;
      __syncthreads();
      if (!flag) continue;
      __threadfence();
      // merge: certify the union of every partition's certificate (this one included)
      for (int x = tid; x < V; x += kT) {
        S.P1[x] = x;
        S.P2[x] = x;
      }
      if (tid == 0) {
        n1 = 0;
        n2 = 0;
        const int32_t e = ld_relaxed(A.gerr + T.g);
        if (e) err = e;
      }
      __syncthreads();
      for (int p = 0; p < T.nparts; p++) {
        const uint32_t* sp = A.slots + T.slot - (int64_t)T.part * stride + (int64_t)p * stride;
        const int32_t pn = (int32_t)(__ldcg(sp) + __ldcg(sp + 1));
        s_certify_packed(S, sp + 2, min(pn, 2 * V), V, &n1, &n2);
        __syncthreads();
      }
      nt = min(n1, V);
      nx = min(n2, V);
    }
    int64_t* cnt = T.count;
    if (err) {
      if (tid == 0) *cnt = err;
      __syncthreads();
      continue;
    }
    const int32_t nb = s_bridges(S, V, nt, nx, T.out, red, &sh);
    if (tid == 0) *cnt = nb;
    __syncthreads();
  }
}

}  // namespace

size_t batched_smem_bytes() { return (size_t)kSmem; }

bool batched_launch(cudaStream_t s, const BatchArgs* dev_args, int num_sms) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  });
  batched_kernel<<<num_sms, kT, kSmem, s>>>(dev_args);
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace bridges
