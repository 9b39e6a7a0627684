// batched.cu -- many small graphs in two persistent launches.
//
// Certification (certify_kernel): four 256-thread groups per block take tasks from a queue with
// two ends (most edges first; one group per block starts with the fewest).  A task is a whole
// graph (V <= 4096) or one partition of its edge list (Sec. 3: the edges split into contiguous
// sets).  The group certifies the task's edges with two concurrent union-finds in SHARED memory
// (Alg. 2: F, then F' from the edges F rejects) and appends the winners to the task's slot in
// global memory, so it holds only the union-finds (8 bytes per vertex) and four graphs share an
// SM: while one runs its warm-up prefix edge by edge (latency bound), the others stream their
// edges.  A graph of up to 1,024 vertices (one task) is certified straight into the bridge
// stage's shared-memory layout and its bridge stage runs right there, beside the other groups'
// streams.
//
// Bridges (bridge_kernel), for the larger graphs: per graph, a group copies its certificate from
// its slot (one task) or offers the F then F' edges of every one of the graph's slots to fresh
// union-finds in shared memory (several: the Sec. 3 merge with fan-in = the number of partitions)
// and runs the bridge stage.  The stage is the same Euler-tour / preorder-range test as final.cu,
// on 16-bit arrays with barriers between phases (list ranking by a ruling set, subtree ranges
// from shuffle windows and chunk extrema), then a rank sort of the packed (a << 12 | b) keys
// (bitonic above the group's thread count).  A graph's fixed cost is its barriers, so graphs of
// up to 3,008 vertices run two per block: the block splits into 512-thread groups with their own
// half of shared memory and their own named barrier, so that one graph's barrier waits overlap
// with the other's work.  Nothing waits on another block, so there is no spin anywhere.
#include <algorithm>

#include "../../include/bridges.h"
#include "batched.h"
#include "common.cuh"

namespace bridges {

namespace {

constexpr int kT = 1024;           // threads per block
constexpr int kVmax = kBatchVmax;  // 4096: a whole block's graph
constexpr int kHalfT = kT / 2;     // threads of a half-block group
constexpr int kHalfVmax = kBatchHalfVmax;  // 3008: a half-block group's graph
constexpr int kQuarterT = kT / 4;     // threads of a quarter-block group
constexpr int kQuarterVmax = kBatchQuarterVmax;  // 1024: a quarter-block (certification) group's graph
constexpr uint16_t kNone16 = 0xffff;
constexpr int kRuleGap = 8;  // list ranking: a ruler every kRuleGap arcs (by index)

constexpr int a16(int x) { return (x + 15) & ~15; }
// Shared-memory layout for graphs of up to VM vertices (bytes, each region a multiple of 16),
// in address order R0, R2, R1, R3, ...:
//   R0  P1 (int32[V]); later each arc's ruler (u16[2V]); later aoff + vbase (u16[V+1] each);
//       later the chunk tables of the range test
//   R1  P2 (int32[V]); later root + cur (u16[V+2] each)
//   R2  F list (u32[V]); later bridge keys (u32[V])
//   R3  F' list (u32[V])
//   R4  chunk minima / maxima (int32[V/32] each)
//   R5  head (int32[V]); later lo (int32[V]); before the stage, with R6, a merge's staging copy
//   R6  next (u16[2V]); later each arc's place in its sublist; later hi (int32[V])
//   R7  succ (u16[2V]); later dflag / dscan (u16[2V+1]); later in-chunk prefix extrema (u16[V] x 2)
//   R8  rnk (u16[2V]); later the vertex at each preorder position
//   R9  pre, sz, par (u16[V] each); earlier the rulers' two packed buffers (3 VM / 4 words each)
template <int VM>
struct Layout {
  static constexpr int kU16 = a16(2 * (VM + 16));  // a u16[V+2] array
  static constexpr int R0 = 2 * kU16 > 4 * VM ? 2 * kU16 : 4 * VM;
  static constexpr int R1 = R0;
  static constexpr int R2 = 4 * VM;
  static constexpr int R3 = 4 * VM;
  static constexpr int R4 = VM / 4;
  static constexpr int R5 = 4 * VM;
  static constexpr int R6 = 4 * VM;
  static constexpr int R7 = a16(2 * (2 * VM + 8));
  static constexpr int R8 = 4 * VM;
  static constexpr int R9 = 6 * VM;
  static constexpr int kBytes = R0 + R1 + R2 + R3 + R4 + R5 + R6 + R7 + R8 + R9;
};
constexpr int cmax(int a, int b) { return a > b ? a : b; }
// a half block's share holds one half-group layout
constexpr int kHalfBytes = Layout<kHalfVmax>::kBytes;
constexpr int kSmem = cmax(Layout<kVmax>::kBytes, 2 * kHalfBytes);
static_assert(kHalfVmax % 32 == 0 && kHalfBytes % 16 == 0, "half layouts: whole chunks, 16-byte regions");
static_assert(kSmem + 2048 <= 227 * 1024, "the bridge kernel's shared memory (with its static part) fits a block");

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
  int32_t* chunk;
  uint16_t* dst;
  int32_t* head;
  uint16_t* next;
  int32_t* lo;
  int32_t* hi;
  uint16_t* succ;
  uint16_t* dflag;
  uint16_t* rnk;
  uint16_t* pre;
  uint16_t* sz;
  uint16_t* par;
};

template <int VM>
__device__ Smem carve_smem(char* base) {
  using L = Layout<VM>;
  Smem s;
  char* c = base;
  s.P1 = reinterpret_cast<int32_t*>(c);
  s.aoff = reinterpret_cast<uint16_t*>(c);
  s.vbase = reinterpret_cast<uint16_t*>(c + L::kU16);
  c += L::R0;
  s.F1 = reinterpret_cast<uint32_t*>(c);
  s.keys = s.F1;
  c += L::R2;
  s.P2 = reinterpret_cast<int32_t*>(c);
  s.root = reinterpret_cast<uint16_t*>(c);
  s.cur = reinterpret_cast<uint16_t*>(c + L::kU16);
  c += L::R1;
  s.F2 = reinterpret_cast<uint32_t*>(c);
  c += L::R3;
  s.chunk = reinterpret_cast<int32_t*>(c);
  c += L::R4;
  s.dst = reinterpret_cast<uint16_t*>(c);
  s.head = reinterpret_cast<int32_t*>(c);
  s.lo = reinterpret_cast<int32_t*>(c);
  c += L::R5;
  s.next = reinterpret_cast<uint16_t*>(c);
  s.hi = reinterpret_cast<int32_t*>(c);
  c += L::R6;
  s.succ = reinterpret_cast<uint16_t*>(c);
  s.dflag = s.succ;
  c += L::R7;
  s.rnk = reinterpret_cast<uint16_t*>(c);
  c += L::R8;
  s.pre = reinterpret_cast<uint16_t*>(c);
  s.sz = s.pre + VM;
  s.par = s.sz + VM;
  return s;
}

// A group of NT threads (whole block, a half or a quarter) working on one task: its thread index
// and its barrier (0 = the block's; named barriers 1, 2 for the bridge kernel's halves and 1 to 4
// for the certification groups, the quarters).
template <int NT>
struct Grp {
  int tid;
  int bar;
  __device__ __forceinline__ void sync() const {
    if (NT == kT)
      __syncthreads();
    else
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(NT) : "memory");
  }
};

// Per-group scalars in shared memory.
struct GroupShared {
  int32_t red[kT / 32];
  int32_t red_b[kT / 32];
  int32_t task, n1, n2, err, flag, sh;
};

// Concurrent union-find in shared memory: the algorithm of uf_link (common.cuh) -- parents are
// compared first (a grandparent equal to the other end's parent also proves one set), a root is
// hooked under the other end's parent, a smaller vertex, so P[x] <= x always.
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
      if (atomicCAS(P + x, x, py) == x) return true;
      continue;
    }
    const int32_t g = VP[px];
    if (g == py) {
      VP[x] = g;
      return false;
    }
    if (g == px) {
      if (atomicCAS(P + px, px, py) == px) return true;
      continue;
    }
    VP[x] = g;
    x = g;
  }
}

// Block-wide exclusive scan of n (<= 2*NT*... ) u16 values in place; returns the total.
template <int NT>
__device__ int32_t block_scan16(const Grp<NT>& G, uint16_t* a, int32_t n, int32_t* red) {
  const int per = (n + NT - 1) / NT;  // contiguous items per thread
  const int lo = min(n, G.tid * per), hi = min(n, lo + per);
  int32_t s = 0;
  for (int i = lo; i < hi; i++) s += a[i];
  const int lane = G.tid & 31, w = G.tid >> 5;
  int32_t incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) red[w] = incl;
  G.sync();
  int32_t base = 0, tot = 0;
  for (int k = 0; k < (NT / 32); k++) {
    if (k < w) base += red[k];
    tot += red[k];
  }
  int32_t run = base + incl - s;
  for (int i = lo; i < hi; i++) {
    const int32_t v = a[i];
    a[i] = (uint16_t)run;
    run += v;
  }
  G.sync();
  return tot;
}

// The same for two arrays of equal length at once (one pair of block barriers for both).
template <int NT>
__device__ void block_scan16_pair(const Grp<NT>& G, uint16_t* a, uint16_t* b, int32_t n, int32_t* red,
                                  int32_t* red_b) {
  const int per = (n + NT - 1) / NT;
  const int lo = min(n, G.tid * per), hi = min(n, lo + per);
  int32_t sa = 0, sb = 0;
  for (int i = lo; i < hi; i++) {
    sa += a[i];
    sb += b[i];
  }
  const int lane = G.tid & 31, w = G.tid >> 5;
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
  G.sync();
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
  G.sync();
}

// Offers edge (a, b) to F, then F'; appends winners (warp-aggregated).  Every lane calls it.
__device__ __forceinline__ void s_settle(const Smem& S, bool need, int32_t a, int32_t b, int32_t* n1, int32_t* n2,
                                         int32_t V) {
  if (!__any_sync(kFull, need)) return;
  int r = 0;
  if (need) r = s_link(S.P1, a, b) ? 1 : (s_link(S.P2, a, b) ? 2 : 0);
  const unsigned m1 = __ballot_sync(kFull, r == 1), m2 = __ballot_sync(kFull, r == 2);
  const int lane = threadIdx.x & 31;  // groups are whole warps
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
template <int NT>
__device__ __forceinline__ void s_flatten(const Grp<NT>& G, int32_t* P, int32_t V) {
  G.sync();
  for (int x = G.tid; x < V; x += NT) {
    int32_t r = x, p = P[x];
    while (p != r) {
      r = p;
      p = P[r];
    }
    P[x] = r;
  }
  G.sync();
}

// Scalar certification of edges [lo, hi): every lane takes one edge per step.
template <int NT>
__device__ void s_certify_scalar(const Grp<NT>& G, const Smem& S, const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                 int64_t lo, int64_t hi, int32_t V, int32_t* n1, int32_t* n2, int32_t* err) {
  volatile int32_t* P2 = S.P2;
  // the next step's edge is loaded before this step's union-find work, so the load's latency
  // overlaps it instead of adding to every step
  int64_t i = lo + G.tid;
  int32_t a = i < hi ? __ldcs(u + i) : 0, b = i < hi ? __ldcs(v + i) : 0;
  for (int64_t t0 = lo; t0 < hi; t0 += NT, i += NT) {
    const bool valid = i < hi;
    const int64_t j = i + NT;
    const int32_t na = j < hi ? __ldcs(u + j) : 0, nb = j < hi ? __ldcs(v + j) : 0;
    bool need = valid;
    if (need && ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V)) {
      *err = BRIDGES_ERANGE;
      need = false;
    }
    if (need && (a == b || P2[a] == P2[b])) need = false;
    s_settle(S, need, a, b, n1, n2, V);
    a = na;
    b = nb;
  }
}

// The lanes' flagged edges of one tile go through the union-finds (bit 4k+c of m: element
// 4*(base + k*NT + tid) + c of ub / vb).  Out of line: rare after the flatten.
template <int NT>
__device__ __noinline__ void s_offer_misses(const Grp<NT>& G, const Smem& S, uint32_t m, const int32_t* __restrict__ ub,
                                            const int32_t* __restrict__ vb, int64_t base, int32_t V, int32_t* n1,
                                            int32_t* n2, int32_t* err) {
  while (__any_sync(kFull, m != 0)) {
    int32_t a = 0, b = 0;
    bool go = false;
    if (m) {
      const int bit = __ffs(m) - 1;
      m &= m - 1;
      const int64_t e = 4 * (base + (int64_t)(bit >> 2) * NT + G.tid) + (bit & 3);
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
template <int NT, int VM>
__device__ __forceinline__ void s_certify_vec(const Grp<NT>& G, const Smem& S, const int32_t* __restrict__ u, const int32_t* __restrict__ v, int64_t lo,
                              int64_t hi, int32_t V, int32_t* n1, int32_t* n2, int32_t* err) {
  constexpr int U = 4;
  if (lo >= hi) return;
  // the vector body starts on a 128-byte line of both arrays when they share their offset within
  // a line (a warp's 512 bytes of loads then touch four lines, not five), else on a 16-byte boundary
  const uintptr_t d = reinterpret_cast<uintptr_t>(u) ^ reinterpret_cast<uintptr_t>(v);
  const uintptr_t amask = (d & 127) == 0 ? 127 : 15;
  int64_t body = lo;
  if ((d & 15) == 0) {
    while (body < hi && (reinterpret_cast<uintptr_t>(u + body) & amask)) body++;
  } else {
    body = hi;
  }
  s_certify_scalar(G, S, u, v, lo, body, V, n1, n2, err);
  const int64_t nunits = (hi - body) >> 2;
  const int32_t* ub = u + body;
  const int32_t* vb = v + body;
  const int4* u4 = reinterpret_cast<const int4*>(ub);
  const int4* v4 = reinterpret_cast<const int4*>(vb);
  volatile int32_t* P2 = S.P2;
  const uint32_t cl = (uint32_t)(VM - 1);
  for (int64_t base = 0; base < nunits; base += (int64_t)NT * U) {
    int4 ua[U], va[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      const int64_t idx = base + (int64_t)k * NT + G.tid;
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
      if (base + (int64_t)k * NT + G.tid >= nunits) continue;
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
    if (__any_sync(kFull, m != 0)) s_offer_misses(G, S, m, ub, vb, base, V, n1, n2, err);
  }
  s_certify_scalar(G, S, u, v, body + 4 * nunits, hi, V, n1, n2, err);
}

// Certifies edges [lo, hi) of (u, v) into S.F1 / S.F2 (appending to *n1 / *n2); ids outside
// [0, V) set *err.  A warm-up prefix goes edge by edge (most of its edges still link; a vector
// tile's miss loop would run as long as its busiest lane), then both union-finds are flattened,
// so that "equal F' parents" afterwards recognises nearly every pair inside one F' component,
// and the rest streams through the vector loop.
template <int NT, int VM>
__device__ void s_certify_range(const Grp<NT>& G, const Smem& S, const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                                int64_t lo, int64_t hi, int64_t warm_edges, int32_t V, int32_t* n1, int32_t* n2,
                                int32_t* err) {
  // the task's prefix (the host's plan: 4V + 2048 unless tuned)
  const int64_t warm = min(hi - lo, max(warm_edges, (int64_t)0));
  s_certify_scalar(G, S, u, v, lo, lo + warm, V, n1, n2, err);
  lo += warm;
  if (lo >= hi) return;
  s_flatten(G, S.P1, V);
  s_flatten(G, S.P2, V);
  s_certify_vec<NT, VM>(G, S, u, v, lo, hi, V, n1, n2, err);
}

// Certifies packed edges (a | b << 16) of a list in shared memory.
template <int NT>
__device__ void s_certify_packed(const Grp<NT>& G, const Smem& S, const uint32_t* e, int32_t n, int32_t V, int32_t* n1, int32_t* n2) {
  volatile int32_t* P2 = S.P2;
  for (int32_t t0 = 0; t0 < n; t0 += NT) {
    const int32_t i = t0 + G.tid;
    const bool valid = i < n;
    const uint32_t x = valid ? e[i] : 0;
    const int32_t a = (int32_t)(x & 0xffff), b = (int32_t)(x >> 16);
    const bool need = valid && a != b && P2[a] != P2[b];
    s_settle(S, need, a, b, n1, n2, V);
  }
}

// Bridges of the certificate in S (F1 = tree, F2 = extra), written sorted to out; returns count.
template <int NT, int VM>
__device__ int32_t s_bridges(const Grp<NT>& G, const Smem& S, int32_t V, int32_t nt, int32_t nx, int32_t* out,
                             int32_t* red, int32_t* red_b, int32_t* sh) {
  const int tid = G.tid;
  // roots (minimum vertex of each tree)
  for (int x = tid; x < V; x += NT) {
    int32_t r = x, p = S.P1[x];
    while (p != r) {
      r = p;
      p = S.P1[r];
    }
    S.root[x] = (uint16_t)r;  // P2 region: F' union-find no longer needed
    S.head[x] = -1;
  }
  G.sync();
  // arcs 2e (a -> b) and 2e + 1 (b -> a) of tree edge e = F1[e] = (a, b): each vertex's outgoing
  // arcs in a list (head, next) built by one atomic exchange per arc
  const int32_t narcs = 2 * nt;
  for (int e = tid; e < nt; e += NT) {
    const uint32_t p = S.F1[e];
    S.next[2 * e] = (uint16_t)atomicExch(S.head + (p & 0xffff), 2 * e);
    S.next[2 * e + 1] = (uint16_t)atomicExch(S.head + (p >> 16), 2 * e + 1);
  }
  G.sync();
  // Euler-tour successors, cut at each root: after arc i into y comes the arc that follows i's
  // twin (y's arc back) in y's list, wrapping to its first arc except at the root
  uint16_t* succ = S.succ;  // R7
  for (int i = tid; i < narcs; i += NT) {
    const uint32_t p = S.F1[i >> 1];
    const int32_t y = (int32_t)((i & 1) ? (p & 0xffff) : (p >> 16));
    uint16_t s = S.next[i ^ 1];
    if (s == kNone16 && S.root[y] != y) s = (uint16_t)S.head[y];
    succ[i] = s;
  }
  if (tid == 0) *sh = 0;
  G.sync();
  // List ranking (rank = arcs after the arc in its tour) by a ruling set: every kRuleGap-th arc
  // by index and the head of every tour (a root's first arc, which no arc points to) start a
  // sublist that ends before the next ruler; one lane walks each sublist, recording for each arc
  // its ruler and its place in the sublist; the rulers' own list is ranked by pointer jumping,
  // four hops per round; then every arc subtracts its place from its ruler's count.  Random
  // shared-memory loads bound this step, and this reads each arc about three times in all where
  // pointer jumping over every arc reads it four times a round.
  //   R0 (free now) and R6 (next, free now): per arc, its ruler and its place (u16 each)
  //   R9 (pre / sz / par, written later): two buffers of packed (next ruler | arcs << 16) words
  //   R1's cur half (free now): the first arc of each extra ruler (heads off the kRuleGap grid)
  // A forest with t trees has at most (2V - 2t) / kRuleGap + t + 1 <= 5V/8 + 1 rulers.
  {
    const int32_t nreg = (narcs + kRuleGap - 1) / kRuleGap;
    for (int x = tid; x < V; x += NT) {
      const int32_t h = S.head[x];
      if (S.root[x] == x && h >= 0 && h % kRuleGap != 0) S.cur[atomicAdd(sh, 1)] = (uint16_t)h;
    }
    G.sync();
    const int32_t nrul = nreg + *sh;
    uint16_t* oruler = reinterpret_cast<uint16_t*>(S.P1);  // R0
    uint16_t* oplace = S.next;                             // R6
    uint32_t* ra = reinterpret_cast<uint32_t*>(S.pre);  // R9: 3 VM / 4 words each
    uint32_t* rb = ra + 3 * VM / 4;
    for (int k = tid; k < nrul; k += NT) {
      uint32_t i = k < nreg ? (uint32_t)(k * kRuleGap) : S.cur[k - nreg];
      uint32_t place = 0, next = kNone16;
      for (int32_t step = 0; step < narcs; step++) {  // a tour is a path: a sublist has < narcs arcs
        oruler[i] = (uint16_t)k;
        oplace[i] = (uint16_t)place;
        place++;
        const uint32_t s = succ[i];
        if (s == kNone16) break;
        if (s % kRuleGap == 0) {
          next = s / kRuleGap;
          break;
        }
        i = s;
      }
      ra[k] = next | (place << 16);
    }
    G.sync();
    int rounds = 0;
    while ((1 << (2 * rounds)) < max(nrul, 1)) rounds++;
    for (int r = 0; r < rounds; r++) {
      for (int k = tid; k < nrul; k += NT) {
        const uint32_t w = ra[k];
        uint32_t nx = w & 0xffffu, acc = w >> 16;
#pragma unroll
        for (int h = 0; h < 3 && nx != kNone16; h++) {
          const uint32_t x = ra[nx];
          acc += x >> 16;
          nx = x & 0xffffu;
        }
        rb[k] = nx | (acc << 16);
      }
      G.sync();
      uint32_t* t = ra;
      ra = rb;
      rb = t;
    }
    // ra[k] >> 16: the arcs from ruler k's first arc to the end of its tour
    for (int i = tid; i < narcs; i += NT) S.rnk[i] = (uint16_t)((ra[oruler[i]] >> 16) - oplace[i] - 1);
    G.sync();
  }
  // per root: tour arcs (aoff) and tree vertices (vbase); P1 region is free now
  if (nt == V - 1) {
    // one spanning tree, whose root is vertex 0 (the minimum of its set): its tour takes every
    // arc and its vertices every preorder number, and no other entry is read
    if (tid == 0) {
      S.aoff[0] = 0;
      S.aoff[1] = (uint16_t)narcs;
      S.vbase[0] = 0;
    }
  } else {
    for (int x = tid; x <= V; x += NT) {
      uint16_t L = 0, nv = 0;
      if (x < V && S.root[x] == x) {
        L = S.head[x] >= 0 ? (uint16_t)(S.rnk[S.head[x]] + 1) : 0;
        nv = (uint16_t)(L / 2 + 1);
      }
      S.aoff[x] = L;
      S.vbase[x] = nv;
    }
    G.sync();
    block_scan16_pair(G, S.aoff, S.vbase, V + 1, red, red_b);
  }
  // tour positions; down arcs (dflag reuses succ, free after ranking)
  for (int i = tid; i <= narcs; i += NT) S.dflag[i] = 0;
  G.sync();
  for (int i = tid; i < narcs; i += NT) {
    const uint32_t pe = S.F1[i >> 1];
    const int32_t a = (int32_t)(pe & 0xffff), b = (int32_t)(pe >> 16);
    const int32_t x = (i & 1) ? b : a, y = (i & 1) ? a : b;  // arc i: x -> y
    const int32_t ri = S.rnk[i], rt = S.rnk[i ^ 1];
    // the tour of x's root r fills positions [aoff[r], aoff[r + 1]); arc i is ri arcs from its end
    const int32_t g = S.aoff[S.root[x] + 1] - 1 - ri;
    if (g < 0 || g >= narcs) continue;
    if (ri > rt) {
      S.dflag[g] = 1;
      S.par[y] = (uint16_t)x;
      S.pre[y] = (uint16_t)g;
      S.sz[y] = (uint16_t)((ri - rt + 1) / 2);
    }
  }
  G.sync();
  block_scan16(G, S.dflag, narcs, red);  // dscan in place
  // preorder numbers; lo / hi (dst and twin are free now)
  for (int x = tid; x < V; x += NT) {
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
    const int32_t q = min(max(p, 0), V - 1);
    S.pre[x] = (uint16_t)q;
    S.rnk[q] = (uint16_t)x;  // the vertex at each preorder position (rnk is free now)
    S.lo[q] = q;
    S.hi[q] = q;
  }
  G.sync();
  for (int e = tid; e < nx; e += NT) {
    const uint32_t p = S.F2[e];
    const int32_t a = (int32_t)(p & 0xffff), b = (int32_t)(p >> 16);
    if (a == b) continue;
    const int32_t pa = S.pre[a], pb = S.pre[b];
    atomicMin(S.lo + pa, pb);
    atomicMin(S.lo + pb, pa);
    atomicMax(S.hi + pa, pb);
    atomicMax(S.hi + pb, pa);
  }
  G.sync();
  // per chunk of 32 preorder positions: the in-chunk prefix minima of lo and maxima of hi (u16, in
  // the dflag region, free now) and the chunk's minimum / maximum
  uint16_t* plo = S.dflag;
  uint16_t* phi = S.dflag + VM;
  int32_t* cmin = S.chunk;
  int32_t* cmax = cmin + VM / 32;
  const int nch = (V + 31) / 32;
  const int lane = tid & 31;
  for (int c = tid >> 5; c < nch; c += (NT / 32)) {  // warp-uniform
    const int i = c * 32 + lane;
    int32_t mn = i < V ? S.lo[i] : INT32_MAX, mx = i < V ? S.hi[i] : INT32_MIN;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t a = __shfl_up_sync(kFull, mn, o), b = __shfl_up_sync(kFull, mx, o);
      if (lane >= o) mn = min(mn, a), mx = max(mx, b);
    }
    if (i < V) {
      plo[i] = (uint16_t)mn;
      phi[i] = (uint16_t)mx;
    }
    if (lane == 31) {
      cmin[c] = mn;
      cmax[c] = mx;
    }
  }
  if (tid == 0) *sh = 0;
  G.sync();
  // superchunks of 32 chunks, a warp each: the extrema of windows of 2^j chunks (j < 6, cut at
  // the superchunk's end), the in-superchunk prefix and suffix extrema and each superchunk's
  // extrema (int32, in the P1 region, free now), so that any run of whole chunks is a few loads
  constexpr int NC = VM / 32;
  static_assert((16 * NC + 2 * (NC / 32 + 1)) * 4 <= Layout<VM>::R0, "the chunk tables fit the P1 region");
  int32_t* wcl = S.P1;           // [6][NC] window minima of lo
  int32_t* wch = wcl + 6 * NC;   // [6][NC] window maxima of hi
  int32_t* pcl = wch + 6 * NC;   // in-superchunk prefix
  int32_t* pch = pcl + NC;
  int32_t* scl = pch + NC;       // in-superchunk suffix
  int32_t* sch = scl + NC;
  int32_t* sml = sch + NC;       // [NC / 32 + 1] superchunk extrema
  int32_t* smh = sml + NC / 32 + 1;
  const int nsc = (nch + 31) / 32;
  if ((tid >> 5) < nsc) {  // warp-uniform
    const int w = tid >> 5, c = w * 32 + lane;
    const int32_t a0 = c < nch ? cmin[c] : INT32_MAX, b0 = c < nch ? cmax[c] : INT32_MIN;
    int32_t wa = a0, wb = b0;
#pragma unroll
    for (int j = 0; j < 6; j++) {
      if (c < nch) {
        wcl[j * NC + c] = wa;
        wch[j * NC + c] = wb;
      }
      if (j < 5) {
        const int o = 1 << j;
        const int32_t ta = __shfl_down_sync(kFull, wa, o), tb = __shfl_down_sync(kFull, wb, o);
        if (lane + o < 32) wa = min(wa, ta), wb = max(wb, tb);
      }
    }
    int32_t pa = a0, pb = b0, sa = a0, sb = b0;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t x1 = __shfl_up_sync(kFull, pa, o), x2 = __shfl_up_sync(kFull, pb, o);
      const int32_t y1 = __shfl_down_sync(kFull, sa, o), y2 = __shfl_down_sync(kFull, sb, o);
      if (lane >= o) pa = min(pa, x1), pb = max(pb, x2);
      if (lane + o < 32) sa = min(sa, y1), sb = max(sb, y2);
    }
    if (c < nch) {
      pcl[c] = pa;
      pch[c] = pb;
      scl[c] = sa;
      sch[c] = sb;
    }
    if (lane == 31) {
      sml[w] = pa;
      smh[w] = pb;
    }
  }
  G.sync();
  // test every tree edge (par(y), y), whose subtree holds the preorder positions [p, p + sz(y)),
  // p = pre(y): a warp takes a chunk of 32 positions, a lane one position.  The subtree's part in
  // the chunk, [p, e), is covered by two power-of-two windows, [p, p + 2^k) and [e - 2^k, e),
  // whose extrema the warp builds and exchanges by shuffles; past the chunk come the whole
  // chunks (two windows within a superchunk, else a suffix, a prefix and the superchunks between)
  // and the last chunk's prefix.
  const uint16_t* vtx = S.rnk;
  for (int c = tid >> 5; c < nch; c += (NT / 32)) {  // warp-uniform
    const int32_t p = c * 32 + lane;
    int32_t wa[6], wb[6];  // extrema of [p, p + 2^j), cut at the chunk's end
    wa[0] = p < V ? S.lo[p] : INT32_MAX;
    wb[0] = p < V ? S.hi[p] : INT32_MIN;
#pragma unroll
    for (int j = 1; j < 6; j++) {
      const int o = 1 << (j - 1);
      const int32_t a = __shfl_down_sync(kFull, wa[j - 1], o), b = __shfl_down_sync(kFull, wb[j - 1], o);
      wa[j] = lane + o < 32 ? min(wa[j - 1], a) : wa[j - 1];
      wb[j] = lane + o < 32 ? max(wb[j - 1], b) : wb[j - 1];
    }
    int32_t y = 0, py = kNone16, r = p;
    if (p < V) {
      y = min((int32_t)vtx[p], V - 1);
      py = S.par[y];
      r = min(V, p + max((int32_t)S.sz[y], 1));
    }
    const bool live = p < V && py != kNone16;
    const int32_t e = min(r, c * 32 + 32);
    const int32_t len = max(e - p, 1);  // lane + len <= 32
    const int k = 31 - __clz(len);
    int32_t mn = INT32_MAX, mx = INT32_MIN;
#pragma unroll
    for (int j = 0; j < 6; j++) {
      const int src = min(max(lane + len - (1 << j), 0), 31);
      const int32_t a = __shfl_sync(kFull, wa[j], src), b = __shfl_sync(kFull, wb[j], src);
      if (k == j) {
        mn = min(wa[j], a);
        mx = max(wb[j], b);
      }
    }
    // past the chunk: whole chunks [c + 1, cr), then chunk cr's prefix up to r - 1
    if (live && r > e) {
      const int32_t cl = c + 1, cr = (r - 1) >> 5;
      mn = min(mn, (int32_t)plo[r - 1]);
      mx = max(mx, (int32_t)phi[r - 1]);
      if (cl < cr) {
        const int32_t s0 = cl >> 5, s1 = (cr - 1) >> 5;
        if (s0 == s1) {
          const int j = 31 - __clz(cr - cl);
          const int32_t c2 = cr - (1 << j);
          mn = min(mn, min(wcl[j * NC + cl], wcl[j * NC + c2]));
          mx = max(mx, max(wch[j * NC + cl], wch[j * NC + c2]));
        } else {
          mn = min(mn, min(scl[cl], pcl[cr - 1]));
          mx = max(mx, max(sch[cl], pch[cr - 1]));
          for (int32_t q = s0 + 1; q < s1; q++) mn = min(mn, sml[q]), mx = max(mx, smh[q]);
        }
      }
    }
    if (live && mn >= p && mx < r) {
      const uint32_t a = (uint32_t)min(y, py), b = (uint32_t)max(y, py);
      const int32_t kk = atomicAdd(sh, 1);
      if (kk < V) S.keys[kk] = (a << 12) | b;
    }
  }
  G.sync();
  const int32_t n = min(*sh, max(V - 1, 0));
  if (n <= NT) {
    // rank sort: keys are unique (a bridge has no parallel copy), every thread ranks one key
    // against all n with broadcast reads; one pass, no barrier
    if (tid < n) {
      const uint32_t mine = S.keys[tid];
      int32_t rank = 0;
      for (int j = 0; j < n; j++) rank += S.keys[j] < mine;
      out[2 * rank] = (int32_t)(mine >> 12);
      out[2 * rank + 1] = (int32_t)(mine & 0xfff);
    }
    G.sync();
    return n;
  }
  int np = 1;
  while (np < n) np <<= 1;
  if (np > VM) {
    // more keys than the threads and a power of two above the key array's capacity: every thread
    // ranks several keys against all n (keys are unique)
    for (int i = tid; i < n; i += NT) {
      const uint32_t mine = S.keys[i];
      int32_t rank = 0;
      for (int j = 0; j < n; j++) rank += S.keys[j] < mine;
      out[2 * rank] = (int32_t)(mine >> 12);
      out[2 * rank + 1] = (int32_t)(mine & 0xfff);
    }
    G.sync();
    return n;
  }
  // bitonic sort of n keys (padded to a power of two with ~0)
  for (int i = n + tid; i < np; i += NT) S.keys[i] = 0xffffffffu;
  G.sync();
  for (int k = 2; k <= np; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < np; i += NT) {
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
      G.sync();
    }
  }
  for (int i = tid; i < n; i += NT) {
    out[2 * i] = (int32_t)(S.keys[i] >> 12);
    out[2 * i + 1] = (int32_t)(S.keys[i] & 0xfff);
  }
  G.sync();
  return n;
}

constexpr int kAT = 256;               // threads of a certification group
constexpr int kAGroups = kT / kAT;     // certification groups per block
static_assert(kAT == kQuarterT, "a certification group runs the quarter-class bridge stages");
// a certification group's shared memory: the union-finds (P1, P2) of a graph of up to kVmax
// vertices, or the whole bridge-stage layout of a quarter-class graph
constexpr int kABytes = cmax(8 * kVmax, Layout<kQuarterVmax>::kBytes);
static_assert(kABytes % 16 == 0, "group regions stay 16-byte aligned");

// The certificate slot of task T (batch_slot_words).
__device__ __forceinline__ uint32_t* task_slot(const BatchArgs& A, const BatchTask& T) { return A.slots + T.slot; }

// Whether T's descriptor can be used (a malformed one is skipped, never used to index memory).
__device__ __forceinline__ bool task_ok(const BatchArgs& A, const BatchTask& T) {
  const int64_t stride = batch_slot_words(T.V);
  return T.V >= 0 && T.V <= kVmax && T.lo >= 0 && T.hi >= T.lo && T.g >= 0 && T.g < A.G && T.nparts >= 1 &&
         T.part >= 0 && T.part < T.nparts && T.count && (T.V <= 1 || T.out) && T.slot >= (int64_t)T.part * stride &&
         T.slot + (int64_t)(T.nparts - T.part) * stride <= A.slot_words;
}

// Certifies task T by group G of NT threads.  A quarter-class graph (one task, at most
// kQuarterVmax vertices) is certified into the bridge stage's layout in the group's shared memory
// and finished here; any other task keeps only its two union-finds in shared memory and appends
// its winners to its slot (the graph's first task also leaves the roots of its forests there).
template <int NT>
__device__ void certify_task(const BatchArgs& A, const BatchTask& T, char* smem, const Grp<NT>& G,
                             GroupShared& gs) {
  const int tid = G.tid;
  if (!task_ok(A, T)) {
    if (tid == 0 && T.g >= 0 && T.g < A.G) atomicExch(A.gerr + T.g, BRIDGES_EINTERNAL);
    return;
  }
  const int32_t V = T.V;
  if (T.cls == 2) {
    if (V > kQuarterVmax || T.nparts != 1) {  // not a quarter-class task: never run past the layout
      if (tid == 0) *T.count = BRIDGES_EINTERNAL;
      return;
    }
    // a quarter-class graph (one task, at most kQuarterVmax vertices): certified straight into the
    // bridge stage's shared-memory layout, then its bridge stage runs here, beside the other
    // groups' streams, instead of in bridge_kernel
    const Smem S = carve_smem<kQuarterVmax>(smem);
    for (int x = tid; x < V; x += NT) {
      S.P1[x] = x;
      S.P2[x] = x;
    }
    if (tid == 0) {
      gs.n1 = 0;
      gs.n2 = 0;
      gs.err = 0;
    }
    G.sync();
    s_certify_range<NT, kQuarterVmax>(G, S, T.u, T.v, T.lo, T.hi, T.warm, V, &gs.n1, &gs.n2, &gs.err);
    G.sync();
    const int32_t nt = min(gs.n1, V), nx = min(gs.n2, V), err = gs.err;
    if (err) {
      if (tid == 0) *T.count = err;
      return;
    }
    const int32_t nb = s_bridges<NT, kQuarterVmax>(G, S, V, nt, nx, T.out, gs.red, gs.red_b, &gs.sh);
    if (tid == 0) *T.count = nb;
    return;
  }
  uint32_t* slot = task_slot(A, T);
  Smem S{};
  S.P1 = reinterpret_cast<int32_t*>(smem);
  S.P2 = S.P1 + kVmax;
  S.F1 = slot + 2;      // global: winners are appended straight to the slot
  S.F2 = slot + 2 + V;
  for (int x = tid; x < V; x += NT) {
    S.P1[x] = x;
    S.P2[x] = x;
  }
  if (tid == 0) {
    gs.n1 = 0;
    gs.n2 = 0;
    gs.err = 0;
  }
  G.sync();
  s_certify_range<NT, kVmax>(G, S, T.u, T.v, T.lo, T.hi, T.warm, V, &gs.n1, &gs.n2, &gs.err);
  if (T.part == 0) {
    // the graph's first task: the roots of its F trees (and, when more tasks follow, of its F'
    // trees), so that the bridge stage starts from this task's union-finds as they stand and
    // offers only the other tasks' edges
    s_flatten(G, S.P1, V);
    if (T.nparts > 1) s_flatten(G, S.P2, V);
    uint16_t* roots1 = reinterpret_cast<uint16_t*>(slot + 2 + 2 * (int64_t)V);
    uint16_t* roots2 = reinterpret_cast<uint16_t*>(slot + 2 + 2 * (int64_t)V + (V + 1) / 2);
    for (int x = tid; x < V; x += NT) {
      roots1[x] = (uint16_t)S.P1[x];
      if (T.nparts > 1) roots2[x] = (uint16_t)S.P2[x];
    }
  }
  G.sync();
  if (tid == 0) {
    slot[0] = (uint32_t)min(gs.n1, V);
    slot[1] = (uint32_t)min(gs.n2, V);
    if (gs.err) atomicExch(A.gerr + T.g, gs.err);
  }
}

// Copies words [0, n) of src (global) to dst(i) (shared memory) with eight loads per thread in
// flight before their stores: a plain copy loop waits for one load per round.
template <int NT, class Dst>
__device__ __forceinline__ void copy_in(const uint32_t* __restrict__ src, int32_t n, int tid, Dst dst) {
  for (int32_t base = 0; base < n; base += 8 * NT) {
    uint32_t r[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int32_t i = base + k * NT + tid;
      r[k] = i < n ? __ldcg(src + i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int32_t i = base + k * NT + tid;
      if (i < n) dst(i, r[k]);
    }
  }
}

// Bridges of the graph whose first task is T (later partitions are skipped): its slots' F and F'
// edges offered to fresh union-finds (one slot: the same two forests again; several: the Sec. 3
// merge), then the bridge stage, by a group of NT threads whose graphs have at most VM vertices.
template <int NT, int VM>
__device__ void bridge_task(const BatchArgs& A, const BatchTask& T, const Smem& S, const Grp<NT>& G, GroupShared& gs) {
  const int tid = G.tid;
  if (T.part != 0 || T.cls == 2) return;  // quarter-class graphs are finished by certify_kernel
  if (!task_ok(A, T) || T.V > VM) {
    if (tid == 0 && T.count) *T.count = BRIDGES_EINTERNAL;
    return;
  }
  const int32_t V = T.V;
  const int64_t stride = batch_slot_words(V);
  if (tid == 0) {
    gs.n1 = 0;
    gs.n2 = 0;
    gs.err = ld_relaxed(A.gerr + T.g);
  }
  // the first task's F and F' as they stand, with the roots of their trees (P1 and P2 then hold
  // each vertex's root: offering those lists again to fresh union-finds would rebuild exactly
  // these forests).  For one task that is the graph's certificate.
  const uint32_t* sp = task_slot(A, T);
  const int32_t nf = min((int32_t)__ldcg(sp), V), nx0 = min((int32_t)__ldcg(sp + 1), V);
  const int32_t rw = (V + 1) / 2;  // words of a roots array (two 16-bit roots a word)
  // one copy of the F region, the F' region and the roots array(s), which follow each other
  copy_in<NT>(sp + 2, 2 * V + (T.nparts > 1 ? 2 * rw : rw), tid, [&](int32_t i, uint32_t w) {
    if (i < V) {
      if (i < nf) S.F1[i] = w;
    } else if (i < 2 * V) {
      if (i - V < nx0) S.F2[i - V] = w;
    } else {
      const int32_t j = i - 2 * V;
      int32_t* P = j < rw ? S.P1 : S.P2;
      const int32_t x = 2 * (j < rw ? j : j - rw);
      if (x < V) P[x] = min((int32_t)(w & 0xffffu), V - 1);
      if (x + 1 < V) P[x + 1] = min((int32_t)(w >> 16), V - 1);
    }
  });
  if (tid == 0) {
    gs.n1 = nf;
    gs.n2 = nx0;
  }
  G.sync();
  // the other tasks: the Sec. 3 merge -- each slot's F and F' edges offered to the union-finds.
  // Each slot is read with all of a thread's loads in flight and filtered on the way: an edge
  // whose ends already have the same F' parent is joined in both forests (F' components lie
  // inside F components, and sets only grow), so only the others are staged in shared memory
  // (the dst region, 2 VM words, free until the bridge stage) and offered, in any order (every
  // order leaves F a spanning forest of the offered edges and F' one of the rest).
  uint32_t* stage = reinterpret_cast<uint32_t*>(S.dst);
  volatile int32_t* P2v = S.P2;
  // two staging counters used in turn (red_b is free until the bridge stage): slot p counts in
  // cnt[p & 1], and cnt[(p + 1) & 1], last read in slot p - 1's pass, is reset after the barrier
  // that ends that pass
  int32_t* cnt = gs.red_b;
  if (tid == 0) {
    cnt[0] = 0;
    cnt[1] = 0;
  }
  for (int p = 1; p < T.nparts; p++) {
    const uint32_t* pp = sp + (int64_t)p * stride;
    const int32_t mf = min((int32_t)__ldcg(pp), V), mx = min((int32_t)__ldcg(pp + 1), V);
    G.sync();  // the previous slot's edges are settled: the stage is free
    if (tid == 0) cnt[(p + 1) & 1] = 0;
    copy_in<NT>(pp + 2, 2 * V, tid, [&](int32_t i, uint32_t w) {
      if (i < V ? i >= mf : i - V >= mx) return;
      const int32_t a = (int32_t)(w & 0xffff), b = (int32_t)(w >> 16);
      if (a < V && b < V && a != b && P2v[a] != P2v[b]) stage[atomicAdd(cnt + (p & 1), 1)] = w;
    });
    G.sync();
    s_certify_packed(G, S, stage, min(cnt[p & 1], 2 * V), V, &gs.n1, &gs.n2);
  }
  G.sync();
  const int32_t nt = min(gs.n1, V), nx = min(gs.n2, V);
  if (gs.err) {
    G.sync();  // every thread has read gs.err before the next task resets it
    if (tid == 0) *T.count = gs.err;
    return;
  }
  const int32_t nb = s_bridges<NT, VM>(G, S, V, nt, nx, T.out, gs.red, gs.red_b, &gs.sh);
  if (tid == 0) *T.count = nb;
}

// Takes tasks first + 0, 1, ... from `queue` until `last` and runs their bridge stage on group G.
template <int NT, int VM>
__device__ void run_queue(const BatchArgs& A, char* smem, const Grp<NT>& G, GroupShared& gs, int32_t* queue,
                          int32_t first, int32_t last) {
  const Smem S = carve_smem<VM>(smem);
  while (true) {
    G.sync();  // every thread of the group is done with the previous task (and with gs.task)
    if (G.tid == 0) gs.task = first + atomicAdd(queue, 1);
    G.sync();
    const int32_t t = gs.task;
    if (t >= last) break;
    bridge_task<NT, VM>(A, A.tasks[t], S, G, gs);
  }
}

// Claims the next position of corder, or -1 when none is left.  One 64-bit word counts the claims
// at both ends (the front's in the low half, the back's in the high half), so one atomic add
// sees both: a front claim f succeeds while f + min(b, nback) < n, a back claim b while b < nback
// and f + b < n (task n - 1 - b).  No position is claimed twice, and none is missed: after a back
// claim fails, every later one fails too and its group claims from the front.
__device__ __noinline__ int32_t claim_task(unsigned long long* q, int32_t n, int32_t nback, bool& back) {
  if (back) {
    const unsigned long long old = atomicAdd(q, 1ull << 32);
    const int64_t f = (int64_t)(old & 0xffffffffull), b = (int64_t)(old >> 32);
    if (b < nback && f + b < n) return (int32_t)(n - 1 - b);
    back = false;
  }
  const unsigned long long old = atomicAdd(q, 1ull);
  const int64_t f = (int64_t)(old & 0xffffffffull), b = (int64_t)(old >> 32);
  return f + min(b, (int64_t)nback) < n ? (int32_t)f : -1;
}

// Certifies tasks on group G in corder: most edges first, or, for a back group, the fewest edges
// first while the last nback tasks last, then from the front.
template <int NT>
__device__ void certify_queue(const BatchArgs& A, char* smem, const Grp<NT>& G, GroupShared& gs, bool back,
                              int32_t ntasks) {
  unsigned long long* q = reinterpret_cast<unsigned long long*>(A.queue + 4);
  const int32_t nback = min(max(A.nback, 0), ntasks);
  while (true) {
    G.sync();
    if (G.tid == 0) gs.task = claim_task(q, ntasks, nback, back);
    G.sync();
    const int32_t t = gs.task;
    if (t < 0) break;
    certify_task<NT>(A, A.tasks[A.corder[t]], smem, G, gs);
  }
}

// Persistent certification: four 256-thread groups per block (named barriers 1-4), each with a
// quarter of the shared memory, take the tasks in corder (most edges first, so that the longest
// lists start early); one group's warm-up prefix (edge by edge, latency bound) overlaps the other
// groups' streams.  The last group of each block starts from the back of corder: the smallest
// graphs are almost all prefix, and taken last they would leave HBM idle at the end of the
// launch; taken beside the long streams they are hidden.  (Whole blocks for the long tasks were
// measured slower: a block alone on its SM has no other group's stream to hide its own prefix
// behind.)
__global__ void __launch_bounds__(kT, 1) certify_kernel(const BatchArgs* __restrict__ dA) {
  const BatchArgs A = *dA;
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ GroupShared gs[kAGroups];
  const int32_t ntasks = *A.d_ntasks;
  const int k = (int)threadIdx.x / kAT;
  certify_queue<kAT>(A, smem_raw + k * kABytes, Grp<kAT>{(int)threadIdx.x % kAT, 1 + k}, gs[k],
                     k == kAGroups - 1, ntasks);
}

// Persistent bridge stages: whole-block tasks first (graphs above kHalfVmax vertices and
// partitioned graphs); then the block splits into two independent half-block groups, each with
// half the shared memory and its own named barrier, for graphs of up to kHalfVmax vertices.  A
// small graph's cost is mostly its barriers, and this overlaps two of them on one SM.  No barrier
// spans groups after the split.  (Quarter-class graphs were finished by certify_kernel.)
__global__ void __launch_bounds__(kT, 1) bridge_kernel(const BatchArgs* __restrict__ dA) {
  const BatchArgs A = *dA;
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ GroupShared gs[3];  // [0] the block, then [1 + h] each half
  const int32_t ntasks = *A.d_ntasks;
  const int32_t nbig = min(max(A.nbig, 0), ntasks);
  const int32_t nmid = min(max(A.nmid, 0), ntasks - nbig);
  run_queue<kT, kVmax>(A, smem_raw, Grp<kT>{(int)threadIdx.x, 0}, gs[0], A.queue, 0, nbig);
  __syncthreads();  // the halves reuse the shared memory
  const int h = (int)threadIdx.x / kHalfT;
  char* half = smem_raw + h * kHalfBytes;
  const Grp<kHalfT> gh{(int)threadIdx.x % kHalfT, 1 + h};
  run_queue<kHalfT, kHalfVmax>(A, half, gh, gs[1 + h], A.queue + 1, nbig, nbig + nmid);
}

// The bridge stage of one graph of 2..kVmax vertices on one block, in place of the grid-wide
// final stage when only the sorted bridges and their count are wanted: the final certificate (F
// and F' in global memory) is packed into the shared-memory layout, F's union-find copied as it
// stands (its roots root the trees), and s_bridges runs with block barriers only -- no grid
// barrier, no cooperative launch.
__global__ void __launch_bounds__(kT, 1) small_final_kernel(const SmallFinalArgs A) {
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ GroupShared gs;
  const Smem S = carve_smem<kVmax>(smem_raw);
  const Grp<kT> G{(int)threadIdx.x, 0};
  const int tid = (int)threadIdx.x;
  const int32_t V = min(max(A.V, 0), kVmax);
  const int32_t nt = min(max(ld_relaxed(A.d_nt), 0), max(V - 1, 0));
  const int32_t nx = min(max(ld_relaxed(A.d_nx), 0), V);
  for (int x = tid; x < V; x += kT) {
    const int32_t p = __ldcg(A.P + x);
    S.P1[x] = (p >= 0 && p <= x) ? p : x;
  }
  int bad = 0;  // a certificate edge out of range (never expected: its edges passed the range test)
  for (int e = tid; e < nt; e += kT) {
    const int32_t a = __ldcg(A.tu + e), b = __ldcg(A.tv + e);
    bad |= (uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V;
    S.F1[e] = (uint32_t)(a & 0xffff) | ((uint32_t)(b & 0xffff) << 16);
  }
  for (int e = tid; e < nx; e += kT) {
    const int32_t a = __ldcg(A.xu + e), b = __ldcg(A.xv + e);
    bad |= (uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V;
    S.F2[e] = (uint32_t)(a & 0xffff) | ((uint32_t)(b & 0xffff) << 16);
  }
  const bool any_bad = __syncthreads_or(bad) != 0;
  int32_t st = ld_relaxed(A.status);  // the same value for every thread: no stage writes it now
  if (st == 0 && any_bad) st = BRIDGES_EINTERNAL;
  if (st != 0) {
    if (tid == 0) *A.count = st;
    return;
  }
  const int32_t nb = s_bridges<kT, kVmax>(G, S, V, nt, nx, A.out, gs.red, gs.red_b, &gs.sh);
  if (tid == 0) *A.count = nb;
}

}  // namespace

size_t batched_smem_bytes() { return (size_t)kSmem; }

bool small_final_launch(cudaStream_t s, const SmallFinalArgs& a) {
  if (a.V < 2 || a.V > kVmax) return false;
  cudaFuncSetAttribute(small_final_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, Layout<kVmax>::kBytes);
  small_final_kernel<<<1, kT, Layout<kVmax>::kBytes, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess;
}

bool batched_launch(cudaStream_t s, const BatchArgs* dev_args, int num_sms) {
  // function attributes are per device: set on every launch (a host-side call; the launches are
  // usually replayed from a CUDA graph anyway)
  cudaFuncSetAttribute(certify_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kAGroups * kABytes);
  cudaFuncSetAttribute(bridge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  certify_kernel<<<num_sms, kT, kAGroups * kABytes, s>>>(dev_args);
  bridge_kernel<<<num_sms, kT, kSmem, s>>>(dev_args);
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace bridges
