// blocks.cu -- articulation points ("failure points", abstract of the paper) on the GPU.
//
// Bridges survive any pair of spanning forests (Alg. 2), cut vertices do not: an arbitrary
// F u F' can split a biconnected graph at a vertex.  This path therefore takes the spanning
// forest T of the bridge path (the F of the final certificate, rooted and numbered in preorder
// by the final stage) and streams the whole edge list a second time against T:
//
//   * A tree edge (x, parent x) is named by the preorder number of x.  Every non-tree edge
//     (a, b) closes a fundamental cycle with T, and all tree edges of one cycle lie in one block
//     (biconnected component).  The blocks restricted to T are exactly the classes of the
//     transitive closure of "lie on a common fundamental cycle", so merging, edge by edge, the
//     classes that each cycle touches ends with one class per block (Tarjan & Vishkin 1985 reach
//     the same classes through their auxiliary graph).
//   * A class is always a connected subtree of T (merges only join classes that share a
//     vertex), so it has one topmost vertex, its head, and every tree path from one of its
//     vertices up to the head stays inside it.  With the classes kept in a union-find over
//     preorder numbers whose root is the minimum element, the root is the class's first edge in
//     preorder, a child of the head: head = parent of the root.  A cycle is walked from each end
//     by jumping from class to head until the walk reaches an ancestor of the other end; the
//     classes met are joined in walk order (each shares a vertex with the previous one).
//   * A vertex is an articulation point iff its tree edges fall into at least two classes
//     (each block through a vertex holds one of its tree edges).
//
// An edge whose two ends lie in one class is redundant: its cycle is inside the class.  Once the
// classes start as the blocks of the certificate S = T u F' (linked in O(V) by Tarjan & Vishkin's
// rules, below) and a short prefix of the list has been walked, nearly every edge is, so
// the stream reuses the forest pass's machinery: a 16-bit label per vertex in shared memory (the
// largest class containing the vertex), two label reads per edge, and the cycle walk only for
// the misses.  Classes only grow, so a stale label is still sound.  When 2V bytes of labels do
// not fit in shared memory, one bit per vertex marks the largest class of all instead (both
// ends in it: redundant), for the vertices below the bitmap's reach; every other edge walks.
//
// For one partition with labels the two streams are fused into one (see "the fused path"
// below): the forest after the certificate's warm-up is rooted early and serves as T for every
// edge inside one of its trees.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "forest.cuh"
#include "stream.cuh"

namespace bridges {

namespace {

constexpr int kUnroll = 4;

struct ApArgs {
  const int32_t* pre;   // [V] vertex -> preorder number (final stage)
  int32_t* Q;           // [V] class union-find over preorder numbers
  const int32_t* PP;    // [V] preorder number of the parent (-1: tree root)
  const int32_t* LAST;  // [V] last preorder number of the subtree
  int32_t V;
  int32_t* status;
  int32_t* hooks;  // successful class merges
};

// Merges the classes of the tree edges on the fundamental cycle of the edge between the
// vertices with preorder numbers A and B; returns the number of successful hooks.
__device__ int32_t cycle_merge(const ApArgs& A, int32_t a, int32_t b) {
  if (a == b) return 0;
  int32_t hooks = 0;
  int32_t last[2];
  for (int side = 0; side < 2; side++) {
    int32_t x = side ? b : a;
    const int32_t y = side ? a : b;
    int32_t prev = -1;
    // climb while x is not an ancestor of y: then x's tree edge is on the cycle
    for (int32_t it = 0; !(x <= y && y <= __ldg(A.LAST + x)); it++) {
      if (it >= A.V) {  // cannot happen on a forest: each step moves strictly up
        set_status(A.status, BRIDGES_EINTERNAL_CODE);
        return hooks;
      }
      if (prev >= 0 && uf_link(A.Q, prev, x)) hooks++;  // prev's class has head x: they touch
      prev = x;
      const int32_t h = __ldg(A.PP + uf_find(A.Q, x));
      if (h < 0) {  // only if the ends lie in different trees of T
        set_status(A.status, BRIDGES_EINTERNAL_CODE);
        return hooks;
      }
      x = h;
    }
    last[side] = prev;
  }
  // both last classes hold the lowest common ancestor
  if (last[0] >= 0 && last[1] >= 0 && uf_link(A.Q, last[0], last[1])) hooks++;
  return hooks;
}

__device__ __forceinline__ bool checked_edge(const ApArgs& A, int32_t a, int32_t b) {
  if ((uint32_t)a >= (uint32_t)A.V || (uint32_t)b >= (uint32_t)A.V) {
    set_status(A.status, BRIDGES_ERANGE_CODE);
    return false;
  }
  return a != b;
}

__device__ __forceinline__ void offer_edge(const ApArgs& A, int32_t a, int32_t b) {
  if (!checked_edge(A, a, b)) return;
  const int32_t h = cycle_merge(A, __ldg(A.pre + a), __ldg(A.pre + b));
  if (h) atomicAdd(A.hooks, h);
}

__device__ __noinline__ void cycle_misses(const ApArgs& A, uint32_t m, const int32_t* __restrict__ u,
                                          const int32_t* __restrict__ v, int64_t base) {
  while (m) {
    const int bit = __ffs(m) - 1;
    m &= m - 1;
    const int64_t e = miss_edge(bit, base);
    offer_edge(A, u[e], v[e]);
  }
}

// The block pass's slow path (see stream_range).
struct CycleSink {
  const ApArgs& A;
  __device__ __forceinline__ void slot(bool need, int32_t a, int32_t b, int64_t) const {
    if (need) offer_edge(A, a, b);
  }
  __device__ __forceinline__ void misses(uint32_t m, const int32_t* ub, const int32_t* vb, int64_t base) const {
    cycle_misses(A, m, ub, vb, base);
  }
};

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// Preorder-indexed copies of T (parent, subtree end, vertex), singleton classes, and the jump of
// Tarjan & Vishkin's rule 2 (below): J[i] = the parent's edge if tree edge i joins it, else i.
__global__ void ap_init_kernel(FinalBufs f, ApBufs b, int32_t V) {
  if (*f.status) return;
  for (int64_t x = gtid(); x < V; x += gstride()) {
    const int32_t i = f.pre[x], p = f.par[x], s = f.sz[x];
    b.flag[x] = 0;
    if ((uint32_t)i >= (uint32_t)V || p >= V || (p >= 0 && (uint32_t)f.pre[p] >= (uint32_t)V) || s < 1 ||
        (int64_t)i + s > V) {
      set_status(f.status, BRIDGES_EINTERNAL_CODE);
      continue;
    }
    const int32_t pp = p >= 0 ? f.pre[p] : -1;
    b.vtx[i] = (int32_t)x;
    b.PP[i] = pp;
    b.LAST[i] = i + s - 1;
    b.Q[i] = i;
    b.csize[i] = INT32_MAX;  // the fused form's renaming takes class minima here
    // rule 2: y's subtree has a certificate neighbour outside p's subtree (p not a root)
    bool join = false;
    if (p >= 0 && f.par[p] >= 0) {
      const int32_t sp = f.sz[p];
      join = f.slo[x] < pp || (int64_t)f.shi[x] > (int64_t)pp + sp - 1;
    }
    b.tmp[i] = join ? pp : i;
  }
  if (gtid() == 0) *b.hooks = 0;
}

constexpr int kChainCap = 64;  // rule-2 chain steps walked directly; longer chains are linked

// Rule 2 alone links every tree edge to its parent's edge along upward chains, so its classes
// are read off by walking the jumps to the chain's top (J[t] == t): Q[i] = top, a valid flat
// union-find (the top is an ancestor: a smaller preorder number).  A walk that needs more than
// kChainCap steps stops there; the edge stays a singleton and records where it stopped (csize)
// for a union-find link in ap_tv_kernel, so the cost stays bounded on long chains.
__global__ void ap_chain_kernel(ApBufs b, int32_t V, const int32_t* status) {
  if (*status) return;
  for (int64_t i = gtid(); i < V; i += gstride()) {
    int32_t t = (int32_t)i;
    int k = 0;
    for (int32_t j = b.tmp[t]; j != t && k < kChainCap; j = b.tmp[t], k++) t = j;
    const bool top = b.tmp[t] == t;
    b.Q[i] = top ? t : (int32_t)i;
    b.csize[i] = top ? -1 : t;
  }
}

// The blocks of the certificate S = T u F' as the starting classes, by the two link rules of
// Tarjan & Vishkin (1985) over T: (1) a non-tree edge of S between two unrelated vertices joins
// their tree edges; (2) a tree edge (y, p), p not a root, joins p's tree edge when y's subtree
// has an S-neighbour outside p's subtree -- read off the subtree minimum / maximum preorder
// (slo / shi) that the bridge test computed.  Every link joins two edges of one fundamental
// cycle, and the closure of the links is the blocks of S restricted to T: each a connected
// subtree of T again once all links are in, which the cycle walk of the later passes needs.
// Rule 2's chains are already flattened by ap_chain_kernel; this kernel adds the links of the
// chains it cut short, then rule 1.
__global__ void ap_tv_kernel(FinalBufs f, ApArgs A, ApBufs b, const int32_t* xu, const int32_t* xv,
                             const int32_t* d_n, int32_t cap) {
  if (*A.status) return;
  const int32_t V = A.V;
  for (int64_t i = gtid(); i < V; i += gstride()) {
    const int32_t t = b.csize[i];
    if (t >= 0) uf_link(A.Q, (int32_t)i, t);
  }
  const int32_t n = min(*d_n, cap);
  for (int64_t e = gtid(); e < n; e += gstride()) {
    const int32_t a = xu[e], c = xv[e];
    if (!checked_edge(A, a, c)) continue;
    const int32_t pa = f.pre[a], pb = f.pre[c];
    const bool related = (pa <= pb && pb <= A.LAST[pa]) || (pb <= pa && pa <= A.LAST[pb]);
    if (!related) uf_link(A.Q, pa, pb);
  }
}

struct PassArgs {
  ApArgs A;
  const int32_t* u;
  const int32_t* v;
  int64_t s;  // edge range [s, t) shared by the grid
  int64_t t;
  const uint16_t* lab;
  int64_t Vpad;
  int32_t Vb;  // MODE 2: vertices covered by the bitmap (a multiple of 128)
};

// MODE 0: no snapshot (every edge walks); 1: 16-bit labels; 2: bitmap of vertices [0, Vb).
template <int MODE, bool VEC>
__global__ void __launch_bounds__(1024, 1) ap_pass_kernel(PassArgs P) {
  extern __shared__ __align__(16) uint16_t slab[];
  __shared__ int32_t stop;
  if (threadIdx.x == 0) stop = *P.A.status;
  __syncthreads();
  if (stop) return;  // block-uniform: the stream below contains barriers
  if (MODE == 1) load_labels(slab, P.lab, P.Vpad);
  if (MODE == 2) load_words(slab, P.lab, (P.Vb / 32 + 4) / 4);
  const CycleSink S{P.A};
  const uint32_t clampv = MODE == 2 ? (uint32_t)P.Vb : (uint32_t)P.A.V;
  if (MODE != 0 && use_tiles(P.s, P.t, gridDim.x, blockDim.x, kUnroll)) {  // the stream, interleaved tiles
    stream_range<MODE, VEC, kUnroll>(S, P.u, P.v, P.s, P.t, clampv, slab, blockIdx.x, gridDim.x);
  } else {  // the prefix (or a short list), a slice per block
    const int64_t n = P.t - P.s;
    const int64_t s = P.s + n * blockIdx.x / gridDim.x, t = P.s + n * (blockIdx.x + 1) / gridDim.x;
    stream_range<MODE, VEC, kUnroll>(S, P.u, P.v, s, t, clampv, slab);
  }
}

// ---- label snapshot: each vertex takes the largest class it belongs to ----
// 1) flatten the classes; reset sizes, proposals and label ids
__global__ void ap_flatten_kernel(ApBufs b, int32_t V, const int32_t* status) {
  if (*status) return;  // T is not valid: its arrays may be partly unset
  for (int64_t i = gtid(); i < V; i += gstride()) {
    int32_t r = (int32_t)i, p = __ldca(b.Q + i);
    while (p != r) {
      r = p;
      p = __ldca(b.Q + r);
    }
    b.Q[i] = r;
    b.csize[i] = 0;
    b.tmp[i] = -1;
    b.best[i] = 0;
  }
  if (gtid() == 0) {
    *b.nlab = 0;
    *b.giant = 0;
  }
}

// 2) class sizes (tree edges per class); lanes with the same root add once per warp
__global__ void ap_count_kernel(ApBufs b, int32_t V, const int32_t* status) {
  if (*status) return;  // T is not valid: its arrays may be partly unset
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < V; base += gstride()) {
    const int64_t i = base + threadIdx.x;
    const bool edge = i < V && b.PP[i] >= 0;
    const int32_t r = edge ? b.Q[i] : -1 - lane;
    const unsigned peers = __match_any_sync(kFull, r);
    if (edge && lane == __ffs(peers) - 1) atomicAdd(b.csize + r, __popc(peers));
  }
}

// 3) every class with >= 2 edges proposes itself to the two ends of each of its edges
__global__ void ap_propose_kernel(ApBufs b, int32_t V, const int32_t* status) {
  if (*status) return;  // T is not valid: its arrays may be partly unset
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < V; base += gstride()) {
    const int64_t i = base + threadIdx.x;
    const int32_t p = i < V ? b.PP[i] : -1;
    uint64_t key = 0;
    if (p >= 0) {
      const int32_t r = b.Q[i];
      const int32_t c = b.csize[r];
      if (c >= 2) key = ((uint64_t)c << 32) | (uint32_t)r;
    }
    if (key) atomicMax(reinterpret_cast<unsigned long long*>(b.best + i), key);
    // siblings share a parent: one proposal per distinct (parent, key) in the warp
    const unsigned peers = __match_any_sync(kFull, p) & __match_any_sync(kFull, key);
    if (key && lane == __ffs(peers) - 1) atomicMax(reinterpret_cast<unsigned long long*>(b.best + p), key);
    // the largest class overall (the bitmap snapshot's), one atomic per warp
    unsigned long long wmax = key;
    for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(kFull, wmax, o));
    if (lane == 0 && wmax) atomicMax(b.giant, wmax);
  }
}

// 4) 16-bit labels by vertex id; classes get ids on first sight (kNoLabel past 65,534)
__global__ void ap_label_kernel(ApBufs b, const int32_t* pre, int32_t V, const int32_t* status) {
  if (*status) return;  // T is not valid: its arrays may be partly unset
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < b.Vpad; base += gstride()) {
    const int64_t x = base + threadIdx.x;
    const uint64_t key = x < V ? b.best[pre[x]] : 0;
    const int32_t r = key ? (int32_t)(uint32_t)key : -1 - lane;
    const unsigned peers = __match_any_sync(kFull, r);
    const int leader = __ffs(peers) - 1;
    int32_t id = -1;
    if (key && lane == leader) {
      int32_t* slot = b.tmp + r;
      id = ld_relaxed(slot);
      if (id < 0) {
        const int32_t fresh = atomicAdd(b.nlab, 1);
        const int32_t old = atomicCAS(slot, -1, fresh);
        id = old < 0 ? fresh : old;
      }
    }
    id = __shfl_sync(kFull, id, leader);
    if (x < b.Vpad) b.lab[x] = (key && id >= 0 && id < (int32_t)kNoLabel) ? (uint16_t)id : kNoLabel;
  }
}

// 4') the bitmap instead of labels: bit x set iff x < min(V, Vb) and the largest class containing
//     x is the largest class of all; the words from Vb / 32 on stay clear (the clamp target of
//     ids past the bitmap and of out-of-range ids)
__global__ void ap_bitmap_kernel(ApBufs b, const int32_t* pre, int32_t V, int32_t Vb, const int32_t* status) {
  if (*status) return;  // T is not valid: its arrays may be partly unset
  const int64_t nw = Vb / 32 + 4;  // a multiple of 4 words: the pass copies 16-byte units
  const unsigned long long g = *b.giant;
  uint32_t* words = reinterpret_cast<uint32_t*>(b.lab);
  for (int64_t w = gtid(); w < nw; w += gstride()) {
    uint32_t bits = 0;
    for (int k = 0; k < 32; k++) {
      const int64_t x = w * 32 + k;
      if (g && x < V && x < Vb && b.best[pre[x]] == g) bits |= 1u << k;
    }
    words[w] = bits;
  }
}

// ---- articulation points from the final classes ----
__global__ void ap_mark_kernel(ApBufs b, int32_t V, const int32_t* status) {
  if (*status) return;
  for (int64_t i = gtid(); i < V; i += gstride()) {
    const int32_t p = b.PP[i];
    if (p < 0) continue;
    const int32_t gi = uf_find_static(b.Q, (int32_t)i);
    // a non-root parent compares with its own tree edge, a root with its first child's edge
    const int32_t gp = uf_find_static(b.Q, b.PP[p] >= 0 ? p : p + 1);
    if (gi != gp) b.flag[b.vtx[p]] = 1;
  }
}

constexpr int kCompactThreads = 1024;
constexpr int kCompactItems = 4;  // flags per thread and tile

// Ordered compaction of the flagged vertices: per-tile counts, one-block scan, scatter.
__global__ void ap_tile_count_kernel(ApBufs b, int32_t V, int64_t ntiles) {
  __shared__ int32_t red[kCompactThreads / 32];
  const int64_t tile_sz = (int64_t)kCompactThreads * kCompactItems;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int32_t c = 0;
    for (int k = 0; k < kCompactItems; k++) {
      const int64_t x = tile * tile_sz + k * kCompactThreads + threadIdx.x;
      c += x < V ? b.flag[x] : 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t t = 0;
      for (int w = 0; w < kCompactThreads / 32; w++) t += red[w];
      b.tiles[tile] = t;
    }
    __syncthreads();
  }
}

// One block: exclusive scan of the tile counts in place; the total (or the status) to *count.
__global__ void ap_tile_scan_kernel(ApBufs b, int64_t ntiles, const int32_t* status, int64_t* count) {
  __shared__ int32_t wsum[kCompactThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t carry = 0;
  for (int64_t t0 = 0; t0 < ntiles; t0 += blockDim.x) {
    const int64_t t = t0 + threadIdx.x;
    const int32_t c = t < ntiles ? b.tiles[t] : 0;
    int32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int32_t before = 0, total = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) {
      if (q < w) before += wsum[q];
      total += wsum[q];
    }
    if (t < ntiles) b.tiles[t] = carry + before + incl - c;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = *status ? (int64_t)*status : (int64_t)carry;
}

__global__ void ap_scatter_kernel(ApBufs b, int32_t V, int64_t ntiles, const int32_t* status, int32_t* out) {
  __shared__ int32_t wsum[kCompactThreads / 32];
  if (*status) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t tile_sz = (int64_t)kCompactThreads * kCompactItems;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int32_t at = b.tiles[tile];
    for (int k = 0; k < kCompactItems; k++) {
      const int64_t x = tile * tile_sz + k * kCompactThreads + threadIdx.x;
      const bool f = x < V && b.flag[x];
      const unsigned m = __ballot_sync(kFull, f);
      if (lane == 0) wsum[w] = __popc(m);
      __syncthreads();
      int32_t before = 0, total = 0;
      for (int q = 0; q < kCompactThreads / 32; q++) {
        if (q < w) before += wsum[q];
        total += wsum[q];
      }
      if (f) out[at + before + __popc(m & lanemask_lt())] = (int32_t)x;
      at += total;
      __syncthreads();
    }
  }
}

// ---- the fused path: the certificate's stream and the block pass in one read of the list ----
//
// The block pass needs a rooted spanning forest, which the bridge path only has at its end.  In
// a dense graph, though, F after the forest pass's warm-up (T_0) already spans nearly every
// vertex, and F only grows: T_0 is a subforest of the final T.  So T_0 is rooted and numbered
// right after the warm-up (the final stage on the partial certificate), its classes are seeded
// (the blocks of T_0 u F'), and one stream then serves both passes: an edge is dropped from
// shared memory when both ends carry the same combined label (same F' component, both in the
// largest class), otherwise it is offered to the union-finds and, unless it just became a tree
// edge, its cycle is merged on T_0 -- its path in the final T is its path in T_0 whenever both
// ends lie in one tree of T_0.  Edges between two trees of T_0 are marked in a bitmap over the
// list and walked once the final T is known, after the classes are renamed from T_0's edges to
// T's (every edge of T_0 is an edge of T).  Walking any edge of the list is a valid merge, so
// the marks need no order and no bound, and the bitmap is never cleared as a whole: a top-level
// bitmap (one bit per word, cleared by every call) says which words this call marked, and the
// walk clears each word it reads.  A stale bit in such a word only adds a walk.

struct FusedArgs {
  ApArgs A;               // classes over T_0: its preorder numbers, parents and subtree ends
  Job J;                  // the certificate's union-finds and lists (one partition)
  const int32_t* root0;   // [V] the root of each vertex's tree in T_0
  uint32_t* keep;         // [E/32 + 1] marks of the edges walked on the final T
  uint32_t* top;          // one bit per word of keep: marked in this call
  const int32_t* u;
  const int32_t* v;
  int64_t s, t;           // edge range of this launch
  const uint16_t* lab;    // combined labels (Vpad entries)
  int64_t Vpad;
};

// One edge per lane (list index i), every lane of the warp calls it; `go`: the lane has a live
// edge (ids in range, not a loop) that missed the snapshot.
template <bool FOREST>
__device__ __forceinline__ void fused_edge(const FusedArgs& F, bool go, int32_t a, int32_t b, int64_t i) {
  int r = 0;
  if (FOREST) {
    r = go ? offer(F.J, a, b) : 0;
    warp_append(r == 1, a, b, F.J.cnt + 0, F.J.f1u, F.J.f1v, F.A.V, F.A.status);
    warp_append(r == 2, a, b, F.J.cnt + 1, F.J.f2u, F.J.f2v, F.A.V, F.A.status);
  }
  // a new edge of T closes no cycle; an edge inside one tree of T_0 is walked now, any other
  // edge once the final T is known
  if (!go || r == 1) return;
  if (__ldg(F.root0 + a) == __ldg(F.root0 + b)) {
    const int32_t h = cycle_merge(F.A, __ldg(F.A.pre + a), __ldg(F.A.pre + b));
    if (h) atomicAdd(F.A.hooks, h);
  } else {
    const int64_t w = i >> 5;
    atomicOr(F.keep + w, 1u << (i & 31));
    atomicOr(F.top + (w >> 5), 1u << (w & 31));
  }
}

template <bool FOREST>
__device__ __noinline__ void fused_misses(const FusedArgs& F, uint32_t m, const int32_t* __restrict__ u,
                                          const int32_t* __restrict__ v, int64_t base) {
  while (__any_sync(kFull, m != 0)) {
    int32_t a = 0, b = 0;
    int64_t e = 0;
    bool go = false;
    if (m) {
      const int bit = __ffs(m) - 1;
      m &= m - 1;
      e = miss_edge(bit, base);
      a = u[e];
      b = v[e];
      go = checked_edge(F.A, a, b);
    }
    fused_edge<FOREST>(F, go, a, b, (u - F.u) + e);
  }
}

template <bool FOREST>
struct FusedSink {
  const FusedArgs& F;
  __device__ __forceinline__ void slot(bool need, int32_t a, int32_t b, int64_t i) const {
    fused_edge<FOREST>(F, need && checked_edge(F.A, a, b), a, b, i);
  }
  __device__ __forceinline__ void misses(uint32_t m, const int32_t* ub, const int32_t* vb, int64_t base) const {
    fused_misses<FOREST>(F, m, ub, vb, base);
  }
};

// FOREST: the edges after the warm-up prefix (certificate and block pass); otherwise the
// prefix itself, which the certificate has already seen (block pass only).
template <bool FOREST, bool VEC>
__global__ void __launch_bounds__(1024, 1) ap_fused_kernel(FusedArgs F) {
  extern __shared__ __align__(16) uint16_t slab[];
  __shared__ int32_t stop;
  if (threadIdx.x == 0) stop = *F.A.status;
  __syncthreads();
  if (stop) return;  // block-uniform: the stream below contains barriers
  load_labels(slab, F.lab, F.Vpad);
  const FusedSink<FOREST> S{F};
  if (FOREST && use_tiles(F.s, F.t, gridDim.x, blockDim.x, kUnroll)) {  // the stream after the prefix, in tiles
    stream_range<1, VEC, kUnroll>(S, F.u, F.v, F.s, F.t, (uint32_t)F.A.V, slab, blockIdx.x, gridDim.x);
  } else {  // the prefix (or a short list), a slice per block
    const int64_t n = F.t - F.s;
    const int64_t s = F.s + n * blockIdx.x / gridDim.x, t = F.s + n * (blockIdx.x + 1) / gridDim.x;
    stream_range<1, VEC, kUnroll>(S, F.u, F.v, s, t, (uint32_t)F.A.V, slab);
  }
}

// The combined snapshot, in place over the certificate's F' labels: a vertex keeps its F' label
// only if it lies in the largest class (whose label id the class root's tmp entry holds).
__global__ void ap_combine_kernel(uint16_t* flab, ApBufs b, int64_t Vpad, int32_t V, const int32_t* status) {
  if (*status) return;
  const unsigned long long g = *b.giant;
  const int32_t gid = g ? b.tmp[(int32_t)(uint32_t)g] : -1;
  for (int64_t x = gtid(); x < Vpad; x += gstride()) {
    const bool keep = x < V && gid >= 0 && gid < (int32_t)kNoLabel && b.lab[x] == (uint16_t)gid;
    if (!keep) flab[x] = kNoLabel;
  }
}

// T_0's classes renamed onto the final T: tree edge i of T_0 (child x, parent p) is the edge of
// T whose child is x or p, whichever T makes the child.  A class of T_0 is a connected subtree of
// T as well, so its renamed edges form one class of T whose root (minimum preorder number) is the
// minimum of its members' new names; b1's union-find is written flat, every member pointing at it.
// Two passes without contention on the big classes: 1) each tree edge records its new name (in
// b0.tmp) and its class (b0.csize, -1 for none), and the lanes of a warp that share a class take
// one atomicMin of their minimum into b1.csize[class]; 2) every new name points at its class's
// minimum.  (b0.tmp and b0.csize are free once the combined snapshot is built.)
__device__ __forceinline__ int32_t renamed(const FinalBufs& f, int32_t x, int32_t p, int32_t* status) {
  if (f.par[x] == p) return f.pre[x];
  if (f.par[p] == x) return f.pre[p];
  set_status(status, BRIDGES_EINTERNAL_CODE);  // T_0 must be part of T
  return -1;
}

__global__ void ap_rename_min_kernel(FinalBufs f, ApBufs b0, ApBufs b1, int32_t V) {
  if (*f.status) return;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < V; base += gstride()) {
    const int64_t i = base + threadIdx.x;
    int32_t n = -1, r = -1;
    if (i < V && b0.PP[i] >= 0) {
      r = uf_find_static(b0.Q, (int32_t)i);
      const int32_t pr = b0.PP[r];
      if (pr < 0) {
        set_status(f.status, BRIDGES_EINTERNAL_CODE);  // a class root is a tree edge
        r = -1;
      } else {
        n = renamed(f, b0.vtx[i], b0.vtx[b0.PP[i]], f.status);
        if (n < 0) r = -1;
      }
    }
    if (i < V) {
      b0.tmp[i] = n;
      b0.csize[i] = r;
    }
    // one reduction per distinct class among the warp's lanes (the whole warp takes part)
    unsigned todo = __ballot_sync(kFull, r >= 0);
    while (todo) {
      const int lead = __ffs(todo) - 1;
      const int32_t key = __shfl_sync(kFull, r, lead);
      const bool mine = r == key && r >= 0;
      todo &= ~__ballot_sync(kFull, mine);
      const int32_t mn = __reduce_min_sync(kFull, mine ? n : INT32_MAX);
      if (lane == lead) atomicMin(b1.csize + key, mn);
    }
  }
}

__global__ void ap_rename_set_kernel(ApBufs b0, ApBufs b1, int32_t V, const int32_t* status) {
  if (*status) return;
  for (int64_t i = gtid(); i < V; i += gstride()) {
    const int32_t r = b0.csize[i];
    if (r >= 0) b1.Q[b0.tmp[i]] = b1.csize[r];
  }
}

// The marked edges, walked on the final T: the words the top level names are read and cleared
// (marks past E are ignored).
__global__ void ap_kept_kernel(ApArgs A, const int32_t* u, const int32_t* v, uint32_t* keep, const uint32_t* top,
                               int64_t ntop, int64_t E) {
  const bool ok = *A.status == 0;
  for (int64_t t = gtid(); t < ntop; t += gstride()) {
    uint32_t words = top[t];
    while (words) {
      const int64_t w = t * 32 + (__ffs(words) - 1);
      words &= words - 1;
      uint32_t bits = keep[w];
      keep[w] = 0;
      while (ok && bits) {
        const int64_t i = w * 32 + (__ffs(bits) - 1);
        bits &= bits - 1;
        if (i < E) offer_edge(A, u[i], v[i]);
      }
    }
  }
}

int grid_of(const Launch& L, int64_t work, int block) {
  const int64_t g = ceil_div(std::max<int64_t>(work, 1), block);
  return (int)std::min<int64_t>(g, (int64_t)L.num_sms * 16);
}

template <int MODE, bool VEC>
void launch_pass(const Launch& L, const PassArgs& a, int grid, int block, size_t smem) {
  auto k = ap_pass_kernel<MODE, VEC>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<grid, block, smem, L.stream>>>(a);
  *L.launches += 1;
}

// Articulation points from the final classes: marking and ordered compaction into out, their
// number (or the status) into *count_dev.
void ap_finish(const Launch& L, const FinalBufs& f, const ApBufs& b, int32_t V, int32_t* out, int64_t* count_dev) {
  const int bs = 256;
  const int64_t ntiles = ceil_div(std::max(V, 1), (int64_t)kCompactThreads * kCompactItems);
  ap_mark_kernel<<<grid_of(L, V, bs), bs, 0, L.stream>>>(b, V, f.status);
  ap_tile_count_kernel<<<grid_of(L, ntiles * kCompactThreads, kCompactThreads), kCompactThreads, 0, L.stream>>>(
      b, V, ntiles);
  ap_tile_scan_kernel<<<1, kCompactThreads, 0, L.stream>>>(b, ntiles, f.status, count_dev);
  ap_scatter_kernel<<<grid_of(L, ntiles * kCompactThreads, kCompactThreads), kCompactThreads, 0, L.stream>>>(
      b, V, ntiles, f.status, out);
  *L.launches += 4;
}

// The classes' starting point on a rooted forest: T's preorder copies, then Tarjan & Vishkin's
// two rules over T u (xu, xv).
void ap_seed(const Launch& L, const FinalBufs& f, const ApBufs& b, int32_t V, const int32_t* xu, const int32_t* xv,
             const int32_t* d_nx) {
  const int bs = 256;
  const int g = grid_of(L, V, bs);
  ap_init_kernel<<<g, bs, 0, L.stream>>>(f, b, V);
  ApArgs A{f.pre, b.Q, b.PP, b.LAST, V, f.status, b.hooks};
  ap_chain_kernel<<<g, bs, 0, L.stream>>>(b, V, f.status);
  ap_tv_kernel<<<g, bs, 0, L.stream>>>(f, A, b, xu, xv, d_nx, V);
  *L.launches += 3;
}

// The snapshot of the classes: mode 1, 16-bit labels (each vertex labelled with the largest
// class containing it); mode 2, the bitmap of the largest class over vertices [0, Vb).
void ap_snapshot(const Launch& L, const FinalBufs& f, const ApBufs& b, int32_t V, int32_t mode, int32_t Vb) {
  const int bs = 256;
  const int g = grid_of(L, V, bs);
  ap_flatten_kernel<<<g, bs, 0, L.stream>>>(b, V, f.status);
  ap_count_kernel<<<g, bs, 0, L.stream>>>(b, V, f.status);
  ap_propose_kernel<<<g, bs, 0, L.stream>>>(b, V, f.status);
  if (mode == 2)
    ap_bitmap_kernel<<<grid_of(L, Vb / 32 + 4, bs), bs, 0, L.stream>>>(b, f.pre, V, Vb, f.status);
  else
    ap_label_kernel<<<grid_of(L, b.Vpad, bs), bs, 0, L.stream>>>(b, f.pre, V, f.status);
  *L.launches += 4;
}

template <bool FOREST, bool VEC>
void launch_fused(const Launch& L, const FusedArgs& a, int grid, int block) {
  auto k = ap_fused_kernel<FOREST, VEC>;
  const size_t smem = (size_t)a.Vpad * 2;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<grid, block, smem, L.stream>>>(a);
  *L.launches += 1;
}

}  // namespace

size_t ap_bytes(int32_t V) {
  const size_t Vs = (size_t)std::max(V, 1);
  const size_t Vpad = align_up(Vs + 1, 8);
  const size_t ntiles = ceil_div((int64_t)Vs, (int64_t)kCompactThreads * kCompactItems);
  size_t s = 4 * 256;                                    // hooks, nlab, count, giant
  s += 7 * align_up(sizeof(int32_t) * Vs, 256);          // Q PP LAST vtx csize tmp flag
  s += align_up(sizeof(uint64_t) * Vs, 256);             // best
  s += align_up(sizeof(int32_t) * (ntiles + 1), 256);    // tiles
  s += align_up(sizeof(uint16_t) * Vpad, 256);           // lab
  return s;
}

ApBufs carve_ap(void* base, int32_t V) {
  ApBufs b{};
  char* c = static_cast<char*>(base);
  const size_t Vs = (size_t)std::max(V, 1);
  const size_t ntiles = ceil_div((int64_t)Vs, (int64_t)kCompactThreads * kCompactItems);
  b.hooks = reinterpret_cast<int32_t*>(c);
  b.nlab = reinterpret_cast<int32_t*>(c + 256);
  b.count = reinterpret_cast<int64_t*>(c + 512);
  b.giant = reinterpret_cast<unsigned long long*>(c + 768);
  c += 4 * 256;
  int32_t** arrs[7] = {&b.Q, &b.PP, &b.LAST, &b.vtx, &b.csize, &b.tmp, &b.flag};
  for (auto a : arrs) {
    *a = reinterpret_cast<int32_t*>(c);
    c += align_up(sizeof(int32_t) * Vs, 256);
  }
  b.best = reinterpret_cast<uint64_t*>(c);
  c += align_up(sizeof(uint64_t) * Vs, 256);
  b.tiles = reinterpret_cast<int32_t*>(c);
  c += align_up(sizeof(int32_t) * (ntiles + 1), 256);
  b.lab = reinterpret_cast<uint16_t*>(c);
  b.Vpad = (int64_t)align_up(Vs + 1, 8);
  return b;
}

void articulation_stage(const Launch& L, const CertPlan& p, const FinalBufs& f, const ApBufs& b, const int32_t* u,
                        const int32_t* v, const int32_t* xu, const int32_t* xv, const int32_t* d_nx, int32_t* out,
                        int64_t* count_dev, cudaEvent_t* ev) {
  const int32_t V = p.V;
  ap_seed(L, f, b, V, xu, xv, d_nx);
  ApArgs A{f.pre, b.Q, b.PP, b.LAST, V, f.status, b.hooks};
  const bool vec = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
  const int grid = (int)std::max<int64_t>(1, (int64_t)p.G * p.M);
  PassArgs a{A, u, v, 0, p.cache ? std::min(p.warm, p.E) : p.E, b.lab, b.Vpad, p.Vb};
  if (a.t > 0) {
    if (vec)
      launch_pass<0, true>(L, a, grid, p.block, 0);
    else
      launch_pass<0, false>(L, a, grid, p.block, 0);
  }
  if (ev) cudaEventRecord(ev[0], L.stream);
  if (p.cache && p.E > a.t) {
    ap_snapshot(L, f, b, V, p.mode, p.Vb);
    if (ev) cudaEventRecord(ev[1], L.stream);
    a.s = a.t;
    a.t = p.E;
    if (p.mode == 2) {
      const size_t smem = (size_t)(p.Vb / 32 + 4) * 4;
      if (vec)
        launch_pass<2, true>(L, a, grid, p.block, smem);
      else
        launch_pass<2, false>(L, a, grid, p.block, smem);
    } else {
      const size_t smem = (size_t)b.Vpad * 2;
      if (vec)
        launch_pass<1, true>(L, a, grid, p.block, smem);
      else
        launch_pass<1, false>(L, a, grid, p.block, smem);
    }
  } else if (ev) {
    cudaEventRecord(ev[1], L.stream);
  }
  if (ev) cudaEventRecord(ev[2], L.stream);
  ap_finish(L, f, b, V, out, count_dev);
}

size_t fused_bytes(int64_t E) {
  const int64_t nw = E / 32 + 1, nt = nw / 32 + 1;
  return align_up(sizeof(uint32_t) * (size_t)nw, 256) + align_up(sizeof(uint32_t) * (size_t)nt, 256);
}

FusedBufs carve_fused(void* base, int64_t E) {
  FusedBufs b{};
  b.nwords = E / 32 + 1;
  b.ntop = b.nwords / 32 + 1;
  b.keep = static_cast<uint32_t*>(base);
  b.top = reinterpret_cast<uint32_t*>(static_cast<char*>(base) + align_up(sizeof(uint32_t) * (size_t)b.nwords, 256));
  return b;
}

void articulation_fused(const Launch& L, const CertPlan& p, const CertBufs& cb, const FinalBufs& f, const ApBufs& b0,
                        const ApBufs& b1, const FusedBufs& fb, const int32_t* u, const int32_t* v, int32_t* out_points,
                        int32_t* out_bridges, int64_t* count_dev, cudaEvent_t* bev, cudaEvent_t* aev,
                        const ChunkSchedule& chunks) {
  const int32_t V = p.V;
  int32_t* cnt = cb.cnt;
  if (chunks.ev) cudaStreamWaitEvent(L.stream, chunks.ev[0], 0);  // the first chunk holds the prefix
  if (bev) cudaEventRecord(bev[0], L.stream);
  if (aev) cudaEventRecord(aev[0], L.stream);
  cudaMemsetAsync(fb.top, 0, sizeof(uint32_t) * (size_t)fb.ntop, L.stream);
  cert_warm(L, p, cb, u, v);
  if (bev) cudaEventRecord(bev[1], L.stream);
  // T_0: F after the warm-up, rooted and numbered (the bridges of this partial certificate are
  // not needed and go to dscan), then the classes of T_0 u F'
  final_stage(L, f, V, cb.f1u, cb.f1v, cnt + 0, V, cb.f2u, cb.f2v, cnt + 1, V, cb.P1, f.dscan);
  ap_seed(L, f, b0, V, cb.f2u, cb.f2v, cnt + 1);
  if (aev) cudaEventRecord(aev[1], L.stream);
  cert_snapshot(L, p, cb);
  ap_snapshot(L, f, b0, V, 1, 0);
  const int bs = 256;
  ap_combine_kernel<<<grid_of(L, cb.Vpad, bs), bs, 0, L.stream>>>(cb.lab, b0, cb.Vpad, V, f.status);
  *L.launches += 1;
  if (bev) cudaEventRecord(bev[2], L.stream);
  if (aev) cudaEventRecord(aev[2], L.stream);
  const bool vec = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
  const int grid = (int)std::max<int64_t>(1, (int64_t)p.G);
  const Job J{cb.P1, cb.P2, cb.f1u, cb.f1v, cb.f2u, cb.f2v, cnt};
  FusedArgs a{ApArgs{f.pre, b0.Q, b0.PP, b0.LAST, V, f.status, b0.hooks}, J, f.root, fb.keep, fb.top, u, v, 0,
              p.warm, cb.lab, cb.Vpad};
  if (vec)
    launch_fused<false, true>(L, a, grid, p.block);
  else
    launch_fused<false, false>(L, a, grid, p.block);
  const int K = chunks.ev ? chunks.K : 1;
  for (int i = 0; i < K; i++) {  // the rest of the list, chunk by chunk behind a host copy
    if (i > 0) cudaStreamWaitEvent(L.stream, chunks.ev[i], 0);
    a.s = chunks.ev ? std::max<int64_t>(p.warm, chunks.C * i) : p.warm;
    a.t = chunks.ev ? std::min<int64_t>(p.E, chunks.C * (i + 1)) : p.E;
    if (a.t <= a.s) continue;
    if (vec)
      launch_fused<true, true>(L, a, grid, p.block);
    else
      launch_fused<true, false>(L, a, grid, p.block);
  }
  if (bev) {
    cudaEventRecord(bev[3], L.stream);
    cudaEventRecord(bev[4], L.stream);
  }
  if (aev) cudaEventRecord(aev[3], L.stream);
  // the final certificate: its bridges and the final T
  final_stage(L, f, V, cb.f1u, cb.f1v, cnt + 0, V, cb.f2u, cb.f2v, cnt + 1, V, cb.P1,
              out_bridges ? out_bridges : f.dscan);
  if (bev) cudaEventRecord(bev[5], L.stream);
  const int g = grid_of(L, V, bs);
  ap_init_kernel<<<g, bs, 0, L.stream>>>(f, b1, V);
  ap_rename_min_kernel<<<g, bs, 0, L.stream>>>(f, b0, b1, V);
  ap_rename_set_kernel<<<g, bs, 0, L.stream>>>(b0, b1, V, f.status);
  const ApArgs A1{f.pre, b1.Q, b1.PP, b1.LAST, V, f.status, b1.hooks};
  ap_kept_kernel<<<grid_of(L, fb.ntop, bs), bs, 0, L.stream>>>(A1, u, v, fb.keep, fb.top, fb.ntop, p.E);
  *L.launches += 4;
  ap_finish(L, f, b1, V, out_points, count_dev);
  if (bev) cudaEventRecord(bev[6], L.stream);
  if (aev) cudaEventRecord(aev[4], L.stream);
}

}  // namespace bridges
