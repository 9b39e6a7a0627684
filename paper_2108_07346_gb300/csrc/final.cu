// final.cu -- bridges of the final certificate (the stand-in for Alg. 1 on X_0, Sec. 3 end).
//
// Input: a spanning forest T of the certificate (its F edges) and the remaining certificate
// edges X (F' plus anything else, each joining two vertices of one tree).  A tree edge
// (p, y), p the parent of y, is a bridge iff no edge of X has exactly one end in the subtree of
// y.  With vertices numbered in preorder, the subtree of y is the range [pre(y), pre(y) +
// size(y)); let lo(x) / hi(x) be the smallest / largest preorder among x and its X-neighbours.
// Then (p, y) is a bridge iff min lo and max hi over the range stay inside the range -- the same
// test as Alg. 1's low[v] > disc[u], evaluated for all tree edges at once (Tarjan 1974;
// Tarjan & Vishkin 1985).
//
// The whole stage is ONE cooperative kernel (every block resident) whose phases are separated
// by a software grid barrier; the work per phase is small (O(V)), so launch overhead, not
// bandwidth, would dominate a kernel-per-phase design.  Phases:
//   tree degrees -> scan -> adjacency + roots -> Euler-tour successors (cut at each tree's root,
//   its minimum vertex) -> list ranking by pointer jumping -> tour positions -> preorder and
//   subtree sizes (scan of "down" arcs) -> lo/hi (atomics over X) -> range min/max structure
//   (32-element chunks, superchunks of >= 1024 elements, a per-block sparse table over the
//   superchunks in shared memory) -> bridge test -> sort of the packed (a<<k | b) keys (all-pairs
//   rank for up to 16,384 bridges, else an in-kernel stable LSD radix sort).
// Every wait in the barrier is bounded: on expiry the block records BRIDGES_ETIMEDOUT in the
// status word and as the call's count, and leaves the kernel; the others follow at their next
// barrier.
#include <algorithm>

#include "common.cuh"

namespace bridges {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 32;           // lo/hi elements per chunk (one warp)
constexpr int kSuperChunks = 32;     // chunks per superchunk at the smallest superchunk size
constexpr int kMaxSup = 1024;        // superchunks covered by the shared-memory table
constexpr int kSupLevels = 11;       // log2(kMaxSup) + 1
constexpr int64_t kRankMax = 16384;  // up to this many bridges: all-pairs rank sort
constexpr unsigned kSpinCap = 1u << 22;
constexpr int kHopsLog = 2;  // pointer-jumping hops per round: 4 (8 was slower: longer load chains)
constexpr int kHops = 1 << kHopsLog;
constexpr int kMaxBlocks = 1024;
constexpr int kScanItems = 8;  // consecutive elements per thread in a grid-scan tile
constexpr size_t kSmemTables = sizeof(int32_t) * 2 * kSupLevels * kMaxSup;

struct FinArgs {
  FinalBufs f;
  int32_t V;
  const int32_t* tu;
  const int32_t* tv;
  const int32_t* d_nt;
  int32_t ct;  // capacity of the tree list
  const int32_t* xu;
  const int32_t* xv;
  const int32_t* d_nx;
  int32_t cx;             // capacity of the extra list
  const int32_t* P_tree;  // union-find of T, or null: built here in f.P
  int32_t* out;
  int kbits;
  int32_t sup_log;  // chunks per superchunk = kSuperChunks << sup_log
  unsigned bar_polls;  // polls a barrier waits before it gives up
  int32_t hold_polls;  // > 0: the last block sleeps this many ~100 ns polls before its first barrier
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid-wide barrier for a cooperative launch.  Returns false if the wait gave up: the status
// word then holds BRIDGES_ETIMEDOUT (or an earlier error) and the caller must leave the kernel.
// Every other block then gives up at its next barrier, so the block that would write the count
// after the last phase never gets there; the count is set to that first error here instead, so
// that a caller never reads the count of an earlier call.  The block's writes are ordered before
// its thread 0 by the block barrier; thread 0's arrival is an acquire-release add (publishes
// them, and the last arriver acquires everyone's), and the release of the new generation / the
// waiters' acquire loads carry them to every block.  No separate fences: about 1.9 us per
// barrier against 2.4 us with fences around a relaxed add (measured, 152 blocks).
__device__ __noinline__ bool grid_barrier(const FinalBufs& f, unsigned polls) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = ld_acquire(f.bar_gen);
    if (atom_add_acq_rel(f.bar_count, 1u) == gridDim.x - 1) {
      atomicExch(f.bar_count, 0u);  // ordered before the release below
      st_release(f.bar_gen, g + 1);
    } else if (!bounded_poll([&] { return ld_acquire(f.bar_gen) != g; }, polls)) {
      const int32_t first = atomicCAS(f.status, 0, BRIDGES_ETIMEDOUT_CODE);
      *f.count = (int64_t)(first != 0 ? first : BRIDGES_ETIMEDOUT_CODE);
      ok = 0;
    }
  }
  __syncthreads();
  return ok != 0;
}

#define BARRIER()                            \
  do {                                       \
    if (!grid_barrier(f, A.bar_polls)) return; \
  } while (0)

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// Block-wide sum (every thread gets the result).
__device__ __forceinline__ int32_t block_sum(int32_t v, int32_t* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int32_t t = 0;
  for (int w = 0; w < kWarps; w++) t += red[w];
  __syncthreads();
  return t;
}

// Block-wide exclusive scan of one value per thread; returns this thread's prefix, *tot the sum.
__device__ __forceinline__ int32_t block_excl(int32_t v, int32_t* red, int32_t* tot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (lane == 31) red[w] = incl;
  __syncthreads();
  int32_t base = 0, t = 0;
  for (int k = 0; k < kWarps; k++) {
    if (k < w) base += red[k];
    t += red[k];
  }
  __syncthreads();
  *tot = t;
  return base + incl - v;
}

// Exclusive scans of one or two int32 arrays of length n (in place allowed); out[n] = total.
// Block b owns a contiguous range.  Contains one grid barrier; the caller adds the one after.
__device__ bool grid_scan(const FinalBufs& f, unsigned polls, const int32_t* in0, int32_t* out0, const int32_t* in1,
                          int32_t* out1, int64_t n, int32_t* red) {
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = min(n, per * (int64_t)blockIdx.x), hi = min(n, lo + per);
  int32_t s0 = 0, s1 = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    s0 += in0[i];
    if (in1) s1 += in1[i];
  }
  s0 = block_sum(s0, red);
  if (in1) s1 = block_sum(s1, red);
  if (threadIdx.x == 0) {
    f.part[blockIdx.x] = s0;
    if (in1) f.part[gridDim.x + blockIdx.x] = s1;
  }
  if (!grid_barrier(f, polls)) return false;
  int32_t c0 = 0, c1 = 0;
  for (int k = threadIdx.x; k < (int)blockIdx.x; k += blockDim.x) {
    c0 += f.part[k];
    if (in1) c1 += f.part[gridDim.x + k];
  }
  c0 = block_sum(c0, red);
  if (in1) c1 = block_sum(c1, red);
  // tiles of blockDim * kScanItems; each thread scans kScanItems consecutive elements itself,
  // so a block barrier pair serves kScanItems elements per thread, not one
  const int64_t tile = (int64_t)blockDim.x * kScanItems;
  for (int64_t t0 = lo; t0 < hi; t0 += tile) {
    const int64_t i0 = t0 + (int64_t)threadIdx.x * kScanItems;
    int32_t a0[kScanItems], a1[kScanItems];
    int32_t s0 = 0, s1 = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
      const int64_t i = i0 + k;
      a0[k] = i < hi ? in0[i] : 0;
      a1[k] = (in1 && i < hi) ? in1[i] : 0;
      s0 += a0[k];
      s1 += a1[k];
    }
    int32_t tot0 = 0, tot1 = 0;
    int32_t e0 = block_excl(s0, red, &tot0);
    int32_t e1 = in1 ? block_excl(s1, red, &tot1) : 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
      const int64_t i = i0 + k;
      if (i < hi) {
        out0[i] = c0 + e0;
        if (in1) out1[i] = c1 + e1;
      }
      e0 += a0[k];
      e1 += a1[k];
    }
    c0 += tot0;
    c1 += tot1;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {  // the last block's carry is the total
    out0[n] = c0;
    if (in1) out1[n] = c1;
  }
  return true;
}

// min of lo[] and max of hi[] over [l, r) by direct reads.
__device__ __forceinline__ void scan_range(const int32_t* lo, const int32_t* hi, int64_t l, int64_t r, int32_t& mn,
                                           int32_t& mx) {
  for (int64_t i = l; i < r; i++) {
    mn = min(mn, lo[i]);
    mx = max(mx, hi[i]);
  }
}

__global__ void __launch_bounds__(kThreads) final_kernel(FinArgs A) {
  extern __shared__ int32_t sm[];  // superchunk sparse tables: [2][kSupLevels][kMaxSup]
  __shared__ int32_t red[kWarps];
  __shared__ uint32_t wcnt[kWarps][256];
  __shared__ uint32_t run[256];
  const FinalBufs& f = A.f;
  const int32_t V = A.V;
  const bool own = A.P_tree == nullptr;
  int32_t* P = own ? f.P : const_cast<int32_t*>(A.P_tree);
  const int32_t nt = min(*A.d_nt, A.ct);
  const int32_t nx = min(*A.d_nx, A.cx);
  const int64_t narcs_cap = 2 * (int64_t)max(V, 1);

  // a test knob: hold the last block back (a bounded sleep) so that the others' first barrier
  // gives up; never set in normal use
  if (A.hold_polls > 0 && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    for (int32_t i = 0; i < A.hold_polls; i++) __nanosleep(100);

  // 0: clear
  for (int64_t i = gtid(); i < V; i += gstride()) {
    f.deg[i] = 0;
    f.cur[i] = 0;
    if (own) f.P[i] = (int32_t)i;
  }
  for (int64_t i = gtid(); i <= narcs_cap; i += gstride()) f.dflag[i] = 0;
  if (gtid() == 0) *f.nkeys = 0;
  BARRIER();

  // 1: tree edges -> degrees (and the forest's union-find when it is ours to build)
  for (int64_t e = gtid(); e < nt; e += gstride()) {
    const int32_t a = A.tu[e], b = A.tv[e];
    if ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V) {
      set_status(f.status, BRIDGES_ERANGE_CODE);
      continue;
    }
    if (own && !uf_link(f.P, a, b)) set_status(f.status, BRIDGES_EINTERNAL_CODE);  // not a forest
    atomicAdd(f.deg + a, 1);
    atomicAdd(f.deg + b, 1);
  }
  BARRIER();
  if (!grid_scan(f, A.bar_polls, f.deg, f.off, nullptr, nullptr, V, red)) return;
  BARRIER();
  const int32_t narcs = (int32_t)min((int64_t)f.off[V], narcs_cap);

  // 2: adjacency (arc slots, twins) and the root (minimum vertex) of every tree
  for (int64_t e = gtid(); e < nt; e += gstride()) {
    const int32_t a = A.tu[e], b = A.tv[e];
    if ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V) continue;
    const int32_t ia = f.off[a] + atomicAdd(f.cur + a, 1);
    const int32_t ib = f.off[b] + atomicAdd(f.cur + b, 1);
    if (ia >= narcs || ib >= narcs) continue;
    f.dst[ia] = b;
    f.dst[ib] = a;
    f.twin[ia] = ib;
    f.twin[ib] = ia;
  }
  for (int64_t x = gtid(); x < V; x += gstride()) f.root[x] = uf_find_static(P, (int32_t)x);
  BARRIER();

  // 3: Euler-tour successor of arc i = (x -> y): the arc after (y -> x) in y's list, cyclically;
  //    the arc that would wrap around to a root's first arc ends that tree's list
  for (int64_t i = gtid(); i < narcs; i += gstride()) {
    const int32_t y = f.dst[i], t = f.twin[i];
    int32_t s;
    if (t + 1 < f.off[y + 1])
      s = t + 1;
    else
      s = f.root[y] == y ? -1 : f.off[y];
    f.sr[i] = make_int2(s, s < 0 ? 0 : 1);
    f.rnk[i] = s < 0 ? 0 : 1;
  }
  BARRIER();

  // 4: list ranking by pointer jumping (Wyllie), kHops hops per round: after round r every arc
  //    knows the arc kHops^r places ahead and the rank sum up to it, so ceil(log_kHops n) rounds
  //    (and barriers) suffice; each round reads the previous round's array only.  Longer hop
  //    chains trade dependent loads (cheap) for barriers (expensive).  Successor and rank share
  //    one 8-byte word, so a hop is one random load (one sector), not two.
  {
    int rounds = 0;
    while ((1LL << (kHopsLog * rounds)) < (int64_t)max(narcs, 1)) rounds++;
    int2* sa = f.sr;
    int2* sb = f.sr2;
    for (int r = 0; r < rounds; r++) {
      const bool last = r == rounds - 1;
      for (int64_t i = gtid(); i < narcs; i += gstride()) {
        const int2 x = sa[i];
        int32_t s = x.x, acc = x.y;
#pragma unroll
        for (int h = 0; h < kHops - 1 && s >= 0; h++) {
          const int2 y = sa[s];
          acc += y.y;
          s = y.x;
        }
        sb[i] = make_int2(s, acc);
        if (last) f.rnk[i] = acc;
      }
      BARRIER();
      int2* t = sa;
      sa = sb;
      sb = t;
    }
  }

  // 5: per root: arcs of its tour (aoff) and vertices of its tree (vbase); scan both
  for (int64_t x = gtid(); x < V; x += gstride()) {
    int32_t L = 0, nv = 0;
    if (f.root[x] == x) {
      L = f.deg[x] > 0 ? f.rnk[f.off[x]] + 1 : 0;
      nv = L / 2 + 1;
    }
    f.aoff[x] = L;
    f.vbase[x] = nv;
  }
  BARRIER();
  if (!grid_scan(f, A.bar_polls, f.aoff, f.aoff, f.vbase, f.vbase, V, red)) return;
  BARRIER();

  // 6: tour positions; down arcs (parent -> child) come before their twins
  for (int64_t i = gtid(); i < narcs; i += gstride()) {
    const int32_t x = f.dst[f.twin[i]];
    const int32_t r = f.root[x];
    const int32_t L = f.rnk[f.off[r]] + 1;
    const int32_t ri = f.rnk[i], rt = f.rnk[f.twin[i]];
    const int32_t g = f.aoff[r] + L - 1 - ri;
    if (g < 0 || g >= narcs) {  // only if the tree input was not a forest
      set_status(f.status, BRIDGES_EINTERNAL_CODE);
      continue;
    }
    const bool down = ri > rt;
    f.dflag[g] = down ? 1 : 0;
    if (down) {
      const int32_t y = f.dst[i];
      f.par[y] = x;
      f.pre[y] = g;  // tour position of y's down arc; turned into a preorder number below
      f.sz[y] = (ri - rt + 1) / 2;
    }
  }
  BARRIER();
  if (!grid_scan(f, A.bar_polls, f.dflag, f.dscan, nullptr, nullptr, narcs, red)) return;
  BARRIER();

  // 7: preorder numbers and subtree sizes; lo / hi start at the vertex itself
  for (int64_t x = gtid(); x < V; x += gstride()) {
    const int32_t r = f.root[x];
    int32_t p;
    if (r == x) {
      p = f.vbase[x];
      const int32_t L = f.deg[x] > 0 ? f.rnk[f.off[x]] + 1 : 0;
      f.sz[x] = L / 2 + 1;
      f.par[x] = -1;
    } else {
      const int32_t g = f.pre[x], a0 = f.aoff[r];
      p = (g >= 0 && g < narcs && a0 >= 0 && a0 < narcs) ? f.vbase[r] + 1 + f.dscan[g] - f.dscan[a0] : -1;
    }
    if (p < 0 || p >= V) {  // only if the tree input was not a forest
      set_status(f.status, BRIDGES_EINTERNAL_CODE);
      p = 0;
    }
    f.pre[x] = p;
    f.lo[p] = p;
    f.hi[p] = p;
  }
  BARRIER();

  // 8: lo / hi over the extra edges
  for (int64_t e = gtid(); e < nx; e += gstride()) {
    const int32_t a = A.xu[e], b = A.xv[e];
    if ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V) {
      set_status(f.status, BRIDGES_ERANGE_CODE);
      continue;
    }
    if (a == b) continue;
    const int32_t pa = f.pre[a], pb = f.pre[b];
    atomicMin(f.lo + pa, pb);
    atomicMin(f.lo + pb, pa);
    atomicMax(f.hi + pa, pb);
    atomicMax(f.hi + pb, pa);
  }
  BARRIER();

  // 9: chunk (32 elements) and superchunk min / max
  const int64_t nchunks = (V + kChunk - 1) / kChunk;
  const int64_t csup = (int64_t)kSuperChunks << A.sup_log;  // chunks per superchunk
  const int64_t nsup = (nchunks + csup - 1) / csup;
  {
    const int lane = threadIdx.x & 31;
    const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
    for (int64_t c = warp; c < nchunks; c += nwarps) {
      const int64_t i = c * kChunk + lane;
      int32_t mn = i < V ? f.lo[i] : INT32_MAX, mx = i < V ? f.hi[i] : INT32_MIN;
      for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(kFull, mn, o));
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
      }
      if (lane == 0) {
        f.cmin[c] = mn;
        f.cmax[c] = mx;
      }
    }
  }
  BARRIER();
  {  // one warp per superchunk
    const int lane = threadIdx.x & 31;
    const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
    for (int64_t s = warp; s < nsup; s += nwarps) {
      int32_t mn = INT32_MAX, mx = INT32_MIN;
      for (int64_t c = s * csup + lane; c < min(nchunks, (s + 1) * csup); c += 32) {
        mn = min(mn, f.cmin[c]);
        mx = max(mx, f.cmax[c]);
      }
      for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(kFull, mn, o));
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
      }
      if (lane == 0) {
        f.smin[s] = mn;
        f.smax[s] = mx;
      }
    }
  }
  BARRIER();

  // 10: per-block sparse tables over the superchunks, then the bridge test
  int levels = 1;
  while ((1LL << levels) <= nsup) levels++;
  const int64_t T = nsup;  // table stride: tmin[k * T + s]
  int32_t* tmin = sm;
  int32_t* tmax = sm + levels * T;
  for (int64_t s = threadIdx.x; s < nsup; s += blockDim.x) {
    tmin[s] = f.smin[s];
    tmax[s] = f.smax[s];
  }
  __syncthreads();
  for (int k = 1; k < levels; k++) {
    const int64_t half = 1LL << (k - 1);
    for (int64_t s = threadIdx.x; s + (1LL << k) <= nsup; s += blockDim.x) {
      tmin[k * T + s] = min(tmin[(k - 1) * T + s], tmin[(k - 1) * T + s + half]);
      tmax[k * T + s] = max(tmax[(k - 1) * T + s], tmax[(k - 1) * T + s + half]);
    }
    __syncthreads();
  }
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < V; base += gstride()) {
    const int64_t y = base + threadIdx.x;
    bool is_bridge = false;
    uint64_t key = 0;
    if (y < V) f.bflag[y] = 0;
    if (y < V && f.par[y] >= 0) {
      const int64_t l = f.pre[y];
      const int64_t r = min((int64_t)V, l + max(f.sz[y], 1));
      int32_t mn = INT32_MAX, mx = INT32_MIN;
      const int64_t cl = (l + kChunk - 1) / kChunk, cr = r / kChunk;  // whole chunks [cl, cr)
      if (cl >= cr) {
        scan_range(f.lo, f.hi, l, r, mn, mx);
      } else {
        scan_range(f.lo, f.hi, l, cl * kChunk, mn, mx);
        scan_range(f.lo, f.hi, cr * kChunk, r, mn, mx);
        const int64_t sl = (cl + csup - 1) / csup, sr = cr / csup;  // whole superchunks [sl, sr)
        if (sl >= sr) {
          scan_range(f.cmin, f.cmax, cl, cr, mn, mx);
        } else {
          scan_range(f.cmin, f.cmax, cl, sl * csup, mn, mx);
          scan_range(f.cmin, f.cmax, sr * csup, cr, mn, mx);
          const int k = 63 - __clzll(sr - sl);
          mn = min(mn, min(tmin[k * T + sl], tmin[k * T + sr - (1LL << k)]));
          mx = max(mx, max(tmax[k * T + sl], tmax[k * T + sr - (1LL << k)]));
        }
      }
      f.slo[y] = mn;
      f.shi[y] = mx;
      if (mn >= l && mx < r) {
        const uint32_t a = (uint32_t)min((int32_t)y, f.par[y]), b = (uint32_t)max((int32_t)y, f.par[y]);
        key = ((uint64_t)a << A.kbits) | b;
        is_bridge = true;
        f.bflag[y] = 1;
      }
    }
    const unsigned m = __ballot_sync(kFull, is_bridge);
    if (m) {
      const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
      int32_t at = 0;
      if (lane == leader) at = atomicAdd(f.nkeys, __popc(m));
      at = __shfl_sync(kFull, at, leader);
      if (is_bridge) {
        const int32_t i = at + __popc(m & lanemask_lt());
        if (i < V)
          f.keys[i] = key;
        else
          set_status(f.status, BRIDGES_EINTERNAL_CODE);
      }
    }
  }
  BARRIER();

  // 11: sort the keys; write (a, b) pairs
  const int32_t cap = max(V - 1, 0);
  const int32_t n = min(*f.nkeys, cap);
  const uint64_t mask = (1ULL << A.kbits) - 1;
  if (n <= kRankMax) {
    // one warp per key: rank = number of smaller keys (keys are unique), lanes split the scan
    const int lane = threadIdx.x & 31;
    const int64_t warp = gtid() >> 5, nwarps = gstride() >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
      const uint64_t mine = f.keys[i];
      int32_t rank = 0;
      for (int32_t j = lane; j < n; j += 32) rank += f.keys[j] < mine;
      for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(kFull, rank, o);
      if (lane == 0) {
        A.out[2 * (int64_t)rank] = (int32_t)(mine >> A.kbits);
        A.out[2 * (int64_t)rank + 1] = (int32_t)(mine & mask);
      }
    }
  } else {
    const int passes = (2 * A.kbits + 7) / 8;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = min((int64_t)n, per * (int64_t)blockIdx.x), hi = min((int64_t)n, lo + per);
    uint64_t* src = f.keys;
    uint64_t* dst = f.keys2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p = 0; p < passes; p++) {
      const int shift = 8 * p;
      if (threadIdx.x < 256) run[threadIdx.x] = 0;
      __syncthreads();
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&run[(src[i] >> shift) & 255], 1u);
      __syncthreads();
      if (threadIdx.x < 256) f.hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = (int32_t)run[threadIdx.x];
      BARRIER();
      if (!grid_scan(f, A.bar_polls, f.hist, f.hist, nullptr, nullptr, (int64_t)256 * gridDim.x, red)) return;
      BARRIER();
      if (threadIdx.x < 256) {
        run[threadIdx.x] = (uint32_t)f.hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x];
        for (int w = 0; w < kWarps; w++) wcnt[w][threadIdx.x] = 0;
      }
      __syncthreads();
      for (int64_t t0 = lo; t0 < hi; t0 += blockDim.x) {  // stable: chunk, warp, lane = index order
        const int64_t i = t0 + threadIdx.x;
        const bool valid = i < hi;
        const uint64_t key = valid ? src[i] : 0;
        const unsigned d = valid ? (unsigned)((key >> shift) & 255) : 256u + lane;
        const unsigned peers = __match_any_sync(kFull, d);
        const unsigned rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < 256) {
          uint32_t acc = run[threadIdx.x];
          for (int w = 0; w < kWarps; w++) {
            const uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = acc;
            acc += c;
          }
          run[threadIdx.x] = acc;
        }
        __syncthreads();
        if (valid) {
          const uint32_t pos = wcnt[warp][d] + rank;
          if (pos < (uint32_t)n) {
            if (p == passes - 1) {
              A.out[2 * (int64_t)pos] = (int32_t)(key >> A.kbits);
              A.out[2 * (int64_t)pos + 1] = (int32_t)(key & mask);
            } else {
              dst[pos] = key;
            }
          }
        }
        __syncthreads();
        if (threadIdx.x < 256)
          for (int w = 0; w < kWarps; w++) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
      }
      BARRIER();
      uint64_t* t = src;
      src = dst;
      dst = t;
    }
  }

  // 12: the count, or the first error
  if (gtid() == 0) {
    int32_t st = *f.status;
    const int32_t nk = *f.nkeys;
    if (st == 0 && nk > cap) st = BRIDGES_EINTERNAL_CODE;  // a forest has at most V-1 edges
    *f.count = st != 0 ? (int64_t)st : (int64_t)nk;
  }
}

#undef BARRIER

int bits_for(int32_t V) {
  int k = 1;
  while ((1LL << k) < (int64_t)V) k++;
  return k;
}

// ---- 2-edge-connected components: union-find over the certificate minus its bridges ----
__global__ void tecc_init_kernel(FinalBufs f, int32_t V) {
  for (int64_t x = gtid(); x < V; x += gstride()) f.P[x] = (int32_t)x;
  if (gtid() == 0) *f.nkeys = 0;
}

__global__ void tecc_link_kernel(FinalBufs f, int32_t V, const int32_t* xu, const int32_t* xv, const int32_t* d_nx,
                                 int32_t cx) {
  if (*f.status) return;  // the bridge stage failed: labels are left untouched
  for (int64_t y = gtid(); y < V; y += gstride())
    if (f.par[y] >= 0 && !f.bflag[y]) uf_link(f.P, (int32_t)y, f.par[y]);
  const int32_t nx = min(*d_nx, cx);
  for (int64_t e = gtid(); e < nx; e += gstride()) {
    const int32_t a = xu[e], b = xv[e];
    if ((uint32_t)a < (uint32_t)V && (uint32_t)b < (uint32_t)V && a != b) uf_link(f.P, a, b);
  }
}

__global__ void tecc_label_kernel(FinalBufs f, int32_t V, int32_t* labels, int64_t* count) {
  const int32_t st = *f.status;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < V; base += gstride()) {
    const int64_t x = base + threadIdx.x;
    bool root = false;
    if (x < V && !st) {
      const int32_t r = uf_find_static(f.P, (int32_t)x);
      labels[x] = r;
      root = r == x;
    }
    const unsigned m = __ballot_sync(kFull, root);
    if (m && (threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(f.nkeys, __popc(m));
  }
}

__global__ void tecc_count_kernel(FinalBufs f, int64_t* count) {
  const int32_t st = *f.status;
  *count = st ? (int64_t)st : (int64_t)*f.nkeys;
}

}  // namespace

void two_edge_components(const Launch& L, const FinalBufs& f, int32_t V, const int32_t* xu, const int32_t* xv,
                         const int32_t* d_nx, int64_t cap_extra, int32_t* labels, int64_t* count_dev) {
  const int bs = 256;
  const int g = (int)std::min<int64_t>(ceil_div(std::max(V, 1), bs), (int64_t)L.num_sms * 16);
  const int32_t cx = (int32_t)std::min<int64_t>(cap_extra, INT32_MAX);
  tecc_init_kernel<<<g, bs, 0, L.stream>>>(f, V);
  tecc_link_kernel<<<g, bs, 0, L.stream>>>(f, V, xu, xv, d_nx, cx);
  tecc_label_kernel<<<g, bs, 0, L.stream>>>(f, V, labels, count_dev);
  tecc_count_kernel<<<1, 1, 0, L.stream>>>(f, count_dev);
  *L.launches += 4;
}

namespace {
}  // namespace

size_t final_bytes(int32_t V) {
  const size_t Vs = (size_t)std::max(V, 1);
  size_t s = 0;
  s += 3 * 256;                                                           // count, nkeys, barrier
  s += 15 * align_up(sizeof(int32_t) * (Vs + 1), 256);                    // V-long arrays
  s += 5 * align_up(sizeof(int32_t) * (2 * Vs + 1), 256);                 // 2V-long arrays
  s += 2 * align_up(sizeof(int2) * (2 * Vs + 1), 256);                    // packed successor / rank
  s += 4 * align_up(sizeof(int32_t) * (Vs / kChunk + 2), 256);            // chunk / superchunk min, max
  s += 2 * align_up(sizeof(uint64_t) * Vs, 256);                          // keys
  s += align_up(sizeof(int32_t) * (256 * (size_t)kMaxBlocks + 1), 256);  // radix histograms
  s += align_up(sizeof(int32_t) * 2 * kMaxBlocks, 256);                   // scan partials
  return s;
}

FinalBufs carve_final(void* base, int32_t V, int32_t* status) {
  FinalBufs f{};
  char* c = static_cast<char*>(base);
  const size_t Vs = (size_t)std::max(V, 1);
  f.status = status;
  f.count = reinterpret_cast<int64_t*>(c);
  c += 256;
  f.nkeys = reinterpret_cast<int32_t*>(c);
  c += 256;
  f.bar_count = reinterpret_cast<unsigned*>(c);
  f.bar_gen = f.bar_count + 1;
  c += 256;
  int32_t** va[15] = {&f.P,   &f.root, &f.deg, &f.off, &f.cur,   &f.aoff, &f.vbase, &f.pre,
                      &f.sz,  &f.par,  &f.lo,  &f.hi,  &f.bflag, &f.slo,  &f.shi};
  for (auto a : va) {
    *a = reinterpret_cast<int32_t*>(c);
    c += align_up(sizeof(int32_t) * (Vs + 1), 256);
  }
  int32_t** va2[5] = {&f.dst, &f.twin, &f.rnk, &f.dflag, &f.dscan};
  for (auto a : va2) {
    *a = reinterpret_cast<int32_t*>(c);
    c += align_up(sizeof(int32_t) * (2 * Vs + 1), 256);
  }
  int2** vp[2] = {&f.sr, &f.sr2};
  for (auto a : vp) {
    *a = reinterpret_cast<int2*>(c);
    c += align_up(sizeof(int2) * (2 * Vs + 1), 256);
  }
  int32_t** vc[4] = {&f.cmin, &f.cmax, &f.smin, &f.smax};
  for (auto a : vc) {
    *a = reinterpret_cast<int32_t*>(c);
    c += align_up(sizeof(int32_t) * (Vs / kChunk + 2), 256);
  }
  f.keys = reinterpret_cast<uint64_t*>(c);
  c += align_up(sizeof(uint64_t) * Vs, 256);
  f.keys2 = reinterpret_cast<uint64_t*>(c);
  c += align_up(sizeof(uint64_t) * Vs, 256);
  f.hist = reinterpret_cast<int32_t*>(c);
  c += align_up(sizeof(int32_t) * (256 * (size_t)kMaxBlocks + 1), 256);
  f.part = reinterpret_cast<int32_t*>(c);
  return f;
}

void final_stage(const Launch& L, const FinalBufs& f, int32_t V, const int32_t* tu, const int32_t* tv,
                 const int32_t* d_nt, int64_t cap_tree, const int32_t* xu, const int32_t* xv, const int32_t* d_nx,
                 int64_t cap_extra, const int32_t* P_tree, int32_t* out) {
  // shared memory: the superchunk sparse tables actually needed, [2][levels][nsup]
  const int64_t nch = ceil_div(std::max(V, 1), kChunk);
  int slg = 0;
  while (ceil_div(nch, (int64_t)kSuperChunks << slg) > kMaxSup) slg++;
  const int64_t nsup = ceil_div(nch, (int64_t)kSuperChunks << slg);
  int levels = 1;
  while ((1LL << levels) <= nsup) levels++;
  const size_t smem = sizeof(int32_t) * 2 * (size_t)levels * (size_t)nsup;
  // function attributes are per device: set on every call (a host-side call, no launch)
  cudaFuncSetAttribute(final_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTables);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, final_kernel, kThreads, smem);
  // one block per SM: more blocks make every grid barrier slower than they make the phases
  // faster -- except on forests of a million vertices and more, where the phases' dependent
  // random loads need the extra threads
  const int occ_blocks = std::max(1, std::min(occ, V >= (1 << 20) ? 2 : 1));
  FinArgs A{};
  A.f = f;
  A.V = V;
  A.tu = tu;
  A.tv = tv;
  A.d_nt = d_nt;
  A.ct = (int32_t)std::min<int64_t>(cap_tree, std::max(V, 1));  // <= V tree edges keep the arcs in bounds
  A.xu = xu;
  A.xv = xv;
  A.d_nx = d_nx;
  A.cx = (int32_t)std::min<int64_t>(cap_extra, INT32_MAX);
  A.P_tree = P_tree;
  A.out = out;
  A.kbits = bits_for(std::max(V, 1));
  // superchunk size: the shared-memory table covers at most kMaxSup superchunks
  const int64_t nchunks = ceil_div(std::max(V, 1), kChunk);
  int sl = 0;
  while (ceil_div(nchunks, (int64_t)kSuperChunks << sl) > kMaxSup) sl++;
  A.sup_log = sl;
  A.bar_polls = L.bar_polls > 0 ? L.bar_polls : kSpinCap;
  A.hold_polls = L.hold_polls;
  // one block per SM at most; small forests take fewer (a block per 256 vertices), which makes
  // every grid barrier cheaper and leaves SMs free for work on other streams (the server)
  const int64_t want = ceil_div(std::max(V, 1), 256);
  const int blocks = (int)std::min<int64_t>({(int64_t)kMaxBlocks, (int64_t)occ_blocks * L.num_sms, want});
  cudaMemsetAsync(f.bar_count, 0, 2 * sizeof(unsigned), L.stream);
  void* args[] = {&A};
  cudaLaunchCooperativeKernel((void*)final_kernel, dim3(blocks), dim3(kThreads), args, smem, L.stream);
  *L.launches += 1;
}

}  // namespace bridges
