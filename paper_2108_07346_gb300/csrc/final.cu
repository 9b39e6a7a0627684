// final.cu -- bridges of the final certificate (the stand-in for Alg. 1 on X_0, Sec. 3 end).
//
// Input: a spanning forest T of the certificate (its F edges) and the remaining certificate
// edges X (F' plus anything else, each joining two vertices of one tree).  A tree edge
// (p, y), p the parent of y, is a bridge iff no edge of X has exactly one end in the subtree of
// y.  With vertices numbered in preorder, the subtree of y is the range [pre(y), pre(y) +
// size(y)); let lo(x) / hi(x) be the smallest / largest preorder among the X-neighbours of the
// vertex numbered x.  Then (p, y) is a bridge iff min lo and max hi over the range stay inside
// the range -- the same test as Alg. 1's low[v] > disc[u], evaluated for all tree edges at once
// (Tarjan 1974; Tarjan & Vishkin 1985).
//
// The whole stage is ONE cooperative kernel (every block resident) whose phases are separated
// by a software grid barrier; the work per phase is small (O(V)), so launch overhead, not
// bandwidth, would dominate a kernel-per-phase design, and the barriers (about 1.9 us each)
// dominate the kernel: the phases are arranged to need few of them.
//   * Arc lists: tree edge e gives arcs 2e (tu -> tv) and 2e+1 (tv -> tu), twins by i ^ 1; each
//     arc is pushed on its tail's list with one atomic exchange (no degree count, scan or
//     placement pass).
//   * One tour for the whole forest: every tree gets an entry element (for root r_k, tree k)
//     whose successor is r_k's first arc; the arc that would wrap around to r_k's first arc
//     instead leads to the next tree's entry.  One list ranking then numbers every tree at
//     once, and a vertex's preorder is the number of down arcs and entries before its own down
//     arc (or entry): one scan, no per-tree offsets.  Trees come in the order of their entries:
//     claimed by atomics, or (ordered) by a scan over the roots, in increasing root order.
//   * List ranking by pointer jumping (Wyllie), four hops per round.
//   * lo / hi start neutral and take the X edges by atomics, at the element and at the 32-element
//     chunk level in one pass; each block reduces the chunks to superchunks and builds a sparse
//     table over those in shared memory; a range query reads the partial chunks with 16-byte
//     loads.
//   * Sort of the packed (a<<k | b) keys: each block sorts a slice in shared memory, then ranks
//     its keys against every sorted slice by binary search (up to 16,384 bridges), else an
//     in-kernel stable LSD radix sort.
// Every wait in the barrier is bounded: on expiry the block records BRIDGES_ETIMEDOUT in the
// status word and as the call's count, and leaves the kernel; the others follow at their next
// barrier.
#include <algorithm>

#include "common.cuh"

namespace bridges {

namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 32;           // lo/hi elements per chunk
constexpr int kSuperChunks = 32;     // chunks per superchunk at the smallest superchunk size
static_assert(kSuperChunks == 32, "superchunk indexes are taken by shifts of 5 + sup_log");
constexpr int kMaxSup = 1024;        // superchunks covered by the shared-memory table
constexpr int kSupLevels = 11;       // log2(kMaxSup) + 1
constexpr int64_t kRankMax = 16384;  // up to this many bridges: slice sort + merge ranking
constexpr int kSortSlice = 256;      // keys per sorted slice at most (the small-n sort)
constexpr unsigned kSpinCap = 1u << 22;
constexpr int kHopsLog = 2;  // pointer-jumping hops per round: 4 (8 was slower: longer load chains)
constexpr int kHops = 1 << kHopsLog;
constexpr int kMaxBlocks = 1024;
constexpr int kScanItems = 8;  // consecutive elements per thread in a grid-scan tile
constexpr size_t kSmemTables = sizeof(int32_t) * 2 * kSupLevels * kMaxSup;
constexpr size_t kSmemSort = sizeof(uint64_t) * (kRankMax + kMaxBlocks);

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
  int32_t ordered;  // trees in increasing order of their roots
  unsigned bar_polls;  // polls a barrier waits before it gives up
  int32_t hold_polls;  // > 0: the last block sleeps this many ~100 ns polls before its first barrier
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch, on a counter that only grows within the launch
// (cleared before it): barrier k ends once the counter reaches k * gridDim.  Thread 0 of each
// block counts its barriers in shared memory (*epoch), arrives with one release add that returns
// nothing, and polls the counter with acquire loads -- one round trip to memory per poll and
// none for the arrival (against about 3 us per barrier for an acquire-release add that returns,
// a generation word and its release store).  The block's writes are ordered before its thread 0
// by the block barrier, the release add publishes them, and the acquire that sees the count
// carries everyone's to the block.  Returns false if the wait gave up: the status word then holds
// BRIDGES_ETIMEDOUT (or an earlier error) and the caller must leave the kernel.  Every other
// block then gives up at its next barrier, so the block that would write the count after the
// last phase never gets there; the count is set to that first error here instead, so that a
// caller never reads the count of an earlier call.
__device__ __noinline__ bool grid_barrier(const FinalBufs& f, unsigned polls, unsigned* epoch) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned target = (*epoch += 1) * gridDim.x;
    red_add_release(f.bar_count, 1u);
    if (!bounded_poll([&] { return (int)(ld_acquire(f.bar_count) - target) >= 0; }, polls)) {
      const int32_t first = atomicCAS(f.status, 0, BRIDGES_ETIMEDOUT_CODE);
      *f.count = (int64_t)(first != 0 ? first : BRIDGES_ETIMEDOUT_CODE);
      ok = 0;
    }
  }
  __syncthreads();
  return ok != 0;
}

#define BARRIER()                                         \
  do {                                                    \
    if (!grid_barrier(f, A.bar_polls, &bar_epoch)) return; \
  } while (0)

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }
// This thread's index among all threads with the warps dealt round-robin over the blocks (warp w
// of block b is global warp w * gridDim + b): a loop over fewer items than threads still spreads
// them over every SM, and each warp still takes 32 consecutive items.
__device__ __forceinline__ int64_t gspread() {
  return (((int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) << 5) + (threadIdx.x & 31);
}

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
__device__ bool grid_scan(const FinalBufs& f, unsigned polls, unsigned* epoch, const int32_t* in0, int32_t* out0,
                          const int32_t* in1, int32_t* out1, int64_t n, int32_t* red) {
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
  if (!grid_barrier(f, polls, epoch)) return false;
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

// Prefix / suffix extrema and power-of-two windows within chunks (per element) and within
// superchunks (per chunk); a window never crosses the end of its chunk (superchunk).
struct RangeArrays {
  const int32_t* epl;  // min of lo from the start of the element's chunk to the element
  const int32_t* esl;  // min of lo from the element to the end of its chunk
  const int32_t* eph;  // max of hi, the same two ways
  const int32_t* esh;
  const int32_t* w4l;  // min of lo over the element and the next 3 (7, 15) of its chunk
  const int32_t* w8l;
  const int32_t* w16l;
  const int32_t* w4h;  // max of hi, the same
  const int32_t* w8h;
  const int32_t* w16h;
  const int32_t* cpl;  // min of the chunk minima from the start of the chunk's superchunk
  const int32_t* csl;  // ... to its end
  const int32_t* cph;
  const int32_t* csh;
  const int32_t* cwl;  // window of 2^k chunks (k >= 1) at cwl + (k - 1) * nch: min of the minima
  const int32_t* cwh;  // max of the maxima, the same
  int64_t nch;
  int kc;  // chunk window levels 1..kc exist
};

// min of lo and max of hi over the preorder range [l, r), 0 <= l < r: a range inside one chunk
// from two windows that cover it; otherwise the ends' partial chunks from the element prefix /
// suffix arrays and the whole chunks between them from two chunk windows (inside one
// superchunk) or from the chunk prefix / suffix arrays and the block's sparse table over whole
// superchunks.  A few loads, all independent.
__device__ __forceinline__ void range_minmax(const FinalBufs& f, const RangeArrays& R, const int32_t* tmin,
                                             const int32_t* tmax, int64_t T, int cslog, int64_t l, int64_t r,
                                             int32_t& mn, int32_t& mx) {
  const int64_t ca = l / kChunk, cb = (r - 1) / kChunk;  // chunks of the two ends
  if (ca == cb) {
    const int n = (int)(r - l);
    if (n < 4) {
#pragma unroll
      for (int k = 0; k < 3; k++)
        if (k < n) {
          mn = min(mn, f.lo[l + k]);
          mx = max(mx, f.hi[l + k]);
        }
      return;
    }
    const int k = min(31 - __clz(n), 4);  // windows of 2^k cover [l, r): 2^(k+1) > n, or k = 4 and n <= 32
    const int32_t* wl = k == 2 ? R.w4l : (k == 3 ? R.w8l : R.w16l);
    const int32_t* wh = k == 2 ? R.w4h : (k == 3 ? R.w8h : R.w16h);
    const int64_t w = 1LL << k;
    mn = min(mn, min(wl[l], wl[r - w]));
    mx = max(mx, max(wh[l], wh[r - w]));
    return;
  }
  mn = min(R.esl[l], R.epl[r - 1]);
  mx = max(R.esh[l], R.eph[r - 1]);
  const int64_t c0 = ca + 1, c1 = cb;  // whole chunks [c0, c1)
  if (c0 >= c1) return;
  const int64_t s0 = c0 >> cslog, s1 = (c1 - 1) >> cslog;  // superchunks of the two ends
  if (s0 == s1) {
    const int64_t n = c1 - c0;
    if (n == 1) {
      mn = min(mn, f.cmin[c0]);
      mx = max(mx, f.cmax[c0]);
      return;
    }
    // the n whole chunks lie in one superchunk and the range's end chunks are not among them,
    // so n <= 2^cslog and n < the chunk count; kc is the largest level below both bounds, so two
    // windows of 2^k chunks, k = min(floor(log2 n), kc), cover them (a whole superchunk, n =
    // 2^cslog, takes k = kc = cslog - 1)
    const int k = min(63 - __clzll(n), R.kc);
    const int32_t* wl = R.cwl + (int64_t)(k - 1) * R.nch;
    const int32_t* wh = R.cwh + (int64_t)(k - 1) * R.nch;
    mn = min(mn, min(wl[c0], wl[c1 - (1LL << k)]));
    mx = max(mx, max(wh[c0], wh[c1 - (1LL << k)]));
    return;
  }
  mn = min(mn, min(R.csl[c0], R.cpl[c1 - 1]));
  mx = max(mx, max(R.csh[c0], R.cph[c1 - 1]));
  const int64_t sl = s0 + 1, sr = s1;  // whole superchunks [sl, sr)
  if (sl >= sr) return;
  const int k = 63 - __clzll(sr - sl);
  mn = min(mn, min(tmin[k * T + sl], tmin[k * T + sr - (1LL << k)]));
  mx = max(mx, max(tmax[k * T + sl], tmax[k * T + sr - (1LL << k)]));
}

// Tail and head of tree arc i (tree edge i >> 1 read from the list); false if that edge is not
// a valid forest edge (an id out of range, or a loop).
__device__ __forceinline__ bool arc_ends(const FinArgs& A, int64_t i, int32_t& x, int32_t& y) {
  const int32_t a = A.tu[i >> 1], b = A.tv[i >> 1];
  x = (i & 1) ? b : a;
  y = (i & 1) ? a : b;
  return (uint32_t)a < (uint32_t)A.V && (uint32_t)b < (uint32_t)A.V && a != b;
}

// Number of keys in the sorted s[0, n) below key.
__device__ __forceinline__ int32_t lower_rank(const uint64_t* s, int32_t n, uint64_t key) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (s[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads) final_kernel(FinArgs A) {
  extern __shared__ __align__(16) int32_t sm[];  // superchunk sparse tables, then sort staging
  __shared__ int32_t red[kWarps];
  __shared__ uint32_t wcnt[kWarps][256];
  __shared__ uint32_t run[256];
  __shared__ unsigned bar_epoch;  // grid barriers passed (thread 0's count)
  if (threadIdx.x == 0) bar_epoch = 0;
  const FinalBufs& f = A.f;
  const int32_t V = A.V;
  const bool own = A.P_tree == nullptr;
  int32_t* P = own ? f.P : const_cast<int32_t*>(A.P_tree);
  const int32_t nt = min(*A.d_nt, A.ct);
  const int32_t nx = min(*A.d_nx, A.cx);
  const int64_t na = 2 * (int64_t)nt;  // tree arcs
  const int64_t nchunks = (V + kChunk - 1) / kChunk;

  // a test knob: hold the last block back (a bounded sleep) so that the others' first barrier
  // gives up; never set in normal use
  if (A.hold_polls > 0 && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    for (int32_t i = 0; i < A.hold_polls; i++) __nanosleep(100);

  // 0: clear
  for (int64_t x = gspread(); x < V; x += gstride()) {
    f.head[x] = -1;
    f.rslot[x] = -1;
    f.slo[x] = -1;
    f.lo[x] = INT32_MAX;
    f.hi[x] = INT32_MIN;
    if (own) f.P[x] = (int32_t)x;
  }
  for (int64_t c = gspread(); c < nchunks; c += gstride()) {
    f.cmin[c] = INT32_MAX;
    f.cmax[c] = INT32_MIN;
  }
  if (gtid() == 0) {
    *f.nkeys = 0;
    *f.nroots = 0;
  }
  BARRIER();

  // 1: arc lists (and the forest's union-find when it is ours to build); with a given
  //    union-find also the roots, below
  for (int64_t e = gspread(); e < nt; e += gstride()) {
    const int32_t a = A.tu[e], b = A.tv[e];
    if ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V) {
      set_status(f.status, BRIDGES_ERANGE_CODE);
      continue;
    }
    if (a == b || (own && !uf_link(f.P, a, b))) {  // not a forest
      set_status(f.status, BRIDGES_EINTERNAL_CODE);
      if (a == b) continue;
    }
    f.next[2 * e] = atomicExch(f.head + a, (int32_t)(2 * e));
    f.next[2 * e + 1] = atomicExch(f.head + b, (int32_t)(2 * e + 1));
  }
  if (own) BARRIER();
  // roots (minimum vertex of each tree); every root gets a tree index: claimed in any order, or
  // (ordered) by a scan over the root flags, in increasing root order
  {
    const int lane = threadIdx.x & 31;
    for (int64_t base = gspread() & ~31LL; base < V; base += gstride()) {
      const int64_t x = base + lane;
      bool is_root = false;
      if (x < V) {
        const int32_t r = uf_find_static(P, (int32_t)x);
        f.root[x] = r;
        is_root = r == x;
        if (A.ordered) f.sz[x] = is_root ? 1 : 0;  // scan input
      }
      if (!A.ordered) {
        const unsigned m = __ballot_sync(kFull, is_root);
        if (m) {
          const int leader = __ffs(m) - 1;
          int32_t at = 0;
          if (lane == leader) at = atomicAdd(f.nroots, __popc(m));
          at = __shfl_sync(kFull, at, leader);
          if (is_root) {
            const int32_t k = at + __popc(m & lanemask_lt());
            f.rslot[x] = k;
            f.rlist[k] = (int32_t)x;
          }
        }
      }
    }
  }
  BARRIER();
  if (A.ordered) {
    if (!grid_scan(f, A.bar_polls, &bar_epoch, f.sz, f.rslot, nullptr, nullptr, V, red)) return;
    BARRIER();
    for (int64_t x = gspread(); x < V; x += gstride()) {
      if (f.root[x] == x)
        f.rlist[f.rslot[x]] = (int32_t)x;
      else
        f.rslot[x] = -1;
    }
    if (gtid() == 0) *f.nroots = f.rslot[V];
    BARRIER();
  }
  const int32_t nr = *f.nroots;
  const int64_t N = na + nr;  // elements of the tour: arcs and tree entries
  if (N > 2 * (int64_t)max(V, 1)) {  // only if the tree input was not a forest
    if (gtid() == 0) {
      const int32_t first = atomicCAS(f.status, 0, BRIDGES_EINTERNAL_CODE);
      *f.count = (int64_t)(first != 0 ? first : BRIDGES_EINTERNAL_CODE);
    }
    return;  // every block leaves here
  }

  // 2: successors.  Arc i = (x -> y): the arc after its twin in y's list; at the end of y's list
  //    the first arc of y's list, unless y is a root: then the entry of the next tree (or the
  //    end).  Entry of tree k: its root's first arc (or, for a one-vertex tree, the next entry).
  for (int64_t i = gspread(); i < N; i += gstride()) {
    int32_t s;
    if (i < na) {
      int32_t x, y;
      if (!arc_ends(A, i, x, y)) {
        f.sr[i] = make_int2(-1, 0);
        f.rnk[i] = 0;
        continue;
      }
      s = f.next[i ^ 1];
      if (s < 0) {
        const int32_t k = f.rslot[y];
        s = k < 0 ? f.head[y] : (k + 1 < nr ? (int32_t)(na + k + 1) : -1);
      }
    } else {
      const int32_t k = (int32_t)(i - na);
      s = f.head[f.rlist[k]];
      if (s < 0) s = k + 1 < nr ? (int32_t)(na + k + 1) : -1;
    }
    f.sr[i] = make_int2(s, s < 0 ? 0 : 1);
    f.rnk[i] = s < 0 ? 0 : 1;
  }
  BARRIER();

  // 3: list ranking by pointer jumping (Wyllie), kHops hops per round: after round r every
  //    element knows the element kHops^r places ahead and the rank sum up to it, so
  //    ceil(log_kHops N) rounds (and barriers) suffice; each round reads the previous round's
  //    array only.  Successor and rank share one 8-byte word, so a hop is one random load.  A
  //    thread's first two elements stay in registers from round to round (a round rewrites only
  //    the thread's own elements, so their words need not be read back: one dependent load less
  //    per round), and their hops run side by side (independent load chains).
  const int64_t i0 = gspread(), i1 = i0 + gstride();
  int2 e0 = i0 < N ? f.sr[i0] : make_int2(-1, 0);
  int2 e1 = i1 < N ? f.sr[i1] : make_int2(-1, 0);
  {
    int rounds = 0;
    while ((1LL << (kHopsLog * rounds)) < max(N, (int64_t)1)) rounds++;
    int2* sa = f.sr;
    int2* sb = f.sr2;
    for (int r = 0; r < rounds; r++) {
      const bool last = r == rounds - 1;
      int32_t s0 = e0.x, a0 = e0.y, s1 = e1.x, a1 = e1.y;
#pragma unroll
      for (int h = 0; h < kHops - 1; h++) {
        const int2 y0 = s0 >= 0 ? sa[s0] : make_int2(s0, 0);
        const int2 y1 = s1 >= 0 ? sa[s1] : make_int2(s1, 0);
        a0 += y0.y;
        s0 = y0.x;
        a1 += y1.y;
        s1 = y1.x;
      }
      e0 = make_int2(s0, a0);
      e1 = make_int2(s1, a1);
      if (i0 < N) {
        sb[i0] = e0;
        if (last) f.rnk[i0] = a0;
      }
      if (i1 < N) {
        sb[i1] = e1;
        if (last) f.rnk[i1] = a1;
      }
      for (int64_t i = i1 + gstride(); i < N; i += gstride()) {  // elements beyond two per thread
        int2 x = sa[i];
#pragma unroll
        for (int h = 0; h < kHops - 1; h++) {
          const int2 y = x.x >= 0 ? sa[x.x] : make_int2(x.x, 0);
          x = make_int2(y.x, x.y + y.y);
        }
        sb[i] = x;
        if (last) f.rnk[i] = x.y;
      }
      BARRIER();
      int2* t = sa;
      sa = sb;
      sb = t;
    }
  }

  // 4: tour positions (N - 1 - rank); a tree arc is a down arc (parent -> child) iff it comes
  //    before its twin; entries count as down arcs (they enter their roots)
  for (int64_t i = gspread(); i < N; i += gstride()) {
    const int32_t ri = i == i0 ? e0.y : (i == i1 ? e1.y : f.rnk[i]);
    const int64_t g = N - 1 - ri;
    if (i < na) {
      int32_t x, y;
      if (!arc_ends(A, i, x, y)) continue;
      const int32_t rt = f.rnk[i ^ 1];
      if (g < 0 || g >= N) {  // only if the tree input was not a forest
        set_status(f.status, BRIDGES_EINTERNAL_CODE);
        continue;
      }
      const bool down = ri > rt;
      f.dflag[g] = down ? 1 : 0;
      if (down) {
        f.par[y] = x;
        f.slo[y] = (int32_t)g;  // tour position of y's down arc (slo serves as scratch until the test)
        f.sz[y] = (ri - rt + 1) / 2;
      }
    } else {
      const int32_t k = (int32_t)(i - na);
      if (g < 0 || g >= N) {
        set_status(f.status, BRIDGES_EINTERNAL_CODE);
        continue;
      }
      const int32_t rn = k + 1 < nr ? f.rnk[i + 1] : -1;  // rank of the next entry
      const int32_t root = f.rlist[k];
      f.dflag[g] = 1;
      f.par[root] = -1;
      f.slo[root] = (int32_t)g;
      f.sz[root] = (ri - rn - 1) / 2 + 1;  // the tree's ri - rn - 1 arcs, two per edge
    }
  }
  BARRIER();
  if (!grid_scan(f, A.bar_polls, &bar_epoch, f.dflag, f.dscan, nullptr, nullptr, N, red)) return;
  BARRIER();

  // 5: preorder numbers (the down arcs and entries before the vertex's own tour position), and in
  //    the same pass lo / hi over the extra edges, per element and per chunk, from the same scan.
  //    An edge between the vertices numbered p < q has exactly one end in a range [l, r) iff
  //    either p lies in it and q >= r (seen as hi[p] >= r) or q lies in it and p < l (seen as
  //    lo[q] < l); q can never fall below a range holding p, nor p above a range holding q.  So
  //    the edge lowers lo[q] to p and raises hi[p] to q only: two element and two chunk atomics.
  {
    auto preorder = [&](int32_t x) {
      const int32_t g = f.slo[x];
      const int32_t p = (g >= 0 && g < N) ? f.dscan[g] : -1;
      if (p < 0 || p >= V) {  // only if the tree input was not a forest
        set_status(f.status, BRIDGES_EINTERNAL_CODE);
        return 0;
      }
      return p;
    };
    for (int64_t x = gspread(); x < V; x += gstride()) f.pre[x] = preorder((int32_t)x);
    for (int64_t e = gspread(); e < nx; e += gstride()) {
      const int32_t a = A.xu[e], b = A.xv[e];
      if ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V) {
        set_status(f.status, BRIDGES_ERANGE_CODE);
        continue;
      }
      if (a == b) continue;
      const int32_t pa = preorder(a), pb = preorder(b);
      const int32_t p = min(pa, pb), q = max(pa, pb);
      atomicMin(f.lo + q, p);
      atomicMax(f.hi + p, q);
      atomicMin(f.cmin + q / kChunk, p);
      atomicMax(f.cmax + p / kChunk, q);
    }
  }
  BARRIER();

  // 6b: within each chunk, prefix and suffix minima of lo (maxima of hi) and their minima over
  //     windows of 4, 8 and 16 elements; within each superchunk, the same over the chunk minima
  //     (maxima) with windows of 2, 4, ... chunks: a range query then reads a few entries.  The
  //     windows are clipped at the end of their chunk (superchunk), which no query crosses.  All
  //     go to arrays that are free by now: dflag, dscan, rnk and sr (per element), sr2 (per chunk).
  const int slog = 5 + A.sup_log;  // log2 of the chunks per superchunk
  const int64_t csup = (int64_t)kSuperChunks << A.sup_log;  // chunks per superchunk
  const int64_t nsup = (nchunks + csup - 1) / csup;
  // chunk window levels 1..kc: up to the largest power of two below both csup and nchunks
  int kc = 0;
  while (kc + 1 < slog && (2LL << kc) <= nchunks) kc++;
  int32_t* sr32 = reinterpret_cast<int32_t*>(f.sr);
  int32_t* cp32 = reinterpret_cast<int32_t*>(f.sr2);
  const RangeArrays R{f.dflag,      f.dflag + V,  f.dscan,           f.dscan + V,      f.rnk,
                      sr32,         sr32 + 2 * V, f.rnk + V,         sr32 + V,         sr32 + 3 * V,
                      cp32,         cp32 + nchunks, cp32 + 2 * nchunks, cp32 + 3 * nchunks, cp32 + 4 * nchunks,
                      cp32 + (4 + (int64_t)kc) * nchunks, nchunks, kc};
  {
    int32_t* epl = const_cast<int32_t*>(R.epl);
    int32_t* esl = const_cast<int32_t*>(R.esl);
    int32_t* eph = const_cast<int32_t*>(R.eph);
    int32_t* esh = const_cast<int32_t*>(R.esh);
    int32_t* cpl = const_cast<int32_t*>(R.cpl);
    int32_t* csl = const_cast<int32_t*>(R.csl);
    int32_t* cph = const_cast<int32_t*>(R.cph);
    int32_t* csh = const_cast<int32_t*>(R.csh);
    int32_t* cwl = const_cast<int32_t*>(R.cwl);
    int32_t* cwh = const_cast<int32_t*>(R.cwh);
    int32_t* ssl = cwh + (int64_t)kc * nchunks;  // superchunk minima
    int32_t* ssh = ssl + nsup;                  // superchunk maxima
    const int lane = threadIdx.x & 31;
    const int64_t warp = gspread() >> 5, nwarps = gstride() >> 5;
    for (int64_t w = warp; w < nchunks + nsup; w += nwarps) {
      if (w < nchunks) {
        const int64_t i = w * kChunk + lane;
        const int32_t l0 = i < V ? f.lo[i] : INT32_MAX, h0 = i < V ? f.hi[i] : INT32_MIN;
        int32_t pl = l0, ph = h0, sl = l0, sh = h0;
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t a = __shfl_up_sync(kFull, pl, o), b = __shfl_up_sync(kFull, ph, o);
          const int32_t c = __shfl_down_sync(kFull, sl, o), d = __shfl_down_sync(kFull, sh, o);
          if (lane >= o) {
            pl = min(pl, a);
            ph = max(ph, b);
          }
          if (lane + o < 32) {
            sl = min(sl, c);
            sh = max(sh, d);
          }
        }
        int32_t wl = l0, wh = h0;  // windows [i, i + 2^k) clipped to the chunk, k = 1..4
        int32_t wl4 = 0, wh4 = 0, wl8 = 0, wh8 = 0;
        for (int o = 1; o < 16; o <<= 1) {
          const int32_t a = __shfl_down_sync(kFull, wl, o), b = __shfl_down_sync(kFull, wh, o);
          if (lane + o < 32) {
            wl = min(wl, a);
            wh = max(wh, b);
          }
          if (o == 2) {
            wl4 = wl;
            wh4 = wh;
          } else if (o == 4) {
            wl8 = wl;
            wh8 = wh;
          }
        }
        if (i < V) {
          epl[i] = pl;
          esl[i] = sl;
          eph[i] = ph;
          esh[i] = sh;
          const_cast<int32_t*>(R.w4l)[i] = wl4;
          const_cast<int32_t*>(R.w4h)[i] = wh4;
          const_cast<int32_t*>(R.w8l)[i] = wl8;
          const_cast<int32_t*>(R.w8h)[i] = wh8;
          const_cast<int32_t*>(R.w16l)[i] = wl;
          const_cast<int32_t*>(R.w16h)[i] = wh;
        }
      } else {  // superchunk w - nchunks: its chunks in runs of 32, carried across runs
        const int64_t c0 = (w - nchunks) * csup, c1 = min(nchunks, c0 + csup);
        int32_t carry_l = INT32_MAX, carry_h = INT32_MIN;
        for (int64_t base = c0; base < c1; base += 32) {
          const int64_t c = base + lane;
          int32_t pl = c < c1 ? f.cmin[c] : INT32_MAX, ph = c < c1 ? f.cmax[c] : INT32_MIN;
          for (int o = 1; o < 32; o <<= 1) {
            const int32_t a = __shfl_up_sync(kFull, pl, o), b = __shfl_up_sync(kFull, ph, o);
            if (lane >= o) {
              pl = min(pl, a);
              ph = max(ph, b);
            }
          }
          pl = min(pl, carry_l);
          ph = max(ph, carry_h);
          if (c < c1) {
            cpl[c] = pl;
            cph[c] = ph;
          }
          carry_l = __shfl_sync(kFull, pl, 31);
          carry_h = __shfl_sync(kFull, ph, 31);
        }
        if (lane == 0) {  // the superchunk's own minimum / maximum, for the blocks' sparse tables
          ssl[w - nchunks] = carry_l;
          ssh[w - nchunks] = carry_h;
        }
        carry_l = INT32_MAX;
        carry_h = INT32_MIN;
        for (int64_t top = c1; top > c0; top -= 32) {  // suffixes, from the superchunk's end
          const int64_t c = top - 32 + lane;
          int32_t sl = c >= c0 ? f.cmin[c] : INT32_MAX, sh = c >= c0 ? f.cmax[c] : INT32_MIN;
          for (int o = 1; o < 32; o <<= 1) {
            const int32_t a = __shfl_down_sync(kFull, sl, o), b = __shfl_down_sync(kFull, sh, o);
            if (lane + o < 32) {
              sl = min(sl, a);
              sh = max(sh, b);
            }
          }
          sl = min(sl, carry_l);
          sh = max(sh, carry_h);
          if (c >= c0) {
            csl[c] = sl;
            csh[c] = sh;
          }
          carry_l = __shfl_sync(kFull, sl, 0);
          carry_h = __shfl_sync(kFull, sh, 0);
        }
        // windows of 2^k chunks by doubling, level k from level k - 1 (written by this warp:
        // __syncwarp orders the lanes' writes before the next level's reads)
        for (int k = 1; k <= kc; k++) {
          const int64_t h = 1LL << (k - 1);
          const int32_t* pl = k == 1 ? f.cmin : cwl + (int64_t)(k - 2) * nchunks;
          const int32_t* ph = k == 1 ? f.cmax : cwh + (int64_t)(k - 2) * nchunks;
          int32_t* ol = cwl + (int64_t)(k - 1) * nchunks;
          int32_t* oh = cwh + (int64_t)(k - 1) * nchunks;
          for (int64_t c = c0 + lane; c < c1; c += 32) {
            const bool in = c + h < c1;
            ol[c] = min(pl[c], in ? pl[c + h] : INT32_MAX);
            oh[c] = max(ph[c], in ? ph[c + h] : INT32_MIN);
          }
          __syncwarp();
        }
      }
    }
  }
  BARRIER();

  // 7: per-block superchunk minima and sparse tables over them, then the bridge test
  int levels = 1;
  while ((1LL << levels) <= nsup) levels++;
  const int64_t T = nsup;  // table stride: tmin[k * T + s]
  int32_t* tmin = sm;
  int32_t* tmax = sm + levels * T;
  {
    const int32_t* ssl = R.cwh + (int64_t)kc * nchunks;  // superchunk minima and maxima (6b)
    for (int64_t s = threadIdx.x; s < nsup; s += blockDim.x) {
      tmin[s] = ssl[s];
      tmax[s] = ssl[nsup + s];
    }
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
  for (int64_t base = gspread() & ~31LL; base < V; base += gstride()) {
    const int64_t y = base + (threadIdx.x & 31);
    bool is_bridge = false;
    uint64_t key = 0;
    if (y < V) f.bflag[y] = 0;
    if (y < V && f.par[y] >= 0) {
      const int64_t l = f.pre[y];
      const int64_t r = min((int64_t)V, l + max(f.sz[y], 1));
      int32_t mn = INT32_MAX, mx = INT32_MIN;
      range_minmax(f, R, tmin, tmax, T, slog, l, r, mn, mx);
      f.slo[y] = min(mn, (int32_t)l);
      f.shi[y] = max(mx, (int32_t)(r - 1));
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

  // 8: sort the keys; write (a, b) pairs
  const int32_t cap = max(V - 1, 0);
  const int32_t n = min(*f.nkeys, cap);
  const uint64_t mask = (1ULL << A.kbits) - 1;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  if (n <= kRankMax) {
    // the keys in slices of at most kSortSlice: block b sorts slices b, b + gridDim, ... (each
    // key's rank among the slice's keys, all pairs in shared memory); then every block ranks its
    // share of the keys against every sorted slice by binary search (keys are unique), a warp
    // per key with its lanes over the slices -- few slices keep the searches few
    uint64_t* S = reinterpret_cast<uint64_t*>(sm);
    const int32_t n32 = n;
    const int32_t nsl = (n32 + kSortSlice - 1) / kSortSlice;
    const int32_t ps = nsl > 0 ? (n32 + nsl - 1) / nsl : 0;  // slice length
    for (int32_t b = blockIdx.x; b < nsl; b += gridDim.x) {  // small grids take several slices
      const int32_t s0 = ps * b, m = min(n32, s0 + ps) - s0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) S[i] = f.keys[s0 + i];
      __syncthreads();
      for (int q = threadIdx.x; q < m; q += blockDim.x) {
        const uint64_t key = S[q];
        int32_t r = 0;
        for (int j = 0; j < m; j++) r += S[j] < key;  // every lane reads the same word
        f.keys2[s0 + r] = key;
      }
      __syncthreads();
    }
    BARRIER();
    // slice b at S + b * sp: an odd stride (in 8-byte words) puts the same position of 16
    // consecutive slices in 16 different bank pairs
    const int32_t sp = ps | 1;
    for (int32_t i = threadIdx.x; i < n32; i += blockDim.x) {
      const int32_t b = i / ps;
      S[b * sp + (i - b * ps)] = f.keys2[i];
    }
    __syncthreads();
    const int32_t k0 = min(n32, (int32_t)per * (int32_t)blockIdx.x), k1 = min(n32, k0 + (int32_t)per);
    const int lane = threadIdx.x & 31;
    for (int32_t i = k0 + (threadIdx.x >> 5); i < k1; i += kWarps) {  // a warp per key
      const int32_t bi = i / ps;
      const uint64_t key = S[bi * sp + (i - bi * ps)];
      int32_t c = 0;
      for (int32_t b = lane; b < nsl; b += 32) c += lower_rank(S + b * sp, min(n32, (b + 1) * ps) - b * ps, key);
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
      if (lane == 0) {
        A.out[2 * (int64_t)c] = (int32_t)(key >> A.kbits);
        A.out[2 * (int64_t)c + 1] = (int32_t)(key & mask);
      }
    }
  } else {
    const int passes = (2 * A.kbits + 7) / 8;
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
      if (!grid_scan(f, A.bar_polls, &bar_epoch, f.hist, f.hist, nullptr, nullptr, (int64_t)256 * gridDim.x, red)) return;
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

  // 9: the count, or the first error
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
  s += 4 * 256;                                                           // count, nkeys, barrier, nroots
  s += 13 * align_up(sizeof(int32_t) * (Vs + 1), 256);                    // V-long arrays
  s += 4 * align_up(sizeof(int32_t) * (2 * Vs + 1), 256);                 // 2V-long arrays
  s += 2 * align_up(sizeof(int2) * (2 * Vs + 1), 256);                    // packed successor / rank
  s += 2 * align_up(sizeof(int32_t) * (Vs / kChunk + 2), 256);            // chunk min, max
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
  c += 256;
  f.nroots = reinterpret_cast<int32_t*>(c);
  c += 256;
  int32_t** va[13] = {&f.P,  &f.root, &f.head,  &f.rslot, &f.rlist, &f.pre, &f.sz,
                      &f.par, &f.bflag, &f.slo, &f.shi,   &f.lo,    &f.hi};
  for (auto a : va) {
    *a = reinterpret_cast<int32_t*>(c);
    c += align_up(sizeof(int32_t) * (Vs + 1), 256);
  }
  int32_t** va2[4] = {&f.next, &f.rnk, &f.dflag, &f.dscan};
  for (auto a : va2) {
    *a = reinterpret_cast<int32_t*>(c);
    c += align_up(sizeof(int32_t) * (2 * Vs + 1), 256);
  }
  int2** vp[2] = {&f.sr, &f.sr2};
  for (auto a : vp) {
    *a = reinterpret_cast<int2*>(c);
    c += align_up(sizeof(int2) * (2 * Vs + 1), 256);
  }
  int32_t** vc[2] = {&f.cmin, &f.cmax};
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
                 int64_t cap_extra, const int32_t* P_tree, int32_t* out, bool ordered) {
  // superchunk size: the shared-memory table covers at most kMaxSup superchunks
  const int64_t nch = ceil_div(std::max(V, 1), kChunk);
  int slg = 0;
  while (ceil_div(nch, (int64_t)kSuperChunks << slg) > kMaxSup) slg++;
  const int64_t nsup = ceil_div(nch, (int64_t)kSuperChunks << slg);
  int levels = 1;
  while ((1LL << levels) <= nsup) levels++;
  // shared memory: the superchunk sparse tables, [2][levels][nsup], and later the sort's
  // staging of up to min(V - 1, kRankMax) keys and a slice's ranks
  const size_t tables = sizeof(int32_t) * 2 * (size_t)levels * (size_t)nsup;
  const size_t sort = kSmemSort;
  const size_t smem = std::max(tables, sort);
  // function attributes are per device: set on every call (a host-side call, no launch)
  cudaFuncSetAttribute(final_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)std::max(kSmemTables, kSmemSort));
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, final_kernel, kThreads, smem);
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
  A.sup_log = slg;
  A.ordered = ordered ? 1 : 0;
  A.bar_polls = L.bar_polls > 0 ? L.bar_polls : kSpinCap;
  A.hold_polls = L.hold_polls;
  // one block per SM at most (more blocks make every grid barrier slower than they make the
  // phases faster); small forests take fewer, one thread per element of the tour (2V), which
  // makes every grid barrier cheaper and leaves SMs free for work on other streams (the server)
  const int64_t want = ceil_div(2 * (int64_t)std::max(V, 1), kThreads);
  const int blocks = (int)std::min<int64_t>({(int64_t)kMaxBlocks, (int64_t)std::max(occ, 1) * L.num_sms, want,
                                             (int64_t)L.num_sms});
  cudaMemsetAsync(f.bar_count, 0, sizeof(unsigned), L.stream);
  void* args[] = {&A};
  cudaLaunchCooperativeKernel((void*)final_kernel, dim3(blocks), dim3(kThreads), args, smem, L.stream);
  *L.launches += 1;
}

}  // namespace bridges
