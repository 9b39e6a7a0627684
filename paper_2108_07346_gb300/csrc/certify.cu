// certify.cu -- sparse certificates on the GPU: the partition forest pass and the merge tree.
//
// Sec. 3 splits the edge list into M sets U_i and certifies each (phase 0); Alg. 2 (Sec. 4.B)
// certifies a set as S = F u F', F a spanning forest and F' a spanning forest of the rest.  On
// one GPU a partition ("job") is a contiguous chunk of the edge list processed by G blocks that
// share two concurrent union-finds in global memory (L2-resident): UF1 builds F and UF2 builds
// F'.  Each edge is offered to UF1; if UF1 rejects it (its ends are already joined) it is
// offered to UF2; if UF2 rejects it too, it is dropped.  Offering the rejected edges of F to
// F' edge by edge is Alg. 2 with the edges taken in one arrival order: F ends up a spanning
// forest of U_i and F' a spanning forest of U_i - F.  Concurrency changes which forests come
// out, never their spanning property (see uf_link), and any pair of forests with that property
// is a certificate: it keeps every cut of the input crossed min(cut, 2) times, so it keeps the
// components and the bridges (Sec. 3, end).
//
// Dense partitions become one giant component after about V ln V edges, after which nearly all
// edges are rejected by both forests.  To reject those from shared memory, each job first
// certifies a warm-up prefix of its chunk through the union-finds, then takes a snapshot: a
// 16-bit label per vertex naming its F' component (components with >= 2 vertices, up to 65,535
// of them).  F' components nest inside F components (every F' edge joins two ends F already
// joined), so two vertices with equal labels are joined in both forests and their edge can be
// dropped exactly; connectivity only grows, so a stale snapshot is still sound.  Other edges
// take the union-find path as before.  When 16-bit labels need more shared memory than a block
// has (V above about 113 k), the snapshot is instead a bitmap of the largest F' component, one
// bit per vertex: an edge with both ends in it is dropped the same way.
//
// The merge tree (Sec. 3 phases) certifies the union of f certificates per merge job.  The
// first child's union-finds already encode its own certificate (every edge of a certificate
// wins its forest when offered in order F then F'), so the merge job adopts them in place and
// only offers the other children's edges, appending winners to the first child's lists.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "forest.cuh"
#include "stream.cuh"

namespace bridges {

namespace {

// One edge slot for every lane of a warp.  `need` says whether this lane's edge must go to the
// union-finds; winners are appended warp-aggregated.
__device__ __forceinline__ void settle(const Job& J, bool need, int32_t a, int32_t b, int32_t cap,
                                       int32_t* status) {
  if (!__any_sync(kFull, need)) return;
  int r = need ? offer(J, a, b) : 0;
  warp_append(r == 1, a, b, J.cnt + 0, J.f1u, J.f1v, cap, status);
  warp_append(r == 2, a, b, J.cnt + 1, J.f2u, J.f2v, cap, status);
}

// Range check and self-loop test of an edge that reached the union-find path.
__device__ __forceinline__ bool checked(int32_t a, int32_t b, int32_t V, int32_t* status) {
  if ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V) {
    set_status(status, BRIDGES_ERANGE_CODE);
    return false;
  }
  return a != b;
}

// Scalar slot for the merge and offer kernels: every lane of the warp calls it (valid may be
// false).
__device__ __forceinline__ void scalar_slot(const Job& J, bool valid, int32_t a, int32_t b, int32_t V,
                                            const uint16_t* slab, bool cache, int32_t* status) {
  settle(J, valid && (!cache || miss_bit(a, b, V, slab)) && checked(a, b, V, status), a, b, V, status);
}

// The edges of this thread's current tile whose bit is set in `m` go through the union-finds.
// Kept out of line so the streaming loop stays small; the edges are re-read (they are still in
// L1/L2).
__device__ __noinline__ void offer_misses(const Job& J, uint32_t m, const int32_t* __restrict__ u,
                                          const int32_t* __restrict__ v, int64_t base, int32_t V, int32_t* status) {
  while (__any_sync(kFull, m != 0)) {
    int32_t a = 0, b = 0;
    bool go = false;
    if (m) {
      const int bit = __ffs(m) - 1;
      m &= m - 1;
      const int64_t e = miss_edge(bit, base);
      a = u[e];
      b = v[e];
      go = checked(a, b, V, status);
    }
    const int r = go ? offer(J, a, b) : 0;
    warp_append(r == 1, a, b, J.cnt + 0, J.f1u, J.f1v, V, status);
    warp_append(r == 2, a, b, J.cnt + 1, J.f2u, J.f2v, V, status);
  }
}

// The forest pass's slow path (see stream_range): Alg. 2's two union-finds.
struct ForestSink {
  const Job& J;
  int32_t V;
  int32_t* status;
  __device__ __forceinline__ void slot(bool need, int32_t a, int32_t b, int64_t) const {
    settle(J, need && checked(a, b, V, status), a, b, V, status);
  }
  __device__ __forceinline__ void misses(uint32_t m, const int32_t* ub, const int32_t* vb, int64_t base) const {
    offer_misses(J, m, ub, vb, base, V, status);
  }
};

constexpr int kUnroll = 4;  // int4 units of u (and of v) in flight per thread: 16 edges

struct LeafArgs {
  const int32_t* u;
  const int32_t* v;
  int64_t E;
  int32_t V;
  int32_t M;
  int32_t G;
  int64_t warm;
  int32_t mode;  // 0: warm-up prefix of each chunk, 1: the rest of each chunk
  int32_t Vb;    // bitmap snapshot: vertices it covers
  int64_t r0, r1;  // mode 1: only edges [r0, r1) of the rest (r1 <= r0: all of it)
  CertBufs b;
};

// Forest pass over the partitions: block -> (job j = blockIdx / G, member m = blockIdx % G);
// the job's G members share its chunk [E j / M, E (j+1) / M) (Sec. 3 partition): the warm-up
// prefix in one slice per member, the cached pass in interleaved tiles when the chunk is long
// enough (use_tiles), else in slices too.
template <int MODE, bool VEC>
__global__ void __launch_bounds__(1024, 1) leaf_kernel(LeafArgs A) {
  extern __shared__ __align__(16) uint16_t slab[];
  const int64_t j = blockIdx.x / A.G, m = blockIdx.x % A.G;
  const int64_t lo = A.E * j / A.M, hi = A.E * (j + 1) / A.M;
  const int64_t w = min(A.warm, hi - lo);
  int64_t a = A.mode == 0 ? lo : lo + w;
  int64_t z = A.mode == 0 ? lo + w : hi;
  if (A.mode == 1 && A.r1 > A.r0) {
    a = max(a, A.r0);
    z = max(a, min(z, A.r1));
  }
  if (MODE == 1) load_labels(slab, A.b.lab + j * A.b.Vpad, A.b.Vpad);
  if (MODE == 2) load_words(slab, A.b.lab + j * A.b.Vpad, (A.Vb / 32 + 4) / 4);
  const Job J = job_of(A.b, A.V, j);
  const ForestSink S{J, A.V, A.b.status};
  const uint32_t clampv = MODE == 2 ? (uint32_t)A.Vb : (uint32_t)A.V;
  if (A.mode == 1 && use_tiles(a, z, A.G, blockDim.x, kUnroll)) {
    stream_range<MODE, VEC, kUnroll>(S, A.u, A.v, a, z, clampv, slab, m, A.G);
  } else {
    const int64_t n = z - a;
    const int64_t s = a + n * m / A.G, t = a + n * (m + 1) / A.G;
    stream_range<MODE, VEC, kUnroll>(S, A.u, A.v, s, t, clampv, slab);
  }
}

struct MergeArgs {
  int32_t V;
  int32_t M;
  int32_t f;
  int32_t G;
  int64_t step;  // parent jobs are j * step
  int64_t sub;   // children are parent + k * sub, k = 1 .. f-1
  CertBufs b;
};

// One merge round (Sec. 3 phase q): parent job i adopts its own certificate and offers the
// F and F' edges of children i + k*sub (k = 1..f-1, those < M).
template <bool CACHE>
__global__ void __launch_bounds__(1024) merge_kernel(MergeArgs A) {
  extern __shared__ __align__(16) uint16_t slab[];
  const int64_t jj = blockIdx.x / A.G, m = blockIdx.x % A.G;
  const int64_t parent = jj * A.step;
  if (CACHE) load_labels(slab, A.b.lab + parent * A.b.Vpad, A.b.Vpad);
  Job J = job_of(A.b, A.V, parent);
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 1; k < A.f; k++) {
    int64_t c = parent + k * A.sub;
    if (c >= A.M) break;
    Job C = job_of(A.b, A.V, c);
    for (int which = 0; which < 2; which++) {
      const int32_t n = min(C.cnt[which], A.V);  // capacity of a list slice
      const int32_t* cu = which ? C.f2u : C.f1u;
      const int32_t* cv = which ? C.f2v : C.f1v;
      for (int64_t i0 = m * nt; i0 < n; i0 += (int64_t)A.G * nt) {
        int64_t i = i0 + tid;
        bool valid = i < n;
        int32_t a = valid ? cu[i] : 0, b = valid ? cv[i] : 0;
        scalar_slot(J, valid, a, b, A.V, slab, CACHE, A.b.status);
      }
    }
  }
}

__global__ void init_kernel(CertBufs b, int32_t V, int32_t M) {
  const int64_t total = (int64_t)M * V;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = (int32_t)(i % V);
    b.P1[i] = x;
    b.P2[i] = x;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * (int64_t)M; i += (int64_t)gridDim.x * blockDim.x)
    b.cnt[i] = 0;
}

// ---- label snapshot of F' for jobs j*step, j < njobs ----
// 1) flatten: P2[x] = root(x) (no link can run now, so roots are fixed and the walk is
//    read-only); reset the per-root label ids (tmp) and the job's label counter.
__global__ void snap_flatten_kernel(CertBufs b, int32_t V, int64_t step, int64_t njobs, int32_t tmp_init) {
  const int64_t total = njobs * V;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = (i / V) * step;
    const int32_t x = (int32_t)(i % V);
    int32_t* P2 = b.P2 + j * V;
    int32_t r = x, p = __ldca(P2 + x);
    while (p != r) {
      r = p;
      p = __ldca(P2 + r);
    }
    P2[x] = r;
    b.tmp[j * V + x] = tmp_init;
    if (x == 0) {
      b.nlab[j] = 0;
      b.giant[j] = 0;
    }
  }
}

// 2) every non-root vertex labels itself with its root's id, handing out an id the first time a
//    root is seen.  Lanes of a warp with the same root elect one lane, so a giant component's
//    root entry is read once per warp, not once per vertex.
__global__ void snap_members_kernel(CertBufs b, int32_t V, int64_t step, int64_t njobs) {
  const int64_t total = njobs * V;
  const int lane = threadIdx.x & 31;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < total; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool in = i < total;
    const int64_t j = in ? (i / V) * step : 0;
    const int32_t x = in ? (int32_t)(i % V) : 0;
    const int32_t r = in ? b.P2[j * V + x] : x;
    const bool member = in && r != x;
    // key unique per (job, root); non-members get a key no other lane has
    const long long key = member ? (long long)(j * V + r) : -1LL - lane;
    const unsigned peers = __match_any_sync(kFull, (unsigned long long)key);
    const int leader = __ffs(peers) - 1;
    int32_t id = -1;
    if (member && lane == leader) {
      int32_t* slot = b.tmp + j * V + r;
      id = ld_relaxed(slot);
      if (id < 0) {
        const int32_t fresh = atomicAdd(b.nlab + j, 1);
        const int32_t old = atomicCAS(slot, -1, fresh);
        id = old < 0 ? fresh : old;
      }
    }
    id = __shfl_sync(kFull, id, leader);
    if (member) b.lab[j * b.Vpad + x] = (id >= 0 && id < (int32_t)kNoLabel) ? (uint16_t)id : kNoLabel;
  }
}

// 3) roots take their own id (kNoLabel for singletons); padding entries, including the
//    sentinel at index V, are kNoLabel.
__global__ void snap_roots_kernel(CertBufs b, int32_t V, int64_t step, int64_t njobs) {
  const int64_t total = njobs * b.Vpad;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = (i / b.Vpad) * step;
    const int64_t x = i % b.Vpad;
    if (x < V && b.P2[j * V + x] != x) continue;  // members were labelled above
    uint16_t l = kNoLabel;
    if (x < V) {
      const int32_t id = b.tmp[j * V + x];
      if (id >= 0 && id < (int32_t)kNoLabel) l = (uint16_t)id;
    }
    b.lab[j * b.Vpad + x] = l;
  }
}

// ---- bitmap snapshot (large V): the largest F' component of each job as one bit per vertex ----
// 1) sizes of the F' components (tmp counts members; the flatten set tmp to 0), lanes with the
//    same root adding once per warp
__global__ void bm_count_kernel(CertBufs b, int32_t V, int64_t njobs) {
  const int64_t total = njobs * V;
  const int lane = threadIdx.x & 31;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < total; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool in = i < total;
    const int64_t j = in ? i / V : 0;
    const int32_t x = in ? (int32_t)(i % V) : 0;
    const long long key = in ? j * (long long)V + b.P2[j * V + x] : -1LL - lane;
    const unsigned peers = __match_any_sync(kFull, (unsigned long long)key);
    if (in && lane == __ffs(peers) - 1) atomicAdd(b.tmp + key, __popc(peers));
  }
}

// 2) the largest component of each job: (size << 32 | ~root), ties to the smaller root
__global__ void bm_best_kernel(CertBufs b, int32_t V, int64_t njobs) {
  const int64_t total = njobs * V;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i / V;
    const int32_t x = (int32_t)(i % V);
    if (b.P2[i] != x) continue;
    const int32_t c = b.tmp[i];
    if (c >= 2) atomicMax(b.giant + j, ((unsigned long long)c << 32) | (0xffffffffu - (uint32_t)x));
  }
}

// 3) the bitmap words (in the job's label area): bit x set iff x < min(V, Vb) lies in the largest
//    component; the word past Vb / 32 stays clear (the clamp target of out-of-range ids)
__global__ void bm_write_kernel(CertBufs b, int32_t V, int32_t Vb, int64_t njobs) {
  const int64_t nw = Vb / 32 + 4;  // a multiple of 4 words: the leaf kernel copies 16-byte units
  const int64_t total = njobs * nw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i / nw, w = i % nw;
    const unsigned long long g = b.giant[j];
    const int32_t root = g ? (int32_t)(0xffffffffu - (uint32_t)(g & 0xffffffffu)) : -1;
    uint32_t bits = 0;
    for (int k = 0; k < 32; k++) {
      const int64_t x = w * 32 + k;
      if (root >= 0 && x < V && x < Vb && b.P2[j * V + x] == root) bits |= 1u << k;
    }
    reinterpret_cast<uint32_t*>(b.lab + j * b.Vpad)[w] = bits;
  }
}

// Range check of edges offered to an existing certificate; the offer is skipped on failure.
__global__ void offer_check_kernel(int32_t* status, int32_t V, const int32_t* u, const int32_t* v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if ((uint32_t)u[i] >= (uint32_t)V || (uint32_t)v[i] >= (uint32_t)V) set_status(status, BRIDGES_ERANGE_CODE);
}

// Offers edges to partition 0's union-finds: its certificate becomes one of the union.
__global__ void offer_kernel(CertBufs b, int32_t V, const int32_t* u, const int32_t* v, int64_t n) {
  if (*b.status) return;
  const Job J = job_of(b, V, 0);
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + threadIdx.x;
    const bool valid = i < n;
    const int32_t a = valid ? u[i] : 0, c = valid ? v[i] : 0;
    scalar_slot(J, valid, a, c, V, nullptr, false, b.status);
  }
}

__global__ void export_kernel(CertBufs b, int32_t cap, int32_t* cu, int32_t* cv, uint8_t* ct) {
  const int32_t V = (cap + 2) / 2;  // each forest list holds at most V entries
  const int32_t n1 = min(min(b.cnt[0], V), cap), n2 = min(min(b.cnt[1], V), cap - n1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n1 + n2; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n1) {
      cu[i] = b.f1u[i];
      cv[i] = b.f1v[i];
      ct[i] = 1;
    } else {
      cu[i] = b.f2u[i - n1];
      cv[i] = b.f2v[i - n1];
      ct[i] = 0;
    }
  }
}

int grid_for(const Launch& L, int64_t work, int block) {
  int64_t g = ceil_div(std::max<int64_t>(work, 1), block);
  return (int)std::min<int64_t>(g, (int64_t)L.num_sms * 16);
}

void snapshot(const Launch& L, const CertPlan& p, const CertBufs& b, int64_t step, int64_t njobs) {
  const int bs = 256;
  int g = grid_for(L, njobs * (int64_t)p.V, bs);
  snap_flatten_kernel<<<g, bs, 0, L.stream>>>(b, p.V, step, njobs, -1);
  snap_members_kernel<<<g, bs, 0, L.stream>>>(b, p.V, step, njobs);
  snap_roots_kernel<<<grid_for(L, njobs * b.Vpad, bs), bs, 0, L.stream>>>(b, p.V, step, njobs);
  *L.launches += 3;
}

// The bitmap snapshot of every job (M partitions after the warm-up).
void snapshot_bitmap(const Launch& L, const CertPlan& p, const CertBufs& b) {
  const int bs = 256;
  const int g = grid_for(L, (int64_t)p.M * p.V, bs);
  snap_flatten_kernel<<<g, bs, 0, L.stream>>>(b, p.V, 1, p.M, 0);
  bm_count_kernel<<<g, bs, 0, L.stream>>>(b, p.V, p.M);
  bm_best_kernel<<<g, bs, 0, L.stream>>>(b, p.V, p.M);
  bm_write_kernel<<<grid_for(L, (int64_t)p.M * (p.Vb / 32 + 4), bs), bs, 0, L.stream>>>(b, p.V, p.Vb, p.M);
  *L.launches += 4;
}

template <int MODE, bool VEC>
void launch_leaf(const Launch& L, const CertPlan& p, const LeafArgs& a, size_t smem) {
  auto k = leaf_kernel<MODE, VEC>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // the warm-up launch is contention-bound on the union-finds: it may use fewer threads
  k<<<(unsigned)((int64_t)p.M * p.G), a.mode == 0 ? p.warm_block : p.block, smem, L.stream>>>(a);
  *L.launches += 1;
}

}  // namespace

CertPlan make_plan(int64_t E, int32_t V, int32_t M, int32_t fan_in, int32_t block, int32_t ctas_per_sm, int64_t warm,
                   int num_sms, size_t smem_optin, int32_t warm_block) {
  CertPlan p{};
  p.E = E;
  p.V = V;
  const double lnv = std::log((double)V + 1.0);
  // Automatic M: one partition.  On one GPU every block already shares one memory, so the
  // paper's partitions only add warm-ups and merge rounds (large workload: 1.74 ms at M = 1,
  // 1.87 at 2, 1.94 at 4, 2.22 at 8, 2.94 at 16); M > 1 keeps Sec. 3's scheme for callers that
  // ask for it and for a future sharded form.
  if (M <= 0) M = 1;
  p.M = std::max(1, std::min(M, 65536));
  p.f = fan_in > 1 ? fan_in : std::max(2, std::min(p.M, 16));
  const int64_t Vpad = (int64_t)align_up((size_t)V + 1, 8);  // entry V: the kNoLabel sentinel
  const size_t lab_bytes = (size_t)Vpad * 2;
  const bool labels_fit = lab_bytes + 1024 <= smem_optin;
  // Too many vertices for 16-bit labels: one bit per vertex marks the largest F' component
  // (vertices past the bitmap's reach, if any, always take the union-find path).  The bitmap
  // lives in the job's label area (2 Vpad bytes >= its (Vb / 32 + 4) words).
  const int64_t bm_cap = (((int64_t)(smem_optin - 1024) / 4 - 4) * 32) / 128 * 128;
  p.mode = labels_fit ? 1 : 2;
  p.Vb = (int32_t)std::min<int64_t>(align_up((size_t)std::max(V, 1), 128), std::max<int64_t>(bm_cap, 128));
  const bool fits = labels_fit || bm_cap >= 128;
  int cps = ctas_per_sm;
  if (cps <= 0) {
    const size_t snap_bytes = labels_fit ? lab_bytes : (size_t)(p.Vb / 32 + 4) * 4;
    cps = fits ? (int)std::max<size_t>(1, std::min<size_t>(4, (228 * 1024) / (snap_bytes + 2048))) : 2;
  }
  p.block = block > 0 ? block : (cps <= 2 ? 1024 : 512);
  p.G = (int32_t)std::max<int64_t>(1, ((int64_t)num_sms * cps) / p.M);
  p.warm_block = p.block;
  const int64_t chunk = ceil_div(std::max<int64_t>(E, 1), p.M);
  // Twice the edges after which F' holds a giant component in a dense random partition: at about
  // 0.6 V ln V the snapshot still misses a few vertices whose edges then all take the union-find
  // path (measured on the large workload: 41 k such edges and a 2.3x slower forest pass at
  // 0.6 V ln V, only the 8.3 k pendant-tree edges at 1.2 V ln V).
  if (warm < 0) {
    warm = (int64_t)std::ceil(1.2 * V * lnv) + 4096;
    // graphs too large for labels (usually sparse): their giant F' component forms within a
    // small fraction of the list, while the V ln V prefix of dense graphs could exceed it; a
    // sixteenth was fastest or near it on R-MAT graphs of 2^17 to 2^22 vertices (E/64 to E/4)
    if (!labels_fit) warm = std::min<int64_t>(warm, chunk / 16 + 4096);
  }
  p.cache = fits && warm > 0 && warm < chunk;
  p.warm = p.cache ? warm : chunk + 1;
  // The warm-up prefix is bound by contention on the union-finds' roots, not by bandwidth: a
  // quarter of the stream's threads certify it fastest (large workload: 0.13-0.16 ms at 256
  // threads per block against 0.27 ms at 1024).  Without a snapshot the warm-up launch is the
  // whole pass and keeps the stream's block size.
  if (warm_block >= 32 && warm_block <= 1024 && warm_block % 32 == 0)
    p.warm_block = warm_block;
  else if (p.cache)
    p.warm_block = std::min(p.block, 256);
  return p;
}

size_t cert_bytes(const CertPlan& p) {
  const size_t MV = (size_t)p.M * (size_t)std::max(p.V, 1);
  const size_t Vpad = align_up((size_t)p.V + 1, 8);
  size_t s = 0;
  s += 256;                                         // status
  s += align_up(sizeof(int32_t) * 2 * p.M, 256);    // cnt
  s += align_up(sizeof(int32_t) * p.M, 256);        // nlab
  s += align_up(sizeof(unsigned long long) * p.M, 256);  // giant
  s += 7 * align_up(sizeof(int32_t) * MV, 256);     // P1 P2 f1u f1v f2u f2v tmp
  s += align_up(sizeof(uint16_t) * Vpad * p.M, 256);  // lab
  return s;
}

CertBufs carve_cert(void* base, const CertPlan& p) {
  CertBufs b{};
  char* c = static_cast<char*>(base);
  const size_t MV = (size_t)p.M * (size_t)std::max(p.V, 1);
  const size_t Vpad = align_up((size_t)p.V + 1, 8);
  b.status = reinterpret_cast<int32_t*>(c);
  c += 256;
  b.cnt = reinterpret_cast<int32_t*>(c);
  c += align_up(sizeof(int32_t) * 2 * p.M, 256);
  b.nlab = reinterpret_cast<int32_t*>(c);
  c += align_up(sizeof(int32_t) * p.M, 256);
  b.giant = reinterpret_cast<unsigned long long*>(c);
  c += align_up(sizeof(unsigned long long) * p.M, 256);
  int32_t** arrs[7] = {&b.P1, &b.P2, &b.f1u, &b.f1v, &b.f2u, &b.f2v, &b.tmp};
  for (auto a : arrs) {
    *a = reinterpret_cast<int32_t*>(c);
    c += align_up(sizeof(int32_t) * MV, 256);
  }
  b.lab = reinterpret_cast<uint16_t*>(c);
  b.Vpad = (int64_t)Vpad;
  return b;
}

void cert_init(const Launch& L, const CertPlan& p, const CertBufs& b) {
  init_kernel<<<grid_for(L, (int64_t)p.M * p.V, 256), 256, 0, L.stream>>>(b, p.V, p.M);
  *L.launches += 1;
}

void cert_warm(const Launch& L, const CertPlan& p, const CertBufs& b, const int32_t* u, const int32_t* v) {
  if (p.E == 0) return;
  const LeafArgs a{u, v, p.E, p.V, p.M, p.G, p.warm, 0, p.Vb, 0, 0, b};
  if (((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(v)) & 15) == 0)
    launch_leaf<0, true>(L, p, a, 0);
  else
    launch_leaf<0, false>(L, p, a, 0);
}

void cert_snapshot(const Launch& L, const CertPlan& p, const CertBufs& b) {
  if (p.E == 0 || !p.cache) return;
  if (p.mode == 1)
    snapshot(L, p, b, 1, p.M);
  else
    snapshot_bitmap(L, p, b);
}

void cert_stream(const Launch& L, const CertPlan& p, const CertBufs& b, const int32_t* u, const int32_t* v, int64_t r0,
                 int64_t r1) {
  if (p.E == 0 || !p.cache) return;
  const LeafArgs a{u, v, p.E, p.V, p.M, p.G, p.warm, 1, p.Vb, r0, r1, b};
  const bool vec = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
  if (p.mode == 1) {
    const size_t smem = (size_t)b.Vpad * 2;
    if (vec)
      launch_leaf<1, true>(L, p, a, smem);
    else
      launch_leaf<1, false>(L, p, a, smem);
  } else {
    const size_t smem = (size_t)(p.Vb / 32 + 4) * 4;
    if (vec)
      launch_leaf<2, true>(L, p, a, smem);
    else
      launch_leaf<2, false>(L, p, a, smem);
  }
}

void cert_leaves(const Launch& L, const CertPlan& p, const CertBufs& b, const int32_t* u, const int32_t* v,
                 cudaEvent_t* ev) {
  if (p.E == 0) return;
  if (ev) cudaEventRecord(ev[0], L.stream);
  cert_warm(L, p, b, u, v);
  if (ev) cudaEventRecord(ev[1], L.stream);
  cert_snapshot(L, p, b);
  if (ev) cudaEventRecord(ev[2], L.stream);
  cert_stream(L, p, b, u, v, 0, 0);
  if (ev) cudaEventRecord(ev[3], L.stream);
}

void cert_merge(const Launch& L, const CertPlan& p, const CertBufs& b) {
  const size_t smem = (size_t)b.Vpad * 2;
  const bool fits = smem + 1024 <= L.smem_optin;
  for (int64_t step = 1; step < p.M;) {
    const int64_t sub = step;
    step *= p.f;
    const int64_t njobs = ceil_div(p.M, step);
    // blocks per merge job: enough for (f-1) certificates of up to 2V edges, within the GPU
    const int block = 512;
    int64_t work = (int64_t)(p.f - 1) * 2 * p.V;
    int64_t G = std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, (int64_t)block * 8),
                                                       std::max<int64_t>(1, (int64_t)L.num_sms * 2 / njobs)));
    MergeArgs a{p.V, p.M, p.f, (int32_t)G, step, sub, b};
    const bool cache = fits && work >= 4 * (int64_t)p.V;
    if (cache) {
      snapshot(L, p, b, step, njobs);
      auto k = merge_kernel<true>;
      if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k<<<(unsigned)(njobs * G), block, smem, L.stream>>>(a);
    } else {
      merge_kernel<false><<<(unsigned)(njobs * G), block, 0, L.stream>>>(a);
    }
    *L.launches += 1;
  }
}

void cert_offer(const Launch& L, const CertPlan& p, const CertBufs& b, const int32_t* u, const int32_t* v, int64_t n) {
  if (n <= 0) return;
  const int g = grid_for(L, n, 256);
  offer_check_kernel<<<g, 256, 0, L.stream>>>(b.status, p.V, u, v, n);
  offer_kernel<<<g, 256, 0, L.stream>>>(b, p.V, u, v, n);
  *L.launches += 2;
}

void cert_export(const Launch& L, const CertPlan& p, const CertBufs& b, int32_t* cu, int32_t* cv, uint8_t* ct) {
  const int32_t cap = 2 * std::max(p.V - 1, 0);
  export_kernel<<<grid_for(L, 2 * (int64_t)p.V, 256), 256, 0, L.stream>>>(b, cap, cu, cv, ct);
  *L.launches += 1;
}

}  // namespace bridges
