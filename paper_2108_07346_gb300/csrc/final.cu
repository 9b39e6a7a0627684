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
// Steps: tree adjacency (degrees, scan, fill) -> Euler tour successors, cut at each tree's root
// (its minimum vertex) -> list ranking by pointer jumping -> tour positions -> preorder and
// subtree sizes (scan of "down" arcs) -> lo/hi by atomics over X -> sparse tables for range
// min/max -> test -> sort.
#include <algorithm>

#include "common.cuh"

namespace bridges {

namespace {

constexpr int kBs = 256;

__global__ void fin_init_kernel(FinalBufs f, int32_t V, int64_t arcs_cap, bool own_uf) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    f.deg[i] = 0;
    f.cur[i] = 0;
    if (own_uf) f.P[i] = (int32_t)i;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < arcs_cap; i += (int64_t)gridDim.x * blockDim.x)
    f.dflag[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *f.nkeys = 0;
}

// Range-checks the tree edges, builds the forest's union-find (when owned) and counts degrees.
__global__ void fin_tree_kernel(FinalBufs f, int32_t V, const int32_t* tu, const int32_t* tv, const int32_t* d_nt,
                                int32_t cap, bool own_uf) {
  const int32_t nt = min(*d_nt, cap);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = tu[e], b = tv[e];
    if ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V) {
      set_status(f.status, BRIDGES_ERANGE_CODE);
      continue;
    }
    if (own_uf && !uf_link(f.P, a, b)) set_status(f.status, BRIDGES_EINTERNAL_CODE);  // not a forest
    atomicAdd(f.deg + a, 1);
    atomicAdd(f.deg + b, 1);
  }
}

__global__ void fin_fill_kernel(FinalBufs f, int32_t V, const int32_t* tu, const int32_t* tv, const int32_t* d_nt,
                                int32_t cap) {
  const int32_t nt = min(*d_nt, cap);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = tu[e], b = tv[e];
    if ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V) continue;
    int32_t ia = f.off[a] + atomicAdd(f.cur + a, 1);
    int32_t ib = f.off[b] + atomicAdd(f.cur + b, 1);
    f.dst[ia] = b;
    f.dst[ib] = a;
    f.twin[ia] = ib;
    f.twin[ib] = ia;
  }
}

__global__ void fin_root_kernel(FinalBufs f, int32_t V, const int32_t* P) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < V; x += (int64_t)gridDim.x * blockDim.x)
    f.root[x] = uf_find_static(const_cast<int32_t*>(P), (int32_t)x);
}

// Euler tour successor of arc i = (x -> y): the arc after (y -> x) in y's list, cyclically.
__global__ void fin_succ_kernel(FinalBufs f, int32_t V) {
  const int32_t narcs = f.off[V];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < narcs; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t y = f.dst[i], t = f.twin[i];
    f.succ[i] = (t + 1 < f.off[y + 1]) ? t + 1 : f.off[y];
    f.rnk[i] = 1;
  }
}

// Each tree's tour starts at its root's first arc; the arc leading back into it ends the list.
__global__ void fin_cut_kernel(FinalBufs f, int32_t V) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < V; x += (int64_t)gridDim.x * blockDim.x) {
    if (f.root[x] == x && f.deg[x] > 0) {
      int32_t last = f.twin[f.off[x + 1] - 1];
      f.succ[last] = -1;
      f.rnk[last] = 0;
    }
  }
}

// One pointer-jumping step (Wyllie): rank += rank[succ], succ = succ[succ].
__global__ void fin_jump_kernel(const int32_t* succ, const int32_t* rnk, int32_t* succ2, int32_t* rnk2,
                                const int32_t* off, int32_t V) {
  const int32_t narcs = off[V];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < narcs; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t s = succ[i];
    if (s >= 0) {
      rnk2[i] = rnk[i] + rnk[s];
      succ2[i] = succ[s];
    } else {
      rnk2[i] = rnk[i];
      succ2[i] = -1;
    }
  }
}

// Per root: arcs in its tour (aoff values) and vertices in its tree (vbase values).
__global__ void fin_rootvals_kernel(FinalBufs f, int32_t V) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < V; x += (int64_t)gridDim.x * blockDim.x) {
    int32_t L = 0, nv = 0;
    if (f.root[x] == x) {
      L = f.deg[x] > 0 ? f.rnk[f.off[x]] + 1 : 0;
      nv = L / 2 + 1;
    }
    f.aoff[x] = L;
    f.vbase[x] = nv;
  }
}

__device__ __forceinline__ int32_t src_of(const FinalBufs& f, int32_t i) { return f.dst[f.twin[i]]; }

// Tour position of every arc; down arcs (parent -> child) come before their twins.
__global__ void fin_down_kernel(FinalBufs f, int32_t V) {
  const int32_t narcs = f.off[V];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < narcs; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = src_of(f, (int32_t)i);
    const int32_t r = f.root[x];
    const int32_t L = f.rnk[f.off[r]] + 1;
    const int32_t ri = f.rnk[i], rt = f.rnk[f.twin[i]];
    const int32_t g = f.aoff[r] + L - 1 - ri;
    const bool down = ri > rt;
    if (g < 0 || g >= narcs) {  // only if the tree input was not a forest
      set_status(f.status, BRIDGES_EINTERNAL_CODE);
      continue;
    }
    f.dflag[g] = down ? 1 : 0;
    if (down) {
      const int32_t y = f.dst[i];
      f.par[y] = x;
      f.pre[y] = g;  // tour position of y's down arc; turned into a preorder number below
      f.sz[y] = (ri - rt + 1) / 2;
    }
  }
}

__global__ void fin_pre_kernel(FinalBufs f, int32_t V) {
  const int32_t narcs = f.off[V];
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < V; x += (int64_t)gridDim.x * blockDim.x) {
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
  }
}

__global__ void fin_lohi_init_kernel(FinalBufs f, int32_t V) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < V; x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = f.pre[x];
    f.stmin[p] = p;
    f.stmax[p] = p;
  }
}

__global__ void fin_extra_kernel(FinalBufs f, int32_t V, const int32_t* xu, const int32_t* xv, const int32_t* d_nx,
                                 int32_t cap) {
  const int32_t nx = min(*d_nx, cap);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nx; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = xu[e], b = xv[e];
    if ((uint32_t)a >= (uint32_t)V || (uint32_t)b >= (uint32_t)V) {
      set_status(f.status, BRIDGES_ERANGE_CODE);
      continue;
    }
    if (a == b) continue;
    const int32_t pa = f.pre[a], pb = f.pre[b];
    atomicMin(f.stmin + pa, pb);
    atomicMin(f.stmin + pb, pa);
    atomicMax(f.stmax + pa, pb);
    atomicMax(f.stmax + pb, pa);
  }
}

__global__ void fin_sparse_kernel(int32_t* stmin, int32_t* stmax, int32_t V, int k) {
  const int64_t half = 1LL << (k - 1);
  const int64_t n = (int64_t)V - (1LL << k) + 1;
  const int32_t* pmin = stmin + (int64_t)(k - 1) * V;
  const int32_t* pmax = stmax + (int64_t)(k - 1) * V;
  int32_t* qmin = stmin + (int64_t)k * V;
  int32_t* qmax = stmax + (int64_t)k * V;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    qmin[i] = min(pmin[i], pmin[i + half]);
    qmax[i] = max(pmax[i], pmax[i + half]);
  }
}

// Tree edge (par(y), y) is a bridge iff no X edge leaves y's preorder range.
__global__ void fin_test_kernel(FinalBufs f, int32_t V, int kbits) {
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < V; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = base + threadIdx.x;
    bool is_bridge = false;
    uint64_t key = 0;
    if (y < V && f.par[y] >= 0) {
      const int32_t p = f.pre[y];
      const int32_t s = max(1, min(f.sz[y], V - p));
      const int k = 31 - __clz(s);
      const int64_t o = (int64_t)k * V;
      const int32_t mn = min(f.stmin[o + p], f.stmin[o + p + s - (1 << k)]);
      const int32_t mx = max(f.stmax[o + p], f.stmax[o + p + s - (1 << k)]);
      if (mn >= p && mx < p + s) {
        const uint32_t a = (uint32_t)min((int32_t)y, f.par[y]), b = (uint32_t)max((int32_t)y, f.par[y]);
        key = ((uint64_t)a << kbits) | b;
        is_bridge = true;
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
}

__global__ void fin_count_kernel(FinalBufs f, int32_t cap) {
  int32_t st = *f.status;
  const int32_t n = *f.nkeys;
  if (st == 0 && n > cap) st = BRIDGES_EINTERNAL_CODE;  // a forest has at most V-1 edges
  *f.count = st != 0 ? (int64_t)st : (int64_t)n;
}

int grid(const Launch& L, int64_t work) {
  int64_t g = ceil_div(std::max<int64_t>(work, 1), kBs);
  return (int)std::min<int64_t>(g, (int64_t)L.num_sms * 16);
}

int levels_for(int32_t V) {
  int K = 1;
  while ((1LL << K) <= V) K++;
  return K;  // levels 0..K-1, 2^(K-1) <= V
}

int bits_for(int32_t V) {
  int k = 1;
  while ((1LL << k) < (int64_t)V) k++;
  return k;
}

}  // namespace

size_t final_bytes(int32_t V) {
  const size_t Vs = (size_t)std::max(V, 1);
  const size_t K = (size_t)levels_for(std::max(V, 1));
  size_t s = 0;
  s += 256;                                                // count
  s += 256;                                                // nkeys
  s += 10 * align_up(sizeof(int32_t) * (Vs + 1), 256);     // V-long arrays
  s += 7 * align_up(sizeof(int32_t) * (2 * Vs + 1), 256);  // 2V-long arrays
  s += 2 * align_up(sizeof(int32_t) * K * Vs, 256);        // sparse tables
  s += 2 * align_up(sizeof(uint64_t) * Vs, 256);           // keys
  const size_t hist = sort_hist_elems((int64_t)Vs);
  s += align_up(sizeof(uint32_t) * hist, 256);
  const size_t st = std::max(scan_tmp_elems(2 * (int64_t)Vs + 1), scan_tmp_elems((int64_t)hist));
  s += align_up(sizeof(int32_t) * st, 256);
  return s;
}

FinalBufs carve_final(void* base, int32_t V, int32_t* status) {
  FinalBufs f{};
  char* c = static_cast<char*>(base);
  const size_t Vs = (size_t)std::max(V, 1);
  f.K = levels_for(std::max(V, 1));
  f.status = status;
  f.count = reinterpret_cast<int64_t*>(c);
  c += 256;
  f.nkeys = reinterpret_cast<int32_t*>(c);
  c += 256;
  int32_t** va[10] = {&f.P, &f.root, &f.deg, &f.off, &f.cur, &f.aoff, &f.vbase, &f.pre, &f.sz, &f.par};
  for (auto a : va) {
    *a = reinterpret_cast<int32_t*>(c);
    c += align_up(sizeof(int32_t) * (Vs + 1), 256);
  }
  int32_t** va2[7] = {&f.dst, &f.twin, &f.succ, &f.succ2, &f.rnk, &f.dflag, &f.dscan};
  for (auto a : va2) {
    *a = reinterpret_cast<int32_t*>(c);
    c += align_up(sizeof(int32_t) * (2 * Vs + 1), 256);
  }
  // the pointer-jumping double buffer of the ranks reuses dscan, which is free until the
  // preorder scan that follows the ranking
  f.rnk2 = f.dscan;
  f.stmin = reinterpret_cast<int32_t*>(c);
  c += align_up(sizeof(int32_t) * (size_t)f.K * Vs, 256);
  f.stmax = reinterpret_cast<int32_t*>(c);
  c += align_up(sizeof(int32_t) * (size_t)f.K * Vs, 256);
  f.keys = reinterpret_cast<uint64_t*>(c);
  c += align_up(sizeof(uint64_t) * Vs, 256);
  f.keys2 = reinterpret_cast<uint64_t*>(c);
  c += align_up(sizeof(uint64_t) * Vs, 256);
  f.hist_elems = sort_hist_elems((int64_t)Vs);
  f.hist = reinterpret_cast<uint32_t*>(c);
  c += align_up(sizeof(uint32_t) * f.hist_elems, 256);
  f.scan_tmp = reinterpret_cast<int32_t*>(c);
  f.scan_tmp_elems = std::max(scan_tmp_elems(2 * (int64_t)Vs + 1), scan_tmp_elems((int64_t)f.hist_elems));
  return f;
}

void final_stage(const Launch& L, const FinalBufs& f, int32_t V, const int32_t* tu, const int32_t* tv,
                 const int32_t* d_nt, int64_t cap_tree, const int32_t* xu, const int32_t* xv, const int32_t* d_nx,
                 int64_t cap_extra, const int32_t* P_tree, int32_t* out) {
  cudaStream_t s = L.stream;
  const bool own = P_tree == nullptr;
  const int64_t arcs_cap = 2 * (int64_t)std::max(V, 1);
  const int gV = grid(L, V), gA = grid(L, arcs_cap), gT = grid(L, cap_tree), gX = grid(L, cap_extra);
  fin_init_kernel<<<std::max(gV, gA), kBs, 0, s>>>(f, V, arcs_cap + 1, own);
  // at most V tree edges keep the 2V arc arrays in bounds whatever the counts say
  const int32_t ct = (int32_t)std::min<int64_t>(cap_tree, std::max(V, 1));
  const int32_t cx = (int32_t)std::min<int64_t>(cap_extra, INT32_MAX);
  fin_tree_kernel<<<gT, kBs, 0, s>>>(f, V, tu, tv, d_nt, ct, own);
  exclusive_scan_i32(L, f.deg, f.off, V, true, f.scan_tmp);
  fin_fill_kernel<<<gT, kBs, 0, s>>>(f, V, tu, tv, d_nt, ct);
  fin_root_kernel<<<gV, kBs, 0, s>>>(f, V, own ? f.P : P_tree);
  fin_succ_kernel<<<gA, kBs, 0, s>>>(f, V);
  fin_cut_kernel<<<gV, kBs, 0, s>>>(f, V);
  *L.launches += 7;
  // list ranking: ceil(log2(arcs)) pointer-jumping rounds
  int rounds = 0;
  while ((1LL << rounds) < arcs_cap) rounds++;
  int32_t *sa = f.succ, *ra = f.rnk, *sb = f.succ2, *rb = f.rnk2;
  for (int r = 0; r < rounds; r++) {
    fin_jump_kernel<<<gA, kBs, 0, s>>>(sa, ra, sb, rb, f.off, V);
    std::swap(sa, sb);
    std::swap(ra, rb);
  }
  *L.launches += rounds;
  if (ra != f.rnk) {
    cudaMemcpyAsync(f.rnk, ra, sizeof(int32_t) * (size_t)arcs_cap, cudaMemcpyDeviceToDevice, s);
  }
  fin_rootvals_kernel<<<gV, kBs, 0, s>>>(f, V);
  exclusive_scan_i32(L, f.aoff, f.aoff, V, true, f.scan_tmp);
  exclusive_scan_i32(L, f.vbase, f.vbase, V, true, f.scan_tmp);
  fin_down_kernel<<<gA, kBs, 0, s>>>(f, V);
  exclusive_scan_i32(L, f.dflag, f.dscan, arcs_cap, true, f.scan_tmp);
  fin_pre_kernel<<<gV, kBs, 0, s>>>(f, V);
  fin_lohi_init_kernel<<<gV, kBs, 0, s>>>(f, V);
  fin_extra_kernel<<<gX, kBs, 0, s>>>(f, V, xu, xv, d_nx, cx);
  *L.launches += 5;
  for (int k = 1; k < f.K; k++) {
    fin_sparse_kernel<<<gV, kBs, 0, s>>>(f.stmin, f.stmax, V, k);
  }
  *L.launches += f.K - 1;
  const int kbits = bits_for(std::max(V, 1));
  fin_test_kernel<<<gV, kBs, 0, s>>>(f, V, kbits);
  *L.launches += 1;
  // at most V-1 bridges: the sort never writes beyond the caller's 2(V-1) output entries
  sort_pairs(L, f.keys, f.keys2, f.nkeys, std::max<int64_t>(V - 1, 0), 2 * kbits, out, f.hist, f.hist_elems,
             f.scan_tmp);
  fin_count_kernel<<<1, 1, 0, s>>>(f, std::max(V - 1, 0));
  *L.launches += 1;
}

}  // namespace bridges
