/*
 * graphgen_dev.cu -- the generator of graphgen.c with its Erdos-Renyi edges drawn on a GPU.
 *
 * INPUTS only: nothing here belongs to the bridge method.  The host builds the graph's layout
 * (gg_layout_make: sizes, structural edges, planted bridges); the device draws the ER pairs of
 * every cluster row, counts them per row, scans the counts and writes every edge at its
 * shuffled position.  Every draw, bijection and position is the host generator's, in integer
 * arithmetic only, so the device graph is bit-identical to gg_generate's (a GPU test checks it).
 * Used where many fresh graphs are needed quickly (the served workload: one new graph per
 * request).
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "graphgen.h"

namespace {

constexpr uint64_t kGolden = 0x9e3779b97f4a7c15ULL;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t ctr) { return mix64(key + ctr * kGolden); }

__device__ __forceinline__ uint64_t perm_apply(const gg_perm& P, uint64_t x) {
  do {
    for (int r = 0; r < 3; r++) {
      x = (x + P.add[r]) & P.mask;
      x = (x * P.mul[r]) & P.mask;
      x ^= x >> P.shift;
    }
  } while (x >= P.n);
  return x;
}

struct Er {
  int64_t Vc;   // core vertices
  int64_t nc;   // clusters
  uint64_t thr;
  uint64_t kER;
};

// first vertex of cluster c, as the host computes it
__device__ __forceinline__ int64_t cl_start(const Er& A, int64_t c) { return (int64_t)(int32_t)((c * A.Vc) / A.nc); }

// cluster of core vertex a: the c with cl_start(c) <= a < cl_start(c + 1)
__device__ __forceinline__ int64_t cluster_of(const Er& A, int64_t a) {
  int64_t c = ((a + 1) * A.nc - 1) / A.Vc;
  while (c + 1 < A.nc && cl_start(A, c + 1) <= a) c++;
  while (c > 0 && cl_start(A, c) > a) c--;
  return c;
}

__device__ __forceinline__ uint64_t er_ctr(int64_t c, int64_t sz, int64_t la, int64_t lb) {
  const uint64_t pidx = (uint64_t)(la * sz - la * (la + 1) / 2 + (lb - la - 1));
  return ((uint64_t)c << 42) ^ pidx;
}

// One warp per core row a: the number of ER edges (a, b), b > a in a's cluster.
__global__ void er_count_kernel(Er A, int64_t* rowcnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < A.Vc; a += nw) {
    const int64_t c = cluster_of(A, a), c0 = cl_start(A, c), sz = cl_start(A, c + 1) - c0, la = a - c0;
    int64_t cnt = 0;
    for (int64_t lb = la + 1 + lane; lb < sz; lb += 32) cnt += draw(A.kER, er_ctr(c, sz, la, lb)) < A.thr;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kFull, cnt, o);
    if (lane == 0) rowcnt[a + 1] = cnt;
  }
}

// Inclusive scan of rowcnt[1..n] in place by one block (rowcnt[0] = 0): row offsets.
__global__ void scan_kernel(int64_t* row, int64_t n) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t lo = 1 + per * t, hi = min(n + 1, lo + per);
  int64_t s = 0;
  for (int64_t i = lo; i < hi; i++) s += row[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t acc = 0;
    for (unsigned k = 0; k < blockDim.x; k++) {
      const int64_t x = part[k];
      part[k] = acc;
      acc += x;
    }
  }
  __syncthreads();
  int64_t acc = part[t];
  for (int64_t i = lo; i < hi; i++) {
    acc += row[i];
    row[i] = acc;
  }
  if (t == 0) row[0] = 0;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

struct Out {
  gg_perm PE;  // edge shuffle
  gg_perm PV;  // vertex relabelling
  int shuffle;
  int relabel;
  int32_t* u;
  int32_t* v;
};

__device__ __forceinline__ void put(const Out& O, int64_t raw, int64_t ra, int64_t rb) {
  const int64_t at = O.shuffle ? (int64_t)perm_apply(O.PE, (uint64_t)raw) : raw;
  O.u[at] = (int32_t)(ra < rb ? ra : rb);
  O.v[at] = (int32_t)(ra < rb ? rb : ra);
}

__device__ __forceinline__ int64_t relabel(const Out& O, int64_t x) {
  return O.relabel ? (int64_t)perm_apply(O.PV, (uint64_t)x) : x;
}

// One warp per core row: the row's ER edges in increasing b take raw positions rowoff[a], ...
__global__ void er_write_kernel(Er A, const int64_t* rowoff, Out O) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < A.Vc; a += nw) {
    const int64_t c = cluster_of(A, a), c0 = cl_start(A, c), sz = cl_start(A, c + 1) - c0, la = a - c0;
    const int64_t ra = relabel(O, a);
    int64_t pos = rowoff[a];
    for (int64_t b0 = la + 1; b0 < sz; b0 += 32) {
      const int64_t lb = b0 + lane;
      const bool hit = lb < sz && draw(A.kER, er_ctr(c, sz, la, lb)) < A.thr;
      const unsigned m = __ballot_sync(kFull, hit);
      if (hit) put(O, pos + __popc(m & lanemask_lt()), ra, relabel(O, c0 + lb));
      pos += __popc(m);
    }
  }
}

// Structural edge i takes raw position n_er + i.
__global__ void struct_write_kernel(const int32_t* su, const int32_t* sv, int64_t n, int64_t n_er, Out O) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    put(O, n_er + i, relabel(O, su[i]), relabel(O, sv[i]));
}

Er er_of(const gg_layout* L) { return Er{L->Vc, L->nc, L->thr, L->kER}; }

// A grid for one warp per row: at most 1,024 blocks of 256 threads, so that a graph's rows never
// queue more blocks than a few waves (work of higher priority sharing the GPU starts between them).
int grid_for(int64_t warps) {
  const int64_t blocks = (warps * 32 + 255) / 256;
  return (int)(blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks));
}

}  // namespace

extern "C" {

/* Count pass: d_rowoff (device, Vc + 1 int64) receives the ER row offsets; *n_er the number of
 * ER edges (the stream is synchronised to read it).  Returns 0, or -1 on a CUDA error. */
int ggd_count(const gg_layout* L, cudaStream_t s, int64_t* d_rowoff, int64_t* n_er) {
  const Er A = er_of(L);
  if (cudaMemsetAsync(d_rowoff, 0, sizeof(int64_t), s) != cudaSuccess) return -1;
  if (A.Vc > 0) {
    er_count_kernel<<<grid_for(A.Vc), 256, 0, s>>>(A, d_rowoff);
    scan_kernel<<<1, 1024, 0, s>>>(d_rowoff, A.Vc);
  }
  if (cudaMemcpyAsync(n_er, d_rowoff + A.Vc, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

/* Write pass: the n_er + n_struct edges of L into (u, v) (device int32 each), given the row
 * offsets of ggd_count and device copies d_su / d_sv of L->su / L->sv.  Enqueue only.  Returns
 * 0, or -1 on a CUDA error. */
int ggd_write(const gg_layout* L, cudaStream_t s, const int64_t* d_rowoff, int64_t n_er, const int32_t* d_su,
              const int32_t* d_sv, int32_t* u, int32_t* v) {
  const Er A = er_of(L);
  Out O{};
  gg_edge_perm(L, n_er + L->n_struct, &O.PE);
  O.PV = L->PV;
  O.shuffle = L->s.shuffle;
  O.relabel = L->s.relabel;
  O.u = u;
  O.v = v;
  if (A.Vc > 0) er_write_kernel<<<grid_for(A.Vc), 256, 0, s>>>(A, d_rowoff, O);
  if (L->n_struct > 0)
    struct_write_kernel<<<(int)((L->n_struct + 255) / 256), 256, 0, s>>>(d_su, d_sv, L->n_struct, n_er, O);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

/* The same for K graphs at once, with one synchronisation: d_rowoff holds the K row-offset
 * arrays one after the other (Vc_k + 1 entries each) followed by K more entries (the counts,
 * gathered for one copy to the host); n_er (host, K) receives the ER edge counts.  Returns 0, or
 * -1 on a CUDA error. */
int ggd_count_many(const gg_layout* const* Ls, int K, cudaStream_t s, int64_t* d_rowoff, int64_t* n_er) {
  int64_t at = 0;
  for (int k = 0; k < K; k++) at += Ls[k]->Vc + 1;
  int64_t* d_counts = d_rowoff + at;
  at = 0;
  for (int k = 0; k < K; k++) {
    const Er A = er_of(Ls[k]);
    if (cudaMemsetAsync(d_rowoff + at, 0, sizeof(int64_t), s) != cudaSuccess) return -1;
    if (A.Vc > 0) {
      er_count_kernel<<<grid_for(A.Vc), 256, 0, s>>>(A, d_rowoff + at);
      scan_kernel<<<1, 1024, 0, s>>>(d_rowoff + at, A.Vc);
    }
    if (cudaMemcpyAsync(d_counts + k, d_rowoff + at + A.Vc, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
      return -1;
    at += A.Vc + 1;
  }
  if (cudaMemcpyAsync(n_er, d_counts, sizeof(int64_t) * (size_t)K, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

/* Writes the K graphs one after the other into (u, v) (graph k at edge offset sum_{j<k} E_j,
 * E_j = n_er[j] + n_struct_j), given ggd_count_many's row offsets and counts; d_struct holds the
 * structural edges on the device, graph after graph, each as its su then its sv (2 n_struct_k
 * int32).  Synchronises the stream before returning.  Returns 0, or -1 on a CUDA error. */
int ggd_write_many(const gg_layout* const* Ls, int K, cudaStream_t s, const int64_t* d_rowoff, const int64_t* n_er,
                   const int32_t* d_struct, int32_t* u, int32_t* v) {
  int64_t at_row = 0, at_edge = 0, at_struct = 0;
  for (int k = 0; k < K; k++) {
    const gg_layout* L = Ls[k];
    const int64_t ns = L->n_struct;
    const int32_t* su = d_struct + at_struct;
    const int32_t* sv = su + ns;
    if (ggd_write(L, s, d_rowoff + at_row, n_er[k], su, sv, u + at_edge, v + at_edge) != 0) return -1;
    at_row += L->Vc + 1;
    at_edge += n_er[k] + ns;
    at_struct += 2 * ns;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // extern "C"
