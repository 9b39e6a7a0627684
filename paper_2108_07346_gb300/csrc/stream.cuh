// stream.cuh -- the streaming loop shared by the certificate's forest pass, the block pass of
// the articulation-point path and the fused pass that serves both: edges are read once with
// 16-byte loads, tested against a snapshot in shared memory (16-bit labels or a bitmap), and
// only the misses reach a slow path in global memory.  Nothing here is visible through the C
// ABI.
#pragma once

#include "common.cuh"

namespace bridges {

// Fast-path test of one edge against the label snapshot.  Ids are clamped to V, whose label is
// kNoLabel, so out-of-range ids (and unlabelled vertices) fall through to the checked path.
__device__ __forceinline__ uint32_t miss_bit(int32_t a, int32_t b, int32_t V, const uint16_t* slab) {
  const uint16_t la = slab[min((uint32_t)a, (uint32_t)V)];
  const uint16_t lb = slab[min((uint32_t)b, (uint32_t)V)];
  return (la == kNoLabel) | (la != lb);
}

// Fast-path test against a membership bitmap (bit x set: vertex x is in the one F' component the
// bitmap marks).  Ids are clamped to clampv, whose bit is always clear, so out-of-range ids and
// vertices beyond the bitmap fall through to the checked path.
__device__ __forceinline__ uint32_t miss_bit_bm(int32_t a, int32_t b, uint32_t clampv, const uint32_t* sbm) {
  const uint32_t ia = min((uint32_t)a, clampv), ib = min((uint32_t)b, clampv);
  return ((sbm[ia >> 5] >> (ia & 31)) & (sbm[ib >> 5] >> (ib & 31)) & 1u) ^ 1u;
}

// The fast-path test of a stream: MODE 0 none (every edge misses), 1 16-bit labels, 2 bitmap.
template <int MODE>
__device__ __forceinline__ uint32_t miss_of(int32_t a, int32_t b, uint32_t clampv, const void* cache) {
  if (MODE == 1) return miss_bit(a, b, (int32_t)clampv, static_cast<const uint16_t*>(cache));
  if (MODE == 2) return miss_bit_bm(a, b, clampv, static_cast<const uint32_t*>(cache));
  return 1u;
}

// Copies n 16-byte words of a snapshot into shared memory.
__device__ __forceinline__ void load_words(void* dst, const void* src, int64_t n16) {
  const int4* s = static_cast<const int4*>(src);
  int4* d = static_cast<int4*>(dst);
  for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

// Copies a label snapshot (Vpad entries, Vpad a multiple of 8) into shared memory.
__device__ __forceinline__ void load_labels(uint16_t* slab, const uint16_t* glab, int64_t Vpad) {
  const int4* src = reinterpret_cast<const int4*>(glab);
  int4* dst = reinterpret_cast<int4*>(slab);
  for (int64_t i = threadIdx.x; i < Vpad / 8; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// Streams edges [s, t) of (u, v): 16-byte loads when both arrays are 16-byte aligned, U int4
// units (4U edges) in flight per thread, the vector body starting on a 128-byte line of both
// arrays (measured on the large workload: a stream with both label lookups per edge ran in 1.24
// ms from a line boundary against 1.36 ms from a 16-byte boundary inside a line, where every
// warp's 512 bytes of loads touch five lines).  A tile is the block's U int4 units per thread;
// with `members` > 1 the range is shared by that many blocks, block `member` taking tiles member,
// member + members, ... (interleaved tiles keep the blocks' loads in one moving window of the
// list; line-aligned, they stream the forest pass as fast as a slice per block and the fused
// articulation stream 2.5% faster); the scalar head and tail (fewer than 32 and 4 edges) go to
// member 0.  With a snapshot in shared memory (MODE 1: labels, clampv = V; MODE 2: bitmap,
// clampv = its first always-clear bit), each edge costs two
// shared-memory reads; a per-thread bit mask collects the misses and one warp vote per tile
// decides whether any lane must take the slow path.  Loop bounds are block-uniform so every
// lane reaches the votes.
//
// The slow path is the Sink:
//   S.slot(need, a, b, i)         every lane of the warp calls it; `need` marks a live edge (list
//                                 index i) that missed the snapshot (scalar head and tail);
//   S.misses(m, ub, vb, base)     the edges of this thread's tile whose bit is set in m (bit
//                                 4k+c: element 4*(base + k*nt + tid) + c of ub / vb, base an
//                                 int64 unit index); every lane of the warp calls it.
template <int MODE, bool VEC, int U, class Sink>
__device__ __forceinline__ void stream_range(const Sink& S, const int32_t* __restrict__ u,
                                             const int32_t* __restrict__ v, int64_t s, int64_t t, uint32_t clampv,
                                             const void* cache, int64_t member = 0, int64_t members = 1) {
  static_assert(4 * U <= 32, "the miss mask holds 32 edges");
  const int tid = threadIdx.x, nt = blockDim.x;
  int64_t s_al = s, t_al = s;
  if (VEC) {
    // The vector body starts on a 128-byte line of both arrays when they sit at the same offset
    // within a line (else on the 16-byte boundary that VEC guarantees at multiples of 4 edges), so
    // that a warp's 512 bytes of loads cover exactly four lines and a tile never shares a line
    // with another block's tile.
    const int64_t lu = (int64_t)(reinterpret_cast<uintptr_t>(u) & 127);
    const int64_t lv = (int64_t)(reinterpret_cast<uintptr_t>(v) & 127);
    const int64_t q = lu == lv ? 32 : 4;         // edges per alignment unit
    const int64_t off = lu == lv ? lu >> 2 : 0;  // the arrays' offset within a line, in edges
    s_al = min((s + off + q - 1) / q * q - off, t);
    t_al = s_al + ((t - s_al) & ~int64_t(3));
  }
  for (int64_t i0 = s; member == 0 && i0 < s_al; i0 += nt) {  // scalar head
    const int64_t i = i0 + tid;
    const bool valid = i < s_al;
    const int32_t a = valid ? ld_stream1(u + i) : 0, b = valid ? ld_stream1(v + i) : 0;
    S.slot(valid && miss_of<MODE>(a, b, clampv, cache), a, b, i);
  }
  if (VEC) {
    const int32_t* ub = u + s_al;
    const int32_t* vb = v + s_al;
    const int4* u4 = reinterpret_cast<const int4*>(ub);
    const int4* v4 = reinterpret_cast<const int4*>(vb);
    const int64_t nunits = (t_al - s_al) >> 2;
    const int64_t tile = (int64_t)nt * U;
    for (int64_t base = member * tile; base < nunits; base += members * tile) {
      const bool full = base + tile <= nunits;
      int4 ua[U], va[U];
#pragma unroll
      for (int k = 0; k < U; k++) {
        const int64_t idx = base + (int64_t)k * nt + tid;
        if (full || idx < nunits) {
          ua[k] = ld_stream4(u4 + idx);
          va[k] = ld_stream4(v4 + idx);
        } else {
          ua[k] = make_int4(0, 0, 0, 0);
          va[k] = make_int4(0, 0, 0, 0);
        }
      }
      uint32_t m = 0;
#pragma unroll
      for (int k = 0; k < U; k++) {
        const bool valid = full || base + (int64_t)k * nt + tid < nunits;
        const uint32_t mk = miss_of<MODE>(ua[k].x, va[k].x, clampv, cache) |
                            (miss_of<MODE>(ua[k].y, va[k].y, clampv, cache) << 1) |
                            (miss_of<MODE>(ua[k].z, va[k].z, clampv, cache) << 2) |
                            (miss_of<MODE>(ua[k].w, va[k].w, clampv, cache) << 3);
        m |= (valid ? mk : 0u) << (4 * k);
      }
      if (__any_sync(kFull, m != 0)) S.misses(m, ub, vb, base);
    }
  }
  for (int64_t i0 = t_al; member == 0 && i0 < t; i0 += nt) {  // scalar tail
    const int64_t i = i0 + tid;
    const bool valid = i < t;
    const int32_t a = valid ? ld_stream1(u + i) : 0, b = valid ? ld_stream1(v + i) : 0;
    S.slot(valid && miss_of<MODE>(a, b, clampv, cache), a, b, i);
  }
}

// Whether `members` blocks of nt threads share [s, t) in interleaved tiles (true) or take one
// slice each (false): tiles only when every block gets at least 16 of them -- a tile is 4U edges
// per thread, so on a short list tiles would leave blocks idle (a 1 M-edge list has 61 tiles of
// 16,384 edges for 152 blocks).
__device__ __forceinline__ bool use_tiles(int64_t s, int64_t t, int64_t members, int nt, int U) {
  return members > 1 && t - s >= 16 * members * (int64_t)nt * 4 * U;
}

// Edge index of bit `bit` of a miss mask (see stream_range).
__device__ __forceinline__ int64_t miss_edge(int bit, int64_t base) {
  return 4 * (base + (int64_t)(bit >> 2) * blockDim.x + threadIdx.x) + (bit & 3);
}

}  // namespace bridges
