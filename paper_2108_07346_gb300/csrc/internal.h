// internal.h -- host-side plumbing shared by the translation units of libbridges.
// Nothing here is part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#define BRIDGES_EINTERNAL_CODE (-8)
#define BRIDGES_ERANGE_CODE (-2)
#define BRIDGES_ETIMEDOUT_CODE (-5)

namespace bridges {

// Sentinel label: "no class", never equal to another vertex's label.
constexpr uint16_t kNoLabel = 0xffff;

// One launch context: the stream and the context's launch counter.
struct Launch {
  cudaStream_t stream;
  int64_t* launches;
  int num_sms;
  size_t smem_optin;  // max dynamic shared memory per block
  // test knobs of the final stage (bridges_opts.test_barrier_polls / test_hold_polls); zero in
  // normal use
  unsigned bar_polls = 0;  // polls a grid barrier waits before it gives up (0: the default cap)
  int32_t hold_polls = 0;  // > 0: its last block sleeps this many ~100 ns polls before the first barrier
};

// Per-call plan for the certificate stages (Sec. 3): M partitions ("jobs"), G blocks per job,
// merge fan-in f, warm-up edges per partition before the label snapshot.
struct CertPlan {
  int64_t E;
  int32_t V;
  int32_t M;
  int32_t f;
  int32_t G;       // blocks per job in the forest pass
  int32_t block;   // threads per block in the forest pass
  int32_t warm_block;  // threads per block of its warm-up launch
  int64_t warm;    // edges per partition certified before the snapshot (>= partition: no cache)
  bool cache;      // a snapshot is taken after the warm-up
  int32_t mode;    // its form: 1 = 16-bit F' labels (2V bytes fit in shared memory), 2 = bitmap
                   // of the largest F' component (for larger V)
  int32_t Vb;      // mode 2: vertices [0, Vb) covered by the bitmap (a multiple of 128)
};

// Device buffers of the certificate stages, carved from the workspace.  Job j owns the V-long
// slices [j*V, (j+1)*V) of P1, P2, f1u, f1v, f2u, f2v, tmp and lab (lab stride Vpad).
struct CertBufs {
  int32_t* status;  // [1] device status word
  int32_t* cnt;     // [2*M] forest sizes |F|, |F'| per job
  int32_t* nlab;    // [M] labels handed out per job
  unsigned long long* giant;  // [M] bitmap snapshot: (size << 32 | ~root) of the largest F' component
  int32_t* P1;
  int32_t* P2;
  int32_t* f1u;
  int32_t* f1v;
  int32_t* f2u;
  int32_t* f2v;
  int32_t* tmp;
  uint16_t* lab;
  int64_t Vpad;  // stride of lab
};

// Device buffers of the final stage (Euler tour, ranges, test, sort), one cooperative kernel.
struct FinalBufs {
  int32_t* status;
  int64_t* count;  // [1] bridges found (device)
  unsigned* bar_count;  // grid barrier: arrivals (grows within a launch)
  int32_t* nroots;  // [1] trees of the forest (one-vertex trees included)
  int32_t* P;      // [V] union-find over the tree (built by the stage when it owns it)
  int32_t* root;   // [V] root (minimum vertex) of each vertex's tree
  int32_t* head;   // [V] first arc of each vertex's arc list (-1: none)
  int32_t* next;   // [2V] next arc of the same tail (-1: last); tree edge e has arcs 2e, 2e+1
  int32_t* rslot;  // [V+1] index of each root's tree in the tour (-1: not a root)
  int32_t* rlist;  // [V] root of each tree index
  int2* sr;        // [2V] Euler-tour successor and rank, packed (one load per pointer jump)
  int2* sr2;       // [2V] its double buffer
  int32_t* rnk;    // [2V] final ranks
  int32_t* dflag;  // [2V+1] 1 at the tour positions of down arcs and tree entries
  int32_t* dscan;  // [2V+1] its exclusive scan
  int32_t* pre;    // [V]
  int32_t* sz;     // [V]
  int32_t* par;    // [V] parent in the rooted tree (-1 for roots)
  int32_t* bflag;  // [V] 1 if the tree edge (par[y], y) is a bridge
  int32_t* slo;    // [V] by vertex y (non-roots): min of lo over y's subtree range (at most pre y)
  int32_t* shi;    // [V] by vertex y (non-roots): max of hi over y's subtree range (at least its end)
  int32_t* lo;     // [V] indexed by preorder: smallest preorder among the X-neighbours
  int32_t* hi;     // [V] largest preorder among the X-neighbours
  int32_t* cmin;   // [V/32] chunk minima of lo
  int32_t* cmax;   // [V/32] chunk maxima of hi
  uint64_t* keys;   // [V]
  uint64_t* keys2;  // [V]
  int32_t* nkeys;   // [1]
  int32_t* hist;    // radix histograms
  int32_t* part;    // per-block scan partials
};

// Device buffers of the articulation-point stage (blocks.cu), indexed by preorder number unless
// noted.
struct ApBufs {
  int32_t* hooks;  // [1] successful class merges
  int32_t* nlab;   // [1] labels handed out
  int64_t* count;  // [1] articulation points found, or the status
  int32_t* Q;      // class union-find over tree edges (edge (x, parent x) = preorder of x)
  int32_t* PP;     // parent's preorder number, -1 for tree roots
  int32_t* LAST;   // last preorder number of the subtree
  int32_t* vtx;    // vertex of each preorder number
  int32_t* csize;  // tree edges per class (snapshot)
  int32_t* tmp;    // label id per class root (snapshot)
  int32_t* flag;   // by vertex id: 1 if an articulation point
  uint64_t* best;  // largest class containing each vertex: (size << 32 | root), 0 if none
  unsigned long long* giant;  // [1] largest class overall: its key in `best`'s form (bitmap snapshot)
  int32_t* tiles;  // compaction tile counts, then offsets
  uint16_t* lab;   // by vertex id: 16-bit class label (kNoLabel: none); Vpad entries, or the
                  // bitmap snapshot's words (bit x: x lies in the largest class)
  int64_t Vpad;
};

// An overlapped host copy: chunk i (edges [C*i, min(E, C*(i+1))) ) is on the device once ev[i]
// has fired; ev null: the whole list is there already.
struct ChunkSchedule {
  cudaEvent_t* ev;
  int64_t C;
  int K;
};

// Buffers of the fused articulation path (blocks.cu).
struct FusedBufs {
  uint32_t* keep;  // [nwords] one mark per edge of the list: walked on the final T
  uint32_t* top;   // [ntop] one bit per word of keep that the current call marked
  int64_t nwords;  // E / 32 + 1
  int64_t ntop;    // nwords / 32 + 1
};

// ---- certify.cu ----
void cert_init(const Launch& L, const CertPlan& p, const CertBufs& b);
// Leaf certificates of the M partitions of (u, v) (Sec. 3 phase 0, Alg. 2 per partition).
void cert_leaves(const Launch& L, const CertPlan& p, const CertBufs& b, const int32_t* u, const int32_t* v,
                 cudaEvent_t* ev /* 4 events or null */);
// The same in its three steps, for callers that interleave them with copies: the warm-up prefix
// of every partition (edges [0, warm) of each chunk must be present), the snapshot, and the
// rest of every chunk restricted to edges [r0, r1) (r1 <= r0: all of it; no-ops without a
// snapshot, when the warm-up covered everything).
void cert_warm(const Launch& L, const CertPlan& p, const CertBufs& b, const int32_t* u, const int32_t* v);
void cert_snapshot(const Launch& L, const CertPlan& p, const CertBufs& b);
void cert_stream(const Launch& L, const CertPlan& p, const CertBufs& b, const int32_t* u, const int32_t* v, int64_t r0,
                 int64_t r1);
// Merge tree (Sec. 3 phases): fan-in f until one certificate remains in job 0.
void cert_merge(const Launch& L, const CertPlan& p, const CertBufs& b);
// Plan for (E, V, M) on this device.
CertPlan make_plan(int64_t E, int32_t V, int32_t M, int32_t fan_in, int32_t block, int32_t ctas_per_sm,
                   int64_t warm, int num_sms, size_t smem_optin, int32_t warm_block = 0);
// Workspace bytes of the certificate stage.
size_t cert_bytes(const CertPlan& p);
CertBufs carve_cert(void* base, const CertPlan& p);
// Copies job 0's certificate into caller arrays (u, v, tree flag), count on device in cnt[0..1].
void cert_export(const Launch& L, const CertPlan& p, const CertBufs& b, int32_t* cu, int32_t* cv, uint8_t* ctree);

// ---- final.cu ----
size_t final_bytes(int32_t V);
FinalBufs carve_final(void* base, int32_t V, int32_t* status);
// 2-edge-connected components after final_stage: labels[x] = minimum vertex of x's component
// (the components of T u X minus its bridges); count_dev receives their number.
void two_edge_components(const Launch& L, const FinalBufs& fb, int32_t V, const int32_t* xu, const int32_t* xv,
                         const int32_t* d_nx, int64_t cap_extra, int32_t* labels, int64_t* count_dev);
// Offers n extra edges to partition 0's union-finds (its certificate grows to a certificate of
// the union).  Ids are range-checked first; on ERANGE nothing is changed.
void cert_offer(const Launch& L, const CertPlan& p, const CertBufs& b, const int32_t* u, const int32_t* v, int64_t n);
// Bridges of T u X (T a spanning forest of every tree it touches, X edges inside trees).
// Counts on device.  P_tree: union-find of T (roots = minimum vertex), or null to build it.
// ordered: trees take consecutive preorder ranges in increasing order of their roots (otherwise
// in an arbitrary order).
void final_stage(const Launch& L, const FinalBufs& fb, int32_t V, const int32_t* tu, const int32_t* tv,
                 const int32_t* d_ntree, int64_t cap_tree, const int32_t* xu, const int32_t* xv,
                 const int32_t* d_nextra, int64_t cap_extra, const int32_t* P_tree, int32_t* out,
                 bool ordered = false);

// ---- blocks.cu ----
size_t ap_bytes(int32_t V);
ApBufs carve_ap(void* base, int32_t V);
// Articulation points of (u, v) after the bridge path: f holds the final stage's rooted forest
// T (pre, par, sz) and (xu, xv, *d_nx) the certificate's non-tree edges.  Streams the edge list
// once more (warm-up of p.warm edges, snapshot in p.mode's form -- 16-bit labels, or for larger
// V a bitmap of vertices [0, p.Vb) -- then the rest) with p's grid (M = 1 plan);
// writes the sorted points to out and their number (or the status) to *count_dev.  ev: three
// events recorded after the warm-up, the snapshot and the stream (or null).
void articulation_stage(const Launch& L, const CertPlan& p, const FinalBufs& f, const ApBufs& b, const int32_t* u,
                        const int32_t* v, const int32_t* xu, const int32_t* xv, const int32_t* d_nx, int32_t* out,
                        int64_t* count_dev, cudaEvent_t* ev);

// Articulation points and bridges with one read of the list (the fused path; single partition
// with a 16-bit label snapshot, p): the forest pass's warm-up, T_0 = F rooted and seeded, the
// combined snapshot, one stream for the certificate and the classes, the final stage (bridges
// to out_bridges, or scratch when null), the classes renamed onto the final T and the marked
// edges walked, the points to out_points and their number (or the status) to *count_dev.
// bev: the bridge path's 8 stage events, aev: the block pass's 5 (either may be null).  With a
// chunk schedule the warm-up waits for the first chunk and the stream follows the copy.
size_t fused_bytes(int64_t E);
FusedBufs carve_fused(void* base, int64_t E);
void articulation_fused(const Launch& L, const CertPlan& p, const CertBufs& cb, const FinalBufs& f, const ApBufs& b0,
                        const ApBufs& b1, const FusedBufs& fb, const int32_t* u, const int32_t* v, int32_t* out_points,
                        int32_t* out_bridges, int64_t* count_dev, cudaEvent_t* bev, cudaEvent_t* aev,
                        const ChunkSchedule& chunks);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace bridges
