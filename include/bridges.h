/*
 * bridges.h -- C ABI of libbridges.so: bridges of an undirected graph via sparse certificates
 * on one GB300 GPU (sm_103a).
 *
 * Method (Kumar & Singh, "An Efficient Parallel Algorithm for finding Bridges in a Dense
 * Graph", arXiv:2108.07346):
 *   - a bridge is an edge whose removal increases the number of connected components (Sec. 1);
 *   - the edge list is split into M partitions U_0..U_{M-1} (Sec. 3); each gets a sparse
 *     certificate S = F u F', F a spanning forest of the partition and F' a spanning forest of
 *     the remaining edges (Alg. 2, Sec. 4.B), |S| <= 2(V-1) (Lemma 1, Sec. 3);
 *   - certificates are merged in a tree, each merge re-certifying the union (Sec. 3 phases);
 *   - the bridges of the final certificate are the bridges of the graph (Sec. 3, end), found
 *     here by an Euler tour with subtree low/high ranges in place of the DFS of Alg. 1.
 *
 * Conventions for every entry point:
 *   - Edge lists are structure-of-arrays: edges_u[i], edges_v[i] (int32) is edge i, in either
 *     order.  Self-loops are allowed and ignored; repeated edges are parallel edges (and hence
 *     never bridges).  Vertex ids must lie in [0, V).
 *   - Output bridges are written as interleaved (a, b) int32 pairs with a < b, sorted
 *     ascending by (a, b); the result is unique, so it is exact and bit-reproducible.
 *     Capacity needed: 2 * max(V-1, 0) int32.
 *   - Pointers named "device" must be device pointers on the context's device; pointers named
 *     "host" must be host pointers (pinned or pageable).  The caller owns every buffer; the
 *     library never frees caller memory.  Input buffers are read-only during the call.
 *   - Streams are cudaStream_t values passed as `struct CUstream_st*` (NULL = legacy stream).
 *   - Return value: >= 0 on success (a count), or a negative bridges_status.  No C++
 *     exception crosses this interface.  Device-side failures (bad vertex id, a bounded wait
 *     that gave up) are reported through a device status word read back by the host; the
 *     device never traps.
 *   - A context is not thread-safe: use one per host thread (or serialise calls).
 */
#ifndef BRIDGES_H
#define BRIDGES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;

typedef enum bridges_status {
  BRIDGES_OK = 0,
  BRIDGES_EINVAL = -1,    /* null pointer, V < 0, E < 0, bad option */
  BRIDGES_ERANGE = -2,    /* a vertex id outside [0, V) */
  BRIDGES_ENOMEM = -3,    /* workspace larger than the context's budget, or allocation failed */
  BRIDGES_ECUDA = -4,     /* a CUDA runtime call failed */
  BRIDGES_ETIMEDOUT = -5, /* a bounded device-side wait gave up */
  BRIDGES_EAGAIN = -6,    /* request can never fit the server's memory budget */
  BRIDGES_EBUSY = -7,     /* result not ready yet */
  BRIDGES_EINTERNAL = -8, /* an internal capacity invariant failed (a bug) */
  BRIDGES_ECANCELED = -9  /* a server request withdrawn by bridges_server_cancel */
} bridges_status;

/* Tuning options.  Zero-initialise and set what you need; zero / negative fields mean
 * "choose automatically". */
typedef struct bridges_opts {
  int32_t M;           /* partitions of the edge list (Sec. 3 "M machines"); <= 0: auto (one
                          partition: on one GPU the merge rounds cost more than they save) */
  int32_t fan_in;      /* certificates merged per merge job; <= 1: auto (Sec. 3 uses 2) */
  int32_t block;       /* threads per block of the forest pass; 0: auto */
  int32_t ctas_per_sm; /* resident blocks per SM for the forest pass; 0: auto */
  int64_t warm_edges;  /* edges per partition certified before the label snapshot;
                          < 0: auto, 0: never snapshot (every edge takes the union-find path) */
  int32_t profile;     /* 1: record per-stage CUDA events on the launch stream */
  int32_t host_read;   /* bridges_find_host: 1 = when the host buffers are pinned and mapped,
                          kernels read them in place over the host link instead of copying
                          them to the device first; 0 = always copy */
  int32_t ap_warm_edges; /* bridges_articulation_points: edges of the list offered to the block
                            pass before its snapshot; 0: auto (2V + 4096 with 16-bit labels,
                            none with the bitmap that larger V takes), > 0: that many, < 0: none
                            (snapshot right after the certificate's own edges) */
  int32_t warm_block;    /* threads per block of the forest pass's warm-up launch (the prefix certified
                            through the union-finds before the snapshot); 0: auto */
  int32_t ap_fused;      /* bridges_articulation_points: 0 = auto (one read of the list for the
                            certificate and the block pass when the plan is one partition with a
                            16-bit label snapshot and the larger workspace of that form fits the
                            context's budget or workspace), < 0 = always the two-pass form */
  int32_t test_barrier_polls; /* for tests of the failure path; 0 in normal use.  > 0: a grid
                                 barrier of the final stage gives up after this many polls
                                 (~100 ns apart; default 2^22) with BRIDGES_ETIMEDOUT */
  int32_t test_hold_polls;    /* for tests of the failure path; 0 in normal use.  > 0: the final
                                 stage's last block sleeps this many ~100 ns polls before its first
                                 barrier, so that a short barrier wait above gives up */
  int32_t test_fail_alloc;    /* for tests of the failure path; 0 in normal use.  n > 0: the n-th
                                 device allocation of the context's own buffers (workspace,
                                 host-call staging, batched descriptors) after the options were
                                 set fails as on a full device: that call returns BRIDGES_ENOMEM,
                                 and the context stays usable (a later call allocates again) */
} bridges_opts;

typedef struct bridges_ctx bridges_ctx;

/* ---------------------------------------------------------------------------------------
 * Contexts.  A context owns a device workspace (grown on demand up to mem_budget_bytes, 0 =
 * no limit) plus a small pinned host area.  bridges_ctx_create returns NULL on failure
 * (bad device, CUDA error).  opts may be NULL (all automatic).
 */
bridges_ctx* bridges_ctx_create(int device, size_t mem_budget_bytes, const bridges_opts* opts);

/* As bridges_ctx_create, but the caller supplies the device workspace (e.g. a framework's
 * allocation); the context then never allocates device memory and returns BRIDGES_ENOMEM for
 * a call that needs more than ws_bytes (see bridges_workspace_bytes).  ws must stay valid until
 * bridges_ctx_destroy and must not be used by anything else meanwhile. */
bridges_ctx* bridges_ctx_create_ws(int device, void* ws_device, size_t ws_bytes, const bridges_opts* opts);

void bridges_ctx_destroy(bridges_ctx* ctx);

/* Device workspace bytes a call with these sizes and the context's options needs (the value
 * of M after automatic choice is used; M <= 0 picks it).  Returns 0 for invalid sizes. */
size_t bridges_workspace_bytes(const bridges_ctx* ctx, int64_t E, int32_t V, int32_t M);

/* ---------------------------------------------------------------------------------------
 * bridges_find_ctx -- the whole path on device-resident input (Sec. 3 end to end).
 *   edges_u, edges_v : device, E int32 each.
 *   out_bridges      : device, capacity 2*max(V-1,0) int32; receives the sorted pairs.
 *   out_count_device : device int64 or NULL; receives the bridge count (or a negative status).
 *   M                : partitions (<= 0: the context's option, else automatic).
 * Synchronous when out_count_device is NULL: waits for the stream and returns the count.
 * When out_count_device is non-NULL the call only enqueues work and returns BRIDGES_OK (0);
 * the count (or a negative status) appears in *out_count_device when the stream reaches it.
 * Errors found on the host (EINVAL, ENOMEM) are returned in both modes.
 */
int64_t bridges_find_ctx(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* edges_u,
                         const int32_t* edges_v, int64_t E, int32_t V, int32_t M, int32_t* out_bridges,
                         int64_t* out_count_device);

/* bridges_find -- plain synchronous call on device pointers, with a per-device default context
 * (created on first use on the current device, workspace grown as needed) and the legacy
 * stream.  Same arguments and result as bridges_find_ctx with out_count_device = NULL. */
int64_t bridges_find(const int32_t* edges_u, const int32_t* edges_v, int64_t E, int32_t V, int32_t M,
                     int32_t* out_bridges);

/* bridges_find_host -- the same computation from HOST buffers: copies the edges to the
 * context's device staging area, runs the path, and copies the sorted bridges back to
 * out_bridges_host.  With one partition (the automatic choice) and a list of 32 M edges or more,
 * the copy runs in chunks on a copy stream of the context while the forest pass streams the
 * chunks already copied; work on `stream` before the call is waited for first.  Synchronous;
 * returns the count.  Host buffers should be pinned for full copy bandwidth and overlap
 * (pageable memory works, slower).  With opts.host_read and pinned, mapped buffers the kernels
 * read the host memory in place instead (no device copy of the edges). */
int64_t bridges_find_host(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* edges_u_host,
                          const int32_t* edges_v_host, int64_t E, int32_t V, int32_t M,
                          int32_t* out_bridges_host);

/* ---------------------------------------------------------------------------------------
 * bridges_find_batched -- G independent graphs in one persistent launch (Sec. 3 per graph).
 *   edges_u, edges_v : device; graph g's edges are entries [edge_off[g], edge_off[g+1]) and its
 *                      vertex ids are local, in [0, V[g]).
 *   edge_off_host    : host, G+1 int64, non-decreasing (read during the call only).
 *   V_host           : host, G int32 (read during the call only).
 *   out_bridges      : device; graph g's sorted pairs start at int32 offset
 *                      sum over h < g of 2*max(V[h]-1, 0).
 *   out_counts_device: device, G int64; graph g's bridge count, or a negative status for that
 *                      graph alone (e.g. BRIDGES_ERANGE).
 * Graphs with V <= 4096 are certified and solved in shared memory by two persistent kernels,
 * replayed as one CUDA graph cached per capacity: the first certifies every task (a graph, or a
 * partition of a graph with many edges) on a 256-thread group and finishes graphs of up to 1,024
 * vertices in place; the second runs the larger graphs' bridge stages (the partitions'
 * certificates merged there), two graphs per block up to 3,008 vertices, else one.  Larger graphs
 * follow through the single-graph path on the same stream.  Enqueue-only: returns BRIDGES_OK or a
 * host-detected error; synchronise the stream before reading the outputs.  The call waits on the
 * host only for the context's batch before last, and a batch starts on the device after the
 * context's previous batch has finished, whichever stream that one ran on.
 */
int64_t bridges_find_batched(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* edges_u,
                             const int32_t* edges_v, const int64_t* edge_off_host, const int32_t* V_host, int32_t G,
                             int32_t* out_bridges, int64_t* out_counts_device);

/* Edge count above which a batched graph is split into partitions (0: automatic, the batch's
 * edges / (3 x SMs) clamped to [2^17, 2^20]).  Returns BRIDGES_OK or BRIDGES_EINVAL. */
int32_t bridges_ctx_set_batch_split(bridges_ctx* ctx, int64_t split_edges);

/* The plan of the batched form, per size bucket (what bridges_batch_autotune picks; a caller may
 * also set one, e.g. from a cache of tuning results).  Graph g belongs to the first bucket b with
 * V[g] <= vmax[b] (vmax increasing; graphs above the last vmax use the last bucket).  Per bucket:
 *   group[b] : threads of the group that runs a graph's bridge stage -- 1024 (a whole block), 512
 *              (half a block) or 256 (the certification group itself, which runs the stage of a
 *              one-partition graph of up to 1,024 vertices right after certifying it); 0 = the
 *              smallest group the graph fits (256 up to 1,024 vertices, 512 up to 3,008, 1024
 *              above).  A group too small for a graph is raised to the smallest that fits.
 *   split[b] : graphs with more edges than this are cut into ceil(E / split) contiguous
 *              partitions (at most 64, Sec. 3's M per graph), each certified by a 256-thread
 *              group; the bridge stage starts from the first partition's two forests and offers
 *              the other partitions' F and F' edges (merge fan-in = M: one merge level, since
 *              every certificate is already in device memory); 0 = automatic (the context's
 *              bridges_ctx_set_batch_split value, else the batch's edges / (3 x SMs) clamped to
 *              [2^17, 2^20]).
 *   warm_per_v[b], warm_add[b] : each task certifies its first warm_per_v * V + warm_add edges one
 *              by one before flattening its union-finds and streaming the rest; both 0 =
 *              automatic (4V + 2048).
 * n = 0 means the automatic plan for every graph.  Plans change only scheduling: results are
 * identical under every plan. */
#define BRIDGES_BATCH_BUCKETS 8
typedef struct bridges_batch_plan {
  int32_t n;
  int32_t vmax[BRIDGES_BATCH_BUCKETS];
  int32_t group[BRIDGES_BATCH_BUCKETS];
  int32_t warm_per_v[BRIDGES_BATCH_BUCKETS];
  int32_t warm_add[BRIDGES_BATCH_BUCKETS];
  int64_t split[BRIDGES_BATCH_BUCKETS];
} bridges_batch_plan;

/* Sets / reads the context's batched plan.  BRIDGES_EINVAL for a malformed plan (n outside
 * [0, 8], vmax not increasing, a group other than 0, 256, 512, 1024, a negative split or warm-up). */
int32_t bridges_ctx_set_batch_plan(bridges_ctx* ctx, const bridges_batch_plan* plan);
int32_t bridges_ctx_get_batch_plan(const bridges_ctx* ctx, bridges_batch_plan* plan);

/* bridges_batch_autotune: tunes the batched plan on a caller's batch (arguments as for
 * bridges_find_batched): buckets of vertex counts up to 256, 512, 1,024, 2,048 and 4,096, and,
 * one bucket at a time (largest first, twice over), every group size the bucket's graphs fit,
 * partition splits of 2^18 to 2^22 edges or automatic, and warm-up prefixes of 2V + 1024, 4V + 2048
 * and 8V + 2048 edges, each timed over `reps` batched calls (CUDA events on `stream`).  A change
 * is kept only when it is at least 0.5% faster (the timing noise of a few calls), and the plan
 * found is then timed against the automatic plan, in turn, three more times: the automatic plan
 * stays unless beaten by the same margin.  The plan kept goes to the context and to *best (may be
 * NULL); *best_us (may be NULL) gets its microseconds per batch.  Graphs above 4,096 vertices are not batched and not tuned.  Uses
 * the context's batched buffers; returns BRIDGES_OK or an error (the plan is then unchanged). */
int32_t bridges_batch_autotune(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* edges_u,
                               const int32_t* edges_v, const int64_t* edge_off_host, const int32_t* V_host, int32_t G,
                               int32_t reps, bridges_batch_plan* best, double* best_us);

/* ---------------------------------------------------------------------------------------
 * Serving: a continuous-batching request loop on one GPU (thread-safe).
 *
 * A request is a graph whose edge arrays are already resident on the device; the caller keeps
 * edges_u / edges_v / out_bridges valid until the request completes.  A scheduler thread keeps
 * up to max_slots units of work in flight, each on its own stream and workspace, so requests
 * overlap on the device.  Queued small graphs (V <= 4096) are gathered into one batched launch
 * (as bridges_find_batched); a large graph runs the single-graph path once its workspace fits
 * in what mem_budget_bytes has left.  The budget counts the workspaces of the single-graph
 * requests running at the time; a slot keeps the workspace it grew to, and batched buffers are
 * not counted, so the memory held can exceed the budget by up to (max_slots - 1) times the
 * largest workspace admitted, plus the batched buffers.  Requests arriving while others run are
 * admitted as slots and memory free up.  Results are exact and identical to a call on the graph alone.
 */
typedef struct bridges_request {
  const int32_t* edges_u; /* device, E int32 */
  const int32_t* edges_v; /* device, E int32 */
  int64_t E;
  int32_t V;
  int32_t M;              /* partitions for the single-graph path (<= 0: automatic) */
  int32_t* out_bridges;   /* device, capacity 2*max(V-1,0) int32 */
} bridges_request;

typedef struct bridges_server bridges_server;

/* max_slots <= 0: 4; max_batch <= 0: 4096 graphs per batched launch; mem_budget_bytes 0: no
 * limit; opts as for contexts (may be NULL).  Returns NULL on failure. */
bridges_server* bridges_server_create(int device, size_t mem_budget_bytes, int32_t max_slots, int32_t max_batch,
                                      const bridges_opts* opts);
/* Queues a request; *ticket identifies it.  BRIDGES_EAGAIN if its workspace exceeds the whole
 * budget (it could never run); BRIDGES_EINVAL for bad arguments. */
int32_t bridges_server_submit(bridges_server* srv, const bridges_request* req, uint64_t* ticket);
/* BRIDGES_EBUSY while the request is queued or running; BRIDGES_OK when done: *count gets the
 * bridge count (or the request's negative status) and *latency_ms the time from submit to
 * completion; the ticket is then released.  Either output pointer may be NULL. */
int32_t bridges_server_poll(bridges_server* srv, uint64_t ticket, int64_t* count, double* latency_ms);
/* As poll, but waits up to timeout_ms; BRIDGES_ETIMEDOUT if the request is still not done. */
int32_t bridges_server_wait(bridges_server* srv, uint64_t ticket, int64_t timeout_ms, int64_t* count,
                            double* latency_ms);
/* Withdraws a request that is still queued (not yet launched): it completes at once with count
 * BRIDGES_ECANCELED (poll / wait then release its ticket as for any request), and the caller may
 * reuse its buffers right away.  BRIDGES_EBUSY if it is already running or done (it then completes
 * normally); BRIDGES_EINVAL for an unknown or already released ticket. */
int32_t bridges_server_cancel(bridges_server* srv, uint64_t ticket);
/* [0] completed, [1] batched launches, [2] single-graph launches, [3] most requests in flight at
 * once, [4] failed launches, [5] queued now.  Returns the number of values written. */
int32_t bridges_server_stats(bridges_server* srv, int64_t* vals, int32_t n);
/* Finishes queued and running requests, then frees everything. */
void bridges_server_destroy(bridges_server* srv);

/* ---------------------------------------------------------------------------------------
 * Stage entry points (for testing and composition).
 *
 * bridges_certificate -- the sparse certificate of the whole edge list after the M-way
 * partition and the merge tree (Sec. 3; Alg. 2 per job).  Writes |S| <= 2*max(V-1,0) edges:
 * cert_u[i], cert_v[i] (device int32) and cert_tree[i] (device uint8: 1 = edge of the final
 * spanning forest F, 0 = edge of F').  Synchronous; returns |S|.  Forests are not unique
 * (concurrent union-find), but S always has the components and the bridges of the input.
 */
int64_t bridges_certificate(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* edges_u,
                            const int32_t* edges_v, int64_t E, int32_t V, int32_t M, int32_t* cert_u,
                            int32_t* cert_v, uint8_t* cert_tree);

/* bridges_from_forest -- the final stage alone (the stand-in for Alg. 1 on X_0): given a
 * spanning forest T (tree_u/tree_v, n_tree device int32 edges, acyclic, ids in [0,V)) and
 * further edges (extra_u/extra_v, n_extra device int32, each joining two vertices of one tree
 * of T), writes the sorted bridges of T u extra to out_bridges (device).  Synchronous; returns
 * the count.  T must be a forest: a cycle in T gives an unspecified result (or
 * BRIDGES_EINTERNAL), never a fault. */
int64_t bridges_from_forest(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* tree_u,
                            const int32_t* tree_v, int64_t n_tree, const int32_t* extra_u,
                            const int32_t* extra_v, int64_t n_extra, int32_t V, int32_t* out_bridges);

/* bridges_rooted_forest -- the rooted, numbered forest that the final stage's bridge test runs
 * on (its Euler tour and list ranking; the DFS of Alg. 1 visits T in such an order).  Given a
 * spanning forest T as for bridges_from_forest, each tree is rooted at its minimum vertex and:
 *   out_parent[x] : x's parent, -1 for a root (vertices on no edge of T are one-vertex trees);
 *   out_pre[x]    : x's preorder number.  The trees take consecutive ranges of [0, V) in
 *                   increasing order of their roots; inside a tree a vertex precedes its
 *                   subtree, and siblings appear in the order of the Euler tour, which follows
 *                   the adjacency lists as built concurrently (not a fixed order);
 *   out_size[x]   : the number of vertices in x's subtree (x included).
 * Each output is a device int32[V] or NULL (not written).  Synchronous; returns BRIDGES_OK or a
 * negative status (EINVAL for bad sizes or pointers, ERANGE for an id outside [0, V)); a cycle
 * in T gives unspecified output or BRIDGES_EINTERNAL, never a fault. */
int64_t bridges_rooted_forest(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* tree_u,
                              const int32_t* tree_v, int64_t n_tree, int32_t V, int32_t* out_parent,
                              int32_t* out_pre, int32_t* out_size);

/* ---------------------------------------------------------------------------------------
 * bridges_find_noalloc -- bridges_find for callers that must not allocate device memory.
 *
 * The paper has no counterpart; this is an interface for callers.  Some programs cannot call
 * cudaMalloc at the point where they need bridges: the device allocator belongs to a framework
 * (its caching allocator would be bypassed and could run out), a latency-critical loop must not
 * block in the driver, or the process reserves all device memory up front.  This entry point
 * allocates nothing: every intermediate buffer lives in one fixed 8 MiB array of device memory
 * that is part of the library itself (each GPU that loads the library holds it until the process
 * exits).  That bounds the graph: a call needs about 1.07 MB plus (132 + 30 M) bytes per vertex,
 * so V may be at most 45,135 with M = 1 (M <= 0 picks 1), 38,095 with M = 2, 29,040 with M = 4
 * and 19,679 with M = 8.  The edge count is not limited by the array.  Larger graphs return
 * BRIDGES_ENOMEM without running anything.
 *
 *   edges_u, edges_v, E, V, M, out_bridges, out_count_device : as for bridges_find_ctx, on the
 *       current device; `stream` is the launch stream.  Synchronous (returns the count) when
 *       out_count_device is NULL, otherwise enqueue-only (returns BRIDGES_OK).
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before capturing any stream into a CUDA graph.  All calls share the one
 * array, and each call leaves its contents behind for the next: calls that can overlap on the
 * GPU (different streams, or several host threads) race on it and must be serialised by the
 * caller.  Calls on one stream are ordered and safe.
 */
int64_t bridges_find_noalloc(struct CUstream_st* stream, const int32_t* edges_u, const int32_t* edges_v, int64_t E,
                             int32_t V, int32_t M, int32_t* out_bridges, int64_t* out_count_device);

/* ---------------------------------------------------------------------------------------
 * 2-edge-connected components and incremental edge additions.
 *
 * bridges_two_edge_components: labels[x] (device, V int32) = the minimum vertex of x's
 * 2-edge-connected component (the components left after deleting every bridge); the bridges
 * themselves go to out_bridges (device, may be NULL).  Synchronous; returns the number of
 * components.
 *
 * Incremental sessions keep the final certificate X of the current graph, and its union-finds,
 * resident on the device.  Adding an edge set Y offers Y to those union-finds, which turns X
 * into a certificate of X u Y and hence of E u Y (the certificate definition of Sec. 3: bridges
 * of E u Y = bridges of X u Y), then reruns the O(V) bridge stage: O(|Y| + V) per query instead
 * of O(|E| + V).  Vertex ids of Y must lie in [0, V) of the reset graph.
 *   bridges_inc_create / _destroy: one session per (device, options); not thread-safe.
 *   bridges_inc_reset(inc, stream, u, v, E, V, M, out): computes the bridges of (u, v) as
 *     bridges_find_ctx does and keeps its certificate; returns the count.
 *   bridges_inc_add(inc, stream, yu, yv, n, out): adds n edges (device); returns the bridge
 *     count of everything added so far.  On BRIDGES_ERANGE the session is unchanged.
 *   bridges_inc_two_edge_components(inc, stream, labels): 2-edge-connected components of the
 *     current graph (after the last reset / add); returns their number.
 *   bridges_inc_certificate_size: |X| of the current certificate (<= 2(V-1)).
 */
int64_t bridges_two_edge_components(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* edges_u,
                                    const int32_t* edges_v, int64_t E, int32_t V, int32_t M, int32_t* labels,
                                    int32_t* out_bridges);

typedef struct bridges_inc bridges_inc;
bridges_inc* bridges_inc_create(int device, const bridges_opts* opts);
void bridges_inc_destroy(bridges_inc* inc);
int64_t bridges_inc_reset(bridges_inc* inc, struct CUstream_st* stream, const int32_t* edges_u, const int32_t* edges_v,
                          int64_t E, int32_t V, int32_t M, int32_t* out_bridges);
int64_t bridges_inc_add(bridges_inc* inc, struct CUstream_st* stream, const int32_t* add_u, const int32_t* add_v,
                        int64_t n, int32_t* out_bridges);
int64_t bridges_inc_two_edge_components(bridges_inc* inc, struct CUstream_st* stream, int32_t* labels);
int64_t bridges_inc_certificate_size(const bridges_inc* inc);

/* ---------------------------------------------------------------------------------------
 * Articulation points ("failure points", abstract of the paper): the vertices whose removal
 * increases the number of connected components.  The paper names them but gives no method;
 * its bridge certificate does not keep them (two arbitrary spanning forests can split a
 * biconnected graph at a vertex), so this call merges, for every edge, the classes of the tree
 * edges on its fundamental cycle with a rooted spanning forest T of the bridge path (Sec. 3);
 * the final classes are the blocks (biconnected components) restricted to T, and a vertex is a
 * cut vertex iff its tree edges lie in two or more of them.  With a single-partition plan that
 * takes a 16-bit label snapshot (opts.ap_fused = 0) both passes share one read of the list: the
 * forest after the certificate's warm-up is rooted early, and edges whose cycle needs the final
 * forest are marked and walked at the end; otherwise the bridge path runs first and the list is
 * streamed a second time.  Parallel edges and self-loops are allowed and change nothing.
 *
 * bridges_articulation_points
 *   edges_u, edges_v, E, V, M : as for bridges_find_ctx (device edges; M for the bridge path).
 *   out_points        : device, capacity max(V, 1) int32; receives the cut vertices in
 *                       increasing order (may be NULL only when V <= 1).
 *   out_bridges       : device, capacity 2*max(V-1, 0) int32, or NULL; receives the sorted
 *                       bridge pairs as bridges_find_ctx does.
 *   out_counts_device : device int64[2] or NULL: [0] the number of cut vertices, [1] the number
 *                       of bridges (either may be a negative status).
 * Synchronous when out_counts_device is NULL (returns the number of cut vertices or a negative
 * status); otherwise enqueue-only, returning BRIDGES_OK.  Errors: as bridges_find_ctx (ERANGE for
 * a vertex id outside [0, V), found on the device; EINVAL / ENOMEM on the host).
 *
 * bridges_articulation_points_host: the same from HOST edge buffers (copied to the context's
 *   device staging area -- in chunks that the (first or only) pass follows as they land, as
 *   bridges_find_host does --
 *   or read in place when opts.host_read is set and they are pinned and mapped); the cut
 *   vertices go to out_points_host (host, capacity max(V, 1)).  Synchronous; returns their
 *   number or a negative status.
 * bridges_articulation_workspace_bytes: workspace a context needs for this call in the form it
 *   would take (the fused form's, when it applies).  A context made with bridges_ctx_create_ws
 *   (or limited by a budget) that holds less runs the two-pass form if that fits, else the call
 *   returns BRIDGES_ENOMEM.
 * bridges_ctx_ap_stage_ms: on a profiling context, the stage times of the last call's block
 *   pass in ms: [0] warm-up (certificate edges + prefix), [1] snapshot, [2] stream,
 *   [3] marking and compaction, [4] the whole block pass; waits for them; returns how many were
 *   written (0 when none are available).
 * bridges_ctx_ap_stage_ms_history: the same five times for each of the last min(max_calls, 32)
 *   calls, oldest first, 5 floats per call; returns the number of calls written.
 */
int64_t bridges_articulation_points(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* edges_u,
                                    const int32_t* edges_v, int64_t E, int32_t V, int32_t M, int32_t* out_points,
                                    int32_t* out_bridges, int64_t* out_counts_device);
int64_t bridges_articulation_points_host(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* edges_u_host,
                                         const int32_t* edges_v_host, int64_t E, int32_t V, int32_t M,
                                         int32_t* out_points_host);
int64_t bridges_articulation_workspace_bytes(const bridges_ctx* ctx, int64_t E, int32_t V, int32_t M);
int32_t bridges_ctx_ap_stage_ms(const bridges_ctx* ctx, float* ms, int32_t n);
int32_t bridges_ctx_ap_stage_ms_history(const bridges_ctx* ctx, float* ms, int32_t max_calls);

/* ---------------------------------------------------------------------------------------
 * Autotuning.
 * bridges_autotune: times candidate plans on the given device-resident input (M in
 * {1,2,4,8,16,32}, fan-in 2 or M, warm-up 0.3/0.45/0.6/0.8/1.2/2.0 x V ln V edges, block 1024,
 * 768 or 512; `reps` timed calls each, CUDA events on `stream`), then the warm-up launch's block
 * size (128 to 1024) for the winner, and keeps the fastest in the context's options (read them
 * back whole with bridges_ctx_get_opts).  best[0..4] receives M, fan-in, warm-up edges, block
 * size and microseconds per call.  Uses a little scratch memory of its own (the output buffers).
 * Returns BRIDGES_OK or an error (the options are then unchanged).
 * bridges_ctx_set_opts: replaces the context's tuning options (e.g. from a cache of tuning
 * results); the profiling flag stays as created.
 * bridges_ctx_get_opts: copies the context's current options to *opts.
 */
int32_t bridges_autotune(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* edges_u,
                         const int32_t* edges_v, int64_t E, int32_t V, int32_t reps, int64_t* best);
int32_t bridges_ctx_set_opts(bridges_ctx* ctx, const bridges_opts* opts);
int32_t bridges_ctx_get_opts(const bridges_ctx* ctx, bridges_opts* opts);

/* bridges_wait_value: a bounded device-side wait -- one thread polls the device int32 *flag
 * (acquire loads, ~100 ns apart) until it equals `value` or max_polls polls were made, on
 * `stream`.  Synchronous: BRIDGES_OK if the value was seen, BRIDGES_ETIMEDOUT if the wait gave
 * up; the context stays usable either way.  This is the primitive behind the library's device
 * barriers (which never wait unboundedly); it is exposed so that callers can order work on a
 * flag written by another stream, and so that tests can check that a wait nothing satisfies ends
 * in an error status instead of a hang. */
int32_t bridges_wait_value(bridges_ctx* ctx, struct CUstream_st* stream, const int32_t* flag_device, int32_t value,
                           int64_t max_polls);

/* ---------------------------------------------------------------------------------------
 * Introspection.
 * bridges_ctx_stage_ms: per-stage device times (ms) of the context's last call, measured with
 * CUDA events on the launch stream when opts.profile = 1: [0] partition warm-up, [1] label
 * snapshot, [2] forest pass, [3] merge tree, [4] final stage (tree, tour, ranges, test, sort),
 * [5] total.  Returns the number of values written (0 if profiling is off).
 * bridges_ctx_launches: kernels launched by the context since creation.
 * bridges_ctx_last_config: the M, fan-in, CTAs per partition, block size and warm-up edges
 * of the last call (5 values), then the last bridges_articulation_points call's block-pass
 * prefix edges (-1: no snapshot) and blocks (values 6 and 7) and its form (value 8: 1 = one
 * fused read of the list, 0 = two passes); returns min(n, 8).
 * bridges_status_string: a static description of a status code.
 */
int32_t bridges_ctx_stage_ms(const bridges_ctx* ctx, float* ms, int32_t n);
/* bridges_ctx_stage_ms_history: the same six values for each of the context's last
 * min(max_calls, 32) profiled calls, oldest first, 6 floats per call; returns the number of
 * calls written.  Waits for those calls to finish. */
int32_t bridges_ctx_stage_ms_history(const bridges_ctx* ctx, float* ms, int32_t max_calls);
int64_t bridges_ctx_launches(const bridges_ctx* ctx);
int32_t bridges_ctx_last_config(const bridges_ctx* ctx, int64_t* vals, int32_t n);
const char* bridges_status_string(int32_t status);

#ifdef __cplusplus
}
#endif

#endif /* BRIDGES_H */
