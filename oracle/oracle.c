/*
 * oracle.c -- plain, slow, sequential CPU oracle for the sparse-certificate bridge method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code, header, table or helper with the CUDA path
 * and includes nothing from it.
 *
 * What it computes, with the passage each function follows (Kumar & Singh, "An Efficient
 * Parallel Algorithm for finding Bridges in a Dense Graph", arXiv:2108.07346):
 *
 *   oracle_certificate      Alg. 2 (Sec. 4.B): F = spanning forest of the edge list by
 *                           union-find, F' = spanning forest of the remaining edges,
 *                           S = F u F'.
 *   oracle_pipeline_cert    Sec. 3: split E into M contiguous sets U_0..U_{M-1}, certify each
 *                           (phase 0), then phases q = 1..ceil(log2 M) replace X_i by the
 *                           certificate of X_i u X_{i+2^(q-1)} for i = 0 mod 2^q (absent
 *                           partners are empty); X_0 is the final certificate.
 *   oracle_certificate_stream   Alg. 2 as one streaming pass (F, else F'), the GPU's form.
 *   oracle_dfs_bridges      Alg. 1 (Sec. 4.A), Tarjan's disc/low test, written iteratively.
 *   oracle_bridges          Sec. 3 end to end: oracle_pipeline_cert then Alg. 1 on X_0.
 *   oracle_chain_bridges    Independent check: Schmidt's chain decomposition (IPL 113, 2013):
 *                           an edge is a bridge iff it lies on no chain.
 *   oracle_brute_bridges    Independent check: the Sec. 1 definition itself -- delete each
 *                           edge and search for another path between its ends (BFS).
 *   oracle_components       Connected components (min vertex id of each component).
 *   oracle_two_edge_components  2-edge-connected components: the components of the graph
 *                           after deleting its bridges (found by Alg. 1); label = min vertex.
 *   oracle_articulation_points  articulation ("failure") points, abstract of the paper: vertices
 *                           whose removal increases the number of components.  Tarjan's DFS
 *                           low/disc test (a root with >= 2 children; another vertex with a
 *                           child whose low >= its disc), iterative.
 *   oracle_brute_articulation   the definition: delete each vertex, count components.
 *   oracle_is_articulation      the same definition for one vertex (sampled checks at full size).
 *   oracle_block_certificate    the articulation-point method of the CUDA path, sequential: the
 *                           blocks restricted to a spanning forest T as classes of fundamental
 *                           cycles, the edges that merge classes, and the cut vertices they give.
 *
 * Readings of the paper used here (each one listed in the design notes):
 *   - Alg. 1 recurses into v when v is NOT yet visited; the timer is global and increments at
 *     every discovery; the parent is skipped by EDGE id, so a doubled edge is never a bridge.
 *   - Alg. 2 builds forests with union-find over the edges in list order (any spanning forest
 *     is a minimum one in an unweighted graph); its DFS traversal is not needed for that.
 *   - "n" in Lemma 1 is |V| of the whole graph; the bound checked is |S| <= 2(|V| - c) with c
 *     the number of components.
 *   - Self-loops are never forest edges and never bridges; parallel edges are kept.
 *   - Output: bridges as (a < b) pairs sorted ascending, two int32 per bridge.
 * Return values: count >= 0, or -1 on invalid input (vertex id outside [0, V)), -2 on
 * allocation failure.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* sequential union-find: union by size, path compression             */
/* ------------------------------------------------------------------ */
typedef struct {
  int32_t* parent;
  int32_t* size;
  int32_t n;
} uf_t;

static int uf_init(uf_t* f, int32_t n) {
  f->n = n;
  f->parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  f->size = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!f->parent || !f->size) return -1;
  for (int32_t i = 0; i < n; i++) {
    f->parent[i] = i;
    f->size[i] = 1;
  }
  return 0;
}

static void uf_reset(uf_t* f) {
  for (int32_t i = 0; i < f->n; i++) {
    f->parent[i] = i;
    f->size[i] = 1;
  }
}

static void uf_free(uf_t* f) {
  free(f->parent);
  free(f->size);
}

static int32_t uf_find(uf_t* f, int32_t x) {
  int32_t r = x;
  while (f->parent[r] != r) r = f->parent[r];
  while (f->parent[x] != r) {
    int32_t nx = f->parent[x];
    f->parent[x] = r;
    x = nx;
  }
  return r;
}

/* returns 1 if x and y were in different sets (and joins them), 0 otherwise */
static int uf_union(uf_t* f, int32_t x, int32_t y) {
  int32_t a = uf_find(f, x), b = uf_find(f, y);
  if (a == b) return 0;
  if (f->size[a] < f->size[b]) {
    int32_t t = a;
    a = b;
    b = t;
  }
  f->parent[b] = a;
  f->size[a] += f->size[b];
  return 1;
}

static int check_ids(const int32_t* u, const int32_t* v, int64_t n, int32_t V) {
  for (int64_t i = 0; i < n; i++)
    if (u[i] < 0 || u[i] >= V || v[i] < 0 || v[i] >= V) return -1;
  return 0;
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

/* sorts (a<b) pairs given as packed keys and writes them out; returns count */
static int64_t emit_sorted(uint64_t* keys, int64_t nb, int32_t* out) {
  qsort(keys, (size_t)nb, sizeof(uint64_t), cmp_u64);
  for (int64_t i = 0; i < nb; i++) {
    out[2 * i] = (int32_t)(keys[i] >> 32);
    out[2 * i + 1] = (int32_t)(keys[i] & 0xffffffffULL);
  }
  return nb;
}

static inline uint64_t pair_key(int32_t a, int32_t b) {
  int32_t lo = a < b ? a : b, hi = a < b ? b : a;
  return ((uint64_t)(uint32_t)lo << 32) | (uint64_t)(uint32_t)hi;
}

/* ------------------------------------------------------------------ */
/* Alg. 2: S = F u F' over an edge list given by ids                  */
/* ------------------------------------------------------------------ */
/* Input: edges ids[0..n) into (u, v) (ids == NULL means ids[i] = first + i).
 * Output: ids of S in out_ids (F first, then F', each in input order), F-membership in
 * out_f1 (may be NULL).  Returns |S|.  f1, f2 are caller-provided union-finds over V. */
static int64_t certificate_impl(const int32_t* u, const int32_t* v, const int64_t* ids, int64_t first, int64_t n,
                                uf_t* f1, uf_t* f2, uint8_t* in_f, int64_t* out_ids, uint8_t* out_f1) {
  uf_reset(f1);
  uf_reset(f2);
  int64_t k = 0;
  /* F: spanning forest of G = (V, E) */
  for (int64_t i = 0; i < n; i++) {
    int64_t e = ids ? ids[i] : first + i;
    in_f[i] = (uint8_t)uf_union(f1, u[e], v[e]);
    if (in_f[i]) {
      out_ids[k] = e;
      if (out_f1) out_f1[k] = 1;
      k++;
    }
  }
  /* F': spanning forest of G' = (V, E - F) */
  for (int64_t i = 0; i < n; i++) {
    if (in_f[i]) continue;
    int64_t e = ids ? ids[i] : first + i;
    if (uf_union(f2, u[e], v[e])) {
      out_ids[k] = e;
      if (out_f1) out_f1[k] = 0;
      k++;
    }
  }
  return k;
}

/* Alg. 2 on the whole edge list.  out_ids needs room for min(E, 2V) entries. */
int64_t oracle_certificate(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int64_t* out_ids,
                           uint8_t* out_f1) {
  if (E < 0 || V < 0) return -1;
  if (check_ids(u, v, E, V)) return -1;
  uf_t f1, f2;
  uint8_t* in_f = (uint8_t*)malloc((size_t)(E > 0 ? E : 1));
  if (uf_init(&f1, V) || uf_init(&f2, V) || !in_f) return -2;
  int64_t k = certificate_impl(u, v, NULL, 0, E, &f1, &f2, in_f, out_ids, out_f1);
  uf_free(&f1);
  uf_free(&f2);
  free(in_f);
  return k;
}

/* Alg. 2 in one streaming pass, as the GPU runs it: each edge in list order is offered to F and,
 * if F rejects it, to F' at once.  The edges F rejects and their order are the same as in the
 * two-pass form (F is the same forest), so the certificate is identical; this form exists to pin
 * that equivalence.  Same output convention as oracle_certificate except that S is listed in
 * list order with its F flags. */
int64_t oracle_certificate_stream(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int64_t* out_ids,
                                  uint8_t* out_f1) {
  if (E < 0 || V < 0) return -1;
  if (check_ids(u, v, E, V)) return -1;
  uf_t f1, f2;
  if (uf_init(&f1, V) || uf_init(&f2, V)) return -2;
  int64_t k = 0;
  for (int64_t e = 0; e < E; e++) {
    if (uf_union(&f1, u[e], v[e])) {
      out_ids[k] = e;
      out_f1[k++] = 1;
    } else if (uf_union(&f2, u[e], v[e])) {
      out_ids[k] = e;
      out_f1[k++] = 0;
    }
  }
  uf_free(&f1);
  uf_free(&f2);
  return k;
}

/* ------------------------------------------------------------------ */
/* Sec. 3: partition, phase-0 certificates, merge phases              */
/* ------------------------------------------------------------------ */
/* Final certificate X_0 as edge ids (out_ids, room for 2V entries) and F-membership of the
 * last certification.  phase_max (may be NULL) receives, for each phase q = 0..Q-1, the
 * largest |X_i| after that phase; *n_phases receives Q = 1 + ceil(log2 M). */
int64_t oracle_pipeline_cert(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t M,
                             int64_t* out_ids, uint8_t* out_f1, int64_t* phase_max, int32_t* n_phases) {
  if (E < 0 || V < 0 || M < 1) return -1;
  if (check_ids(u, v, E, V)) return -1;
  const int64_t cap = 2 * (int64_t)(V > 0 ? V : 1);
  int64_t maxpart = E / M + 1;
  int64_t scratch = maxpart > 2 * cap ? maxpart : 2 * cap;
  int64_t** X = (int64_t**)calloc((size_t)M, sizeof(int64_t*));
  int64_t* nX = (int64_t*)calloc((size_t)M, sizeof(int64_t));
  int64_t* merged = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * cap));
  uint8_t* in_f = (uint8_t*)malloc((size_t)scratch);
  uint8_t* f1flag = (uint8_t*)malloc((size_t)cap);
  uf_t f1, f2;
  if (!X || !nX || !merged || !in_f || !f1flag || uf_init(&f1, V) || uf_init(&f2, V)) return -2;
  int32_t q = 0;
  /* phase 0: machine i certifies G_i = (V, U_i), U_i the i-th contiguous chunk */
  int64_t pmax = 0;
  for (int32_t i = 0; i < M; i++) {
    int64_t lo = (E * (int64_t)i) / M, hi = (E * (int64_t)(i + 1)) / M;
    X[i] = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    if (!X[i]) return -2;
    nX[i] = certificate_impl(u, v, NULL, lo, hi - lo, &f1, &f2, in_f, X[i], i == 0 ? f1flag : NULL);
    if (nX[i] > pmax) pmax = nX[i];
  }
  if (phase_max) phase_max[q] = pmax;
  q++;
  /* merge phases: step s = 2^(q-1); machine i (i = 0 mod 2s) certifies X_i u X_{i+s}, the
   * partner being empty when i + s >= M */
  for (int64_t s = 1; s < M; s *= 2) {
    pmax = 0;
    for (int64_t i = 0; i < M; i += 2 * s) {
      int64_t n = nX[i];
      memcpy(merged, X[i], sizeof(int64_t) * (size_t)n);
      if (i + s < M) {
        memcpy(merged + n, X[i + s], sizeof(int64_t) * (size_t)nX[i + s]);
        n += nX[i + s];
      }
      nX[i] = certificate_impl(u, v, merged, 0, n, &f1, &f2, in_f, X[i], i == 0 ? f1flag : NULL);
      if (nX[i] > pmax) pmax = nX[i];
    }
    if (phase_max) phase_max[q] = pmax;
    q++;
  }
  int64_t kfinal = nX[0];
  if (out_f1) memcpy(out_f1, f1flag, (size_t)kfinal);
  memcpy(out_ids, X[0], sizeof(int64_t) * (size_t)kfinal);
  if (n_phases) *n_phases = q;
  for (int32_t i = 0; i < M; i++) free(X[i]);
  free(X);
  free(nX);
  free(merged);
  free(in_f);
  free(f1flag);
  uf_free(&f1);
  uf_free(&f2);
  return kfinal;
}

/* ------------------------------------------------------------------ */
/* adjacency (CSR) over an edge list given by ids                     */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t* off; /* V + 1 */
  int32_t* nbr; /* 2n */
  int64_t* eid; /* 2n: position of the edge in the input list */
} csr_t;

static int csr_build(csr_t* g, const int32_t* u, const int32_t* v, const int64_t* ids, int64_t n, int32_t V) {
  g->off = (int64_t*)calloc((size_t)V + 1, sizeof(int64_t));
  g->nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * n + 1));
  g->eid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * n + 1));
  if (!g->off || !g->nbr || !g->eid) return -1;
  for (int64_t i = 0; i < n; i++) {
    int64_t e = ids ? ids[i] : i;
    g->off[u[e] + 1]++;
    g->off[v[e] + 1]++;
  }
  for (int32_t x = 0; x < V; x++) g->off[x + 1] += g->off[x];
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(V > 0 ? V : 1));
  if (!cur) return -1;
  memcpy(cur, g->off, sizeof(int64_t) * (size_t)V);
  for (int64_t i = 0; i < n; i++) {
    int64_t e = ids ? ids[i] : i;
    int32_t a = u[e], b = v[e];
    g->nbr[cur[a]] = b;
    g->eid[cur[a]++] = i;
    g->nbr[cur[b]] = a;
    g->eid[cur[b]++] = i;
  }
  free(cur);
  return 0;
}

static void csr_free(csr_t* g) {
  free(g->off);
  free(g->nbr);
  free(g->eid);
}

/* ------------------------------------------------------------------ */
/* Alg. 1: DFS-Bridge (iterative)                                     */
/* ------------------------------------------------------------------ */
static int64_t dfs_bridges_impl(const int32_t* u, const int32_t* v, const int64_t* ids, int64_t n, int32_t V,
                                int32_t* out) {
  csr_t g;
  if (csr_build(&g, u, v, ids, n, V)) return -2;
  int64_t* disc = (int64_t*)calloc((size_t)(V > 0 ? V : 1), sizeof(int64_t));
  int64_t* low = (int64_t*)malloc(sizeof(int64_t) * (size_t)(V > 0 ? V : 1));
  int32_t* st_v = (int32_t*)malloc(sizeof(int32_t) * (size_t)(V > 0 ? V : 1));
  int64_t* st_pe = (int64_t*)malloc(sizeof(int64_t) * (size_t)(V > 0 ? V : 1));
  int64_t* st_it = (int64_t*)malloc(sizeof(int64_t) * (size_t)(V > 0 ? V : 1));
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(V > 0 ? V : 1));
  if (!disc || !low || !st_v || !st_pe || !st_it || !keys) return -2;
  int64_t time = 0, nb = 0;
  for (int32_t s = 0; s < V; s++) {
    if (disc[s]) continue;
    int64_t sp = 0;
    st_v[0] = s;
    st_pe[0] = -1;
    st_it[0] = g.off[s];
    disc[s] = low[s] = ++time;
    while (sp >= 0) {
      int32_t x = st_v[sp];
      if (st_it[sp] < g.off[x + 1]) {
        int64_t k = st_it[sp]++;
        int32_t w = g.nbr[k];
        int64_t e = g.eid[k];
        if (e == st_pe[sp]) continue; /* the edge we came in by */
        if (!disc[w]) {               /* not visited: recurse */
          sp++;
          st_v[sp] = w;
          st_pe[sp] = e;
          st_it[sp] = g.off[w];
          disc[w] = low[w] = ++time;
        } else if (disc[w] < low[x]) {
          low[x] = disc[w];
        }
      } else {
        /* x finished: fold its low into its parent and test the tree edge */
        if (sp > 0) {
          int32_t p = st_v[sp - 1];
          if (low[x] < low[p]) low[p] = low[x];
          if (low[x] > disc[p]) keys[nb++] = pair_key(p, x);
        }
        sp--;
      }
    }
  }
  int64_t r = emit_sorted(keys, nb, out);
  csr_free(&g);
  free(disc);
  free(low);
  free(st_v);
  free(st_pe);
  free(st_it);
  free(keys);
  return r;
}

/* Alg. 1 on a whole edge list.  out needs 2*max(V-1, 0) int32. */
int64_t oracle_dfs_bridges(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t* out) {
  if (E < 0 || V < 0) return -1;
  if (check_ids(u, v, E, V)) return -1;
  return dfs_bridges_impl(u, v, NULL, E, V, out);
}

/* Sec. 3 end to end: the certificate pipeline with M machines, then Alg. 1 on X_0. */
int64_t oracle_bridges(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t M, int32_t* out) {
  if (E < 0 || V < 0 || M < 1) return -1;
  int64_t* ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * (int64_t)V + 2));
  if (!ids) return -2;
  int64_t k = oracle_pipeline_cert(u, v, E, V, M, ids, NULL, NULL, NULL);
  if (k < 0) {
    free(ids);
    return k;
  }
  int64_t r = dfs_bridges_impl(u, v, ids, k, V, out);
  free(ids);
  return r;
}

/* ------------------------------------------------------------------ */
/* Independent check 1: chain decomposition (Schmidt 2013)            */
/* ------------------------------------------------------------------ */
int64_t oracle_chain_bridges(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t* out) {
  if (E < 0 || V < 0) return -1;
  if (check_ids(u, v, E, V)) return -1;
  csr_t g;
  if (csr_build(&g, u, v, NULL, E, V)) return -2;
  size_t Vs = (size_t)(V > 0 ? V : 1);
  int64_t* pre = (int64_t*)malloc(sizeof(int64_t) * Vs);
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * Vs);
  int32_t* par = (int32_t*)malloc(sizeof(int32_t) * Vs);
  int64_t* pedge = (int64_t*)malloc(sizeof(int64_t) * Vs);
  int64_t* it = (int64_t*)malloc(sizeof(int64_t) * Vs);
  int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * Vs);
  uint8_t* visited = (uint8_t*)calloc(Vs, 1);
  uint8_t* on_chain = (uint8_t*)calloc((size_t)(E > 0 ? E : 1), 1);
  uint8_t* is_tree = (uint8_t*)calloc((size_t)(E > 0 ? E : 1), 1);
  if (!pre || !order || !par || !pedge || !it || !stack || !visited || !on_chain || !is_tree) return -2;
  for (int32_t x = 0; x < V; x++) pre[x] = -1;
  int64_t cnt = 0;
  /* plain DFS: preorder numbers and tree (parent) edges */
  for (int32_t s = 0; s < V; s++) {
    if (pre[s] >= 0) continue;
    int64_t sp = 0;
    stack[0] = s;
    pre[s] = cnt;
    order[cnt++] = s;
    par[s] = -1;
    pedge[s] = -1;
    it[s] = g.off[s];
    while (sp >= 0) {
      int32_t x = stack[sp];
      if (it[x] < g.off[x + 1]) {
        int64_t k = it[x]++;
        int32_t w = g.nbr[k];
        if (pre[w] < 0) {
          pre[w] = cnt;
          order[cnt++] = w;
          par[w] = x;
          pedge[w] = g.eid[k];
          is_tree[g.eid[k]] = 1;
          it[w] = g.off[w];
          stack[++sp] = w;
        }
      } else {
        sp--;
      }
    }
  }
  /* back edges: every non-tree, non-loop edge joins an ancestor (smaller preorder) and a
   * descendant; chains start at the ancestor, vertices taken in preorder */
  int64_t* boff = (int64_t*)calloc(Vs + 1, sizeof(int64_t));
  int32_t* bto = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  int64_t* beid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
  if (!boff || !bto || !beid) return -2;
  for (int64_t e = 0; e < E; e++) {
    if (is_tree[e] || u[e] == v[e]) continue;
    int32_t anc = pre[u[e]] < pre[v[e]] ? u[e] : v[e];
    boff[anc + 1]++;
  }
  for (int32_t x = 0; x < V; x++) boff[x + 1] += boff[x];
  int64_t* bcur = (int64_t*)malloc(sizeof(int64_t) * Vs);
  memcpy(bcur, boff, sizeof(int64_t) * Vs);
  for (int64_t e = 0; e < E; e++) {
    if (is_tree[e] || u[e] == v[e]) continue;
    int32_t anc = pre[u[e]] < pre[v[e]] ? u[e] : v[e];
    int32_t des = anc == u[e] ? v[e] : u[e];
    bto[bcur[anc]] = des;
    beid[bcur[anc]++] = e;
  }
  for (int64_t i = 0; i < cnt; i++) {
    int32_t x = order[i];
    for (int64_t k = boff[x]; k < boff[x + 1]; k++) {
      visited[x] = 1;
      on_chain[beid[k]] = 1;
      int32_t w = bto[k];
      while (!visited[w]) {
        visited[w] = 1;
        on_chain[pedge[w]] = 1;
        w = par[w];
      }
    }
  }
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * Vs);
  int64_t nb = 0;
  for (int32_t x = 0; x < V; x++)
    if (pedge[x] >= 0 && !on_chain[pedge[x]]) keys[nb++] = pair_key(par[x], x);
  int64_t r = emit_sorted(keys, nb, out);
  csr_free(&g);
  free(pre);
  free(order);
  free(par);
  free(pedge);
  free(it);
  free(stack);
  free(visited);
  free(on_chain);
  free(is_tree);
  free(boff);
  free(bto);
  free(beid);
  free(bcur);
  free(keys);
  return r;
}

/* ------------------------------------------------------------------ */
/* Independent check 2: the definition (delete each edge, BFS)        */
/* ------------------------------------------------------------------ */
int64_t oracle_brute_bridges(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t* out) {
  if (E < 0 || V < 0) return -1;
  if (check_ids(u, v, E, V)) return -1;
  csr_t g;
  if (csr_build(&g, u, v, NULL, E, V)) return -2;
  size_t Vs = (size_t)(V > 0 ? V : 1);
  uint8_t* seen = (uint8_t*)malloc(Vs);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * Vs);
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(E > 0 ? E : 1));
  if (!seen || !queue || !keys) return -2;
  int64_t nb = 0;
  for (int64_t e = 0; e < E; e++) {
    if (u[e] == v[e]) continue;
    memset(seen, 0, Vs);
    int64_t qh = 0, qt = 0;
    queue[qt++] = u[e];
    seen[u[e]] = 1;
    while (qh < qt && !seen[v[e]]) {
      int32_t x = queue[qh++];
      for (int64_t k = g.off[x]; k < g.off[x + 1]; k++) {
        if (g.eid[k] == e) continue; /* the deleted edge */
        int32_t w = g.nbr[k];
        if (!seen[w]) {
          seen[w] = 1;
          queue[qt++] = w;
        }
      }
    }
    if (!seen[v[e]]) keys[nb++] = pair_key(u[e], v[e]);
  }
  int64_t r = emit_sorted(keys, nb, out);
  csr_free(&g);
  free(seen);
  free(queue);
  free(keys);
  return r;
}

/* ------------------------------------------------------------------ */
/* connected components: label = min vertex id of the component       */
/* ------------------------------------------------------------------ */
int32_t oracle_components(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t* label) {
  if (E < 0 || V < 0) return -1;
  if (check_ids(u, v, E, V)) return -1;
  uf_t f;
  if (uf_init(&f, V)) return -2;
  for (int64_t e = 0; e < E; e++) uf_union(&f, u[e], v[e]);
  int32_t* minv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(V > 0 ? V : 1));
  for (int32_t x = 0; x < V; x++) minv[x] = INT32_MAX;
  int32_t ncomp = 0;
  for (int32_t x = 0; x < V; x++) {
    int32_t r = uf_find(&f, x);
    if (minv[r] == INT32_MAX) ncomp++;
    if (x < minv[r]) minv[r] = x;
  }
  for (int32_t x = 0; x < V; x++) label[x] = minv[uf_find(&f, x)];
  free(minv);
  uf_free(&f);
  return ncomp;
}

/* ------------------------------------------------------------------ */
/* 2-edge-connected components: components of G minus its bridges     */
/* ------------------------------------------------------------------ */
int32_t oracle_two_edge_components(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t* label) {
  if (E < 0 || V < 0) return -1;
  if (check_ids(u, v, E, V)) return -1;
  int32_t* br = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * (int64_t)V + 2));
  if (!br) return -2;
  int64_t nb = dfs_bridges_impl(u, v, NULL, E, V, br);
  if (nb < 0) {
    free(br);
    return (int32_t)nb;
  }
  /* an edge is deleted iff it is a bridge; a bridge has no parallel copy, so matching the pair
   * (a, b) identifies it */
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nb + 1));
  for (int64_t i = 0; i < nb; i++) keys[i] = pair_key(br[2 * i], br[2 * i + 1]);
  uf_t f;
  if (uf_init(&f, V)) return -2;
  for (int64_t e = 0; e < E; e++) {
    if (u[e] == v[e]) continue;
    uint64_t k = pair_key(u[e], v[e]);
    if (bsearch(&k, keys, (size_t)nb, sizeof(uint64_t), cmp_u64)) continue;
    uf_union(&f, u[e], v[e]);
  }
  int32_t* minv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(V > 0 ? V : 1));
  for (int32_t x = 0; x < V; x++) minv[x] = INT32_MAX;
  int32_t nc = 0;
  for (int32_t x = 0; x < V; x++) {
    int32_t r = uf_find(&f, x);
    if (minv[r] == INT32_MAX) nc++;
    if (x < minv[r]) minv[r] = x;
  }
  for (int32_t x = 0; x < V; x++) label[x] = minv[uf_find(&f, x)];
  free(minv);
  free(keys);
  free(br);
  uf_free(&f);
  return nc;
}

/* ------------------------------------------------------------------ */
/* articulation points                                                 */
/* ------------------------------------------------------------------ */
static int64_t emit_vertices(uint8_t* flag, int32_t V, int32_t* out) {
  int64_t n = 0;
  for (int32_t x = 0; x < V; x++)
    if (flag[x]) out[n++] = x;
  return n;
}

int64_t oracle_articulation_points(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t* out) {
  if (E < 0 || V < 0) return -1;
  if (check_ids(u, v, E, V)) return -1;
  csr_t g;
  if (csr_build(&g, u, v, NULL, E, V)) return -2;
  size_t Vs = (size_t)(V > 0 ? V : 1);
  int64_t* disc = (int64_t*)calloc(Vs, sizeof(int64_t));
  int64_t* low = (int64_t*)malloc(sizeof(int64_t) * Vs);
  int32_t* st_v = (int32_t*)malloc(sizeof(int32_t) * Vs);
  int64_t* st_pe = (int64_t*)malloc(sizeof(int64_t) * Vs);
  int64_t* st_it = (int64_t*)malloc(sizeof(int64_t) * Vs);
  int64_t* nchild = (int64_t*)calloc(Vs, sizeof(int64_t));
  uint8_t* ap = (uint8_t*)calloc(Vs, 1);
  if (!disc || !low || !st_v || !st_pe || !st_it || !nchild || !ap) return -2;
  int64_t time = 0;
  for (int32_t s = 0; s < V; s++) {
    if (disc[s]) continue;
    int64_t sp = 0;
    st_v[0] = s;
    st_pe[0] = -1;
    st_it[0] = g.off[s];
    disc[s] = low[s] = ++time;
    while (sp >= 0) {
      int32_t x = st_v[sp];
      if (st_it[sp] < g.off[x + 1]) {
        int64_t k = st_it[sp]++;
        int32_t w = g.nbr[k];
        int64_t e = g.eid[k];
        if (e == st_pe[sp]) continue;
        if (!disc[w]) {
          nchild[x]++;
          sp++;
          st_v[sp] = w;
          st_pe[sp] = e;
          st_it[sp] = g.off[w];
          disc[w] = low[w] = ++time;
        } else if (disc[w] < low[x]) {
          low[x] = disc[w];
        }
      } else {
        if (sp > 0) {
          int32_t p = st_v[sp - 1];
          if (low[x] < low[p]) low[p] = low[x];
          /* a non-root p separates its child's subtree when nothing there reaches above p */
          if (sp - 1 > 0 && low[x] >= disc[p]) ap[p] = 1;
        }
        sp--;
      }
    }
    if (nchild[s] >= 2) ap[s] = 1; /* a root separates its >= 2 children */
  }
  int64_t n = emit_vertices(ap, V, out);
  csr_free(&g);
  free(disc);
  free(low);
  free(st_v);
  free(st_pe);
  free(st_it);
  free(nchild);
  free(ap);
  return n;
}

/* components of the graph with vertex `skip` deleted (skip < 0: none), ignoring that vertex */
static int32_t count_components_without(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t skip,
                                        uf_t* f) {
  uf_reset(f);
  for (int64_t e = 0; e < E; e++) {
    if (u[e] == skip || v[e] == skip) continue;
    uf_union(f, u[e], v[e]);
  }
  int32_t c = 0;
  for (int32_t x = 0; x < V; x++)
    if (x != skip && uf_find(f, x) == x) c++;
  return c;
}

int64_t oracle_brute_articulation(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t* out) {
  if (E < 0 || V < 0) return -1;
  if (check_ids(u, v, E, V)) return -1;
  uf_t f;
  if (uf_init(&f, V)) return -2;
  uint8_t* ap = (uint8_t*)calloc((size_t)(V > 0 ? V : 1), 1);
  const int32_t base = count_components_without(u, v, E, V, -1, &f);
  for (int32_t x = 0; x < V; x++) {
    /* deleting x removes its own component when x is isolated; otherwise compare */
    int isolated = 1;
    for (int64_t e = 0; e < E && isolated; e++)
      if ((u[e] == x || v[e] == x) && u[e] != v[e]) isolated = 0;
    if (isolated) continue;
    if (count_components_without(u, v, E, V, x, &f) > base) ap[x] = 1;
  }
  int64_t n = emit_vertices(ap, V, out);
  free(ap);
  uf_free(&f);
  return n;
}

/* The definition for one vertex x: 1 if deleting x (and its edges) leaves more components than
 * the graph has, not counting x itself; an isolated x (only self-loops) is never one. */
int32_t oracle_is_articulation(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int32_t x) {
  if (E < 0 || V < 0 || x < 0 || x >= V) return -1;
  if (check_ids(u, v, E, V)) return -1;
  int isolated = 1;
  for (int64_t e = 0; e < E && isolated; e++)
    if ((u[e] == x || v[e] == x) && u[e] != v[e]) isolated = 0;
  if (isolated) return 0;
  uf_t f;
  if (uf_init(&f, V)) return -2;
  const int32_t base = count_components_without(u, v, E, V, -1, &f);
  const int32_t without = count_components_without(u, v, E, V, x, &f);
  uf_free(&f);
  return without > base ? 1 : 0;
}

/* The block certificate of a spanning forest T (the GPU's articulation-point method, restated
 * sequentially).  T = the first forest of Alg. 2 (union-find over the edges in input order), each
 * tree rooted at its minimum vertex.  Tree edge (x, parent x) is named by x.  Every non-tree edge
 * closes a fundamental cycle with T, and the tree edges of one cycle lie in one block; so the
 * blocks, restricted to T, are the classes of the transitive closure of "on a common fundamental
 * cycle".  Edges are taken in input order: an edge whose cycle touches at least two current
 * classes merges them and is kept, any other adds nothing to the block structure and is dropped.
 * Each kept edge lowers the class count, so at most V - 1 are kept.  A vertex is an articulation
 * point iff its incident tree edges fall into at least two classes (each block through it holds
 * one of its tree edges).  Returns |T| + kept, fills out_ids (room for 2V) / out_tree flags and
 * the sorted articulation points (out_points, *out_np). */
int64_t oracle_block_certificate(const int32_t* u, const int32_t* v, int64_t E, int32_t V, int64_t* out_ids,
                                 uint8_t* out_tree, int32_t* out_points, int64_t* out_np) {
  if (E < 0 || V < 0) return -1;
  if (check_ids(u, v, E, V)) return -1;
  size_t Vs = (size_t)(V > 0 ? V : 1);
  uf_t f;
  if (uf_init(&f, V)) return -2;
  uint8_t* in_t = (uint8_t*)calloc((size_t)(E > 0 ? E : 1), 1);
  int64_t* tids = (int64_t*)malloc(sizeof(int64_t) * Vs);
  int64_t nt = 0;
  for (int64_t e = 0; e < E; e++)
    if (uf_union(&f, u[e], v[e])) {
      in_t[e] = 1;
      tids[nt++] = e;
    }
  /* root every tree at its minimum vertex: parent and depth by an explicit-stack traversal */
  csr_t t;
  if (csr_build(&t, u, v, tids, nt, V)) return -2;
  int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * Vs);
  int32_t* depth = (int32_t*)malloc(sizeof(int32_t) * Vs);
  int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * Vs);
  for (int32_t x = 0; x < V; x++) parent[x] = -2;
  for (int32_t s = 0; s < V; s++) {
    if (parent[s] != -2) continue;
    parent[s] = -1;
    depth[s] = 0;
    int32_t sp = 0;
    stack[sp++] = s;
    while (sp) {
      int32_t x = stack[--sp];
      for (int64_t k = t.off[x]; k < t.off[x + 1]; k++) {
        int32_t w = t.nbr[k];
        if (parent[w] != -2) continue;
        parent[w] = x;
        depth[w] = depth[x] + 1;
        stack[sp++] = w;
      }
    }
  }
  /* classes of tree edges */
  uf_t g;
  if (uf_init(&g, V)) return -2;
  int32_t* path = (int32_t*)malloc(sizeof(int32_t) * Vs);
  int64_t k = 0;
  for (int64_t i = 0; i < nt; i++) {
    out_ids[k] = tids[i];
    out_tree[k++] = 1;
  }
  for (int64_t e = 0; e < E; e++) {
    if (in_t[e] || u[e] == v[e]) continue;
    int32_t x = u[e], y = v[e], n = 0;
    while (x != y) { /* the tree path between the ends: climb the deeper end */
      if (depth[x] >= depth[y]) {
        path[n++] = x;
        x = parent[x];
      } else {
        path[n++] = y;
        y = parent[y];
      }
    }
    int merged = 0;
    for (int32_t j = 1; j < n; j++) merged |= uf_union(&g, path[0], path[j]);
    if (merged) {
      out_ids[k] = e;
      out_tree[k++] = 0;
    }
  }
  uint8_t* ap = (uint8_t*)calloc(Vs, 1);
  int32_t* first = (int32_t*)malloc(sizeof(int32_t) * Vs);
  for (int32_t x = 0; x < V; x++) first[x] = -1;
  for (int32_t c = 0; c < V; c++) {
    int32_t p = parent[c];
    if (p < 0) continue;
    int32_t gc = uf_find(&g, c);
    if (parent[p] >= 0) {
      if (gc != uf_find(&g, p)) ap[p] = 1; /* child edge and parent edge in different blocks */
    } else if (first[p] < 0) {
      first[p] = gc;
    } else if (first[p] != gc) {
      ap[p] = 1; /* a root whose child edges span two blocks */
    }
  }
  *out_np = emit_vertices(ap, V, out_points);
  uf_free(&f);
  uf_free(&g);
  csr_free(&t);
  free(in_t);
  free(tids);
  free(parent);
  free(depth);
  free(stack);
  free(path);
  free(ap);
  free(first);
  return k;
}
