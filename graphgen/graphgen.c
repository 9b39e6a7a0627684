/*
 * graphgen.c -- seeded synthetic graph generators.
 *
 * This module produces INPUTS only.  It holds none of the bridge method's
 * arithmetic (no union-find, no forests, no DFS); both the CPU oracle and the
 * CUDA path consume what it writes.
 *
 * Workload shapes follow the paper's setting of dense graphs with few
 * vertices and many edges (Sec. 3, Figs. 2-4): Erdos-Renyi clusters joined by
 * a random inter-cluster tree, plus planted pendant vertices, pendant paths,
 * pendant trees and two-edge vertices whose bridge status is known by
 * construction (Sec. 1 definition of a bridge).
 *
 * Randomness: every draw comes from a counter-based generator, SplitMix64's
 * output function (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) applied to key + counter * golden-gamma, so the
 * result is independent of the thread count.  Vertex relabelling and edge
 * shuffling use a keyed bijection on the next power of two with cycle walking
 * (Black & Rogaway, "Ciphers with arbitrary finite domains", CT-RSA 2002).  Floating point is used only to turn a density into
 * an integer threshold and to draw log-uniform sizes; the file is compiled
 * with -ffp-contract=off and calls no libm routine, so x86-64 and aarch64
 * builds produce identical graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "graphgen.h"
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9e3779b97f4a7c15ULL

enum {
  ST_ER = 1,
  ST_STRUCT = 2,
  ST_VPERM = 3,
  ST_EPERM = 4,
  ST_PARAM = 5,
};

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(seed ^ mix64(stream * GOLDEN + 0x5851f42d4c957f2dULL));
}

static inline uint64_t draw(uint64_t key, uint64_t ctr) { return mix64(key + ctr * GOLDEN); }

typedef struct {
  uint64_t key;
  uint64_t ctr;
} seq_rng;

static inline uint64_t seq_next(seq_rng* r) { return draw(r->key, ++r->ctr); }

/* uniform integer in [0, n), n >= 1 (multiply-shift; bias < 2^-32) */
static inline uint64_t seq_below(seq_rng* r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)seq_next(r) * n) >> 64);
}

/* uniform double in [0, 1) */
static inline double seq_unit(seq_rng* r) { return (double)(seq_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* 2^x for 0 <= x < 64 without libm: integer part by ldexp-free scaling, fractional part by
 * the Taylor series of exp(f ln 2) to 30 terms (ample for double). */
static double exp2_det(double x) {
  int ip = (int)x;
  double f = x - (double)ip;
  const double ln2 = 0.69314718055994530942;
  double t = f * ln2, term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; k++) {
    term = term * t / (double)k;
    sum = sum + term;
  }
  double p = 1.0;
  for (int i = 0; i < ip; i++) p = p * 2.0;
  return sum * p;
}

/* ---------------- keyed bijection on [0, n) ----------------
 * Three rounds of (add key, multiply by an odd key, xor-shift right) on b = ceil(log2 n) bits;
 * each step is a bijection of [0, 2^b), so their composition is one.  Cycle walking maps it onto
 * [0, n) (Black & Rogaway 2002); since 2^b < 2n the expected walk is below two steps. */
typedef gg_perm perm_t;

static void perm_init(perm_t* P, uint64_t n, uint64_t seed, uint64_t stream) {
  int b = 1;
  while (b < 62 && (1ULL << b) < n) b++;
  P->mask = (1ULL << b) - 1;
  P->shift = b / 2 + 1;
  P->n = n;
  uint64_t key = stream_key(seed, stream);
  for (int r = 0; r < 3; r++) {
    P->add[r] = draw(key, 2 * (uint64_t)r + 1) & P->mask;
    P->mul[r] = (draw(key, 2 * (uint64_t)r + 2) | 1ULL) & P->mask;
  }
}

static inline uint64_t perm_once(const perm_t* P, uint64_t x) {
  for (int r = 0; r < 3; r++) {
    x = (x + P->add[r]) & P->mask;
    x = (x * P->mul[r]) & P->mask;
    x ^= x >> P->shift;
  }
  return x;
}

static inline uint64_t perm_apply(const perm_t* P, uint64_t x) {
  do {
    x = perm_once(P, x);
  } while (x >= P->n);
  return x;
}

/* ---------------- specification (gg_spec, gg_graph, gg_layout: graphgen.h) ---------------- */
static inline int32_t cluster_start(const gg_spec* s, int64_t c) {
  return (int32_t)((c * (int64_t)s->core_vertices) / s->n_clusters);
}

static inline uint64_t density_threshold(double p) {
  if (p <= 0.0) return 0;
  if (p >= 1.0) return UINT64_MAX;
  double t = p * 18446744073709551616.0;
  if (t >= 18446744073709551615.0) return UINT64_MAX;
  return (uint64_t)t;
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

/* counter for the ER trial of local pair (la, lb), la < lb, in cluster c of size sz */
static inline uint64_t er_ctr(int64_t c, int64_t sz, int64_t la, int64_t lb) {
  uint64_t pidx = (uint64_t)(la * sz - la * (la + 1) / 2 + (lb - la - 1));
  return ((uint64_t)c << 42) ^ pidx;
}

static int validate(const gg_spec* s) {
  if (s->n_clusters < 1 || s->core_vertices < s->n_clusters) return -1;
  if (s->n_paths > 0 && (s->path_min < 1 || s->path_max < s->path_min)) return -1;
  if (s->n_trees > 0 && (s->tree_min < 1 || s->tree_max < s->tree_min)) return -1;
  if ((s->n_extra_pairs > 0 || s->n_extra > 0) && s->n_clusters < 2) return -1;
  if (s->n_two_edge > 0 && s->core_vertices < 2) return -1;
  if (s->n_pendant < 0 || s->n_paths < 0 || s->n_extra_pairs < 0 || s->n_extra < 0 || s->n_trees < 0 ||
      s->n_two_edge < 0)
    return -1;
  return 0;
}

/* Everything of the graph of *s except its Erdos-Renyi edges: the sizes, the structural edges
 * (cluster tree, extra edges, pendant vertices, paths and trees, two-edge vertices) in raw ids,
 * and the planted bridges after relabelling.  The ER edges depend on the cluster sizes only, so
 * they can be drawn anywhere (host or device) from (kER, thr) and added in row order. */
gg_layout* gg_layout_make(const gg_spec* s_in) {
  gg_layout* L = (gg_layout*)calloc(1, sizeof(gg_layout));
  if (!L) return NULL;
  L->s = *s_in;
  const gg_spec* s = &L->s;
  if (validate(s)) {
    free(L);
    return NULL;
  }
  const int64_t Vc = s->core_vertices;
  const int64_t nc = s->n_clusters;
  L->Vc = Vc;
  L->nc = nc;
  L->thr = density_threshold(s->p);
  L->kER = stream_key(s->seed, ST_ER);
  int32_t* rowcl = (int32_t*)malloc((size_t)Vc * sizeof(int32_t));
  if (!rowcl) {
    free(L);
    return NULL;
  }
  for (int64_t c = 0; c < nc; c++)
    for (int64_t a = cluster_start(s, c); a < cluster_start(s, c + 1); a++) rowcl[a] = (int32_t)c;

  /* ---- structural edges (sequential stream) ---- */
  seq_rng R = {stream_key(s->seed, ST_STRUCT), 0};
  int64_t n_path_edges = 0, n_tree_edges = 0;
  /* sizes are drawn first so the vertex and edge counts are known */
  int32_t* path_len = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->n_paths + 1));
  int32_t* tree_sz = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->n_trees + 1));
  for (int i = 0; i < s->n_paths; i++) {
    path_len[i] = s->path_min + (int32_t)seq_below(&R, (uint64_t)(s->path_max - s->path_min + 1));
    n_path_edges += path_len[i];
  }
  for (int i = 0; i < s->n_trees; i++) {
    tree_sz[i] = s->tree_min + (int32_t)seq_below(&R, (uint64_t)(s->tree_max - s->tree_min + 1));
    n_tree_edges += tree_sz[i]; /* size-1 internal edges + 1 hanging edge */
  }
  const int64_t n_ctree = nc - 1;
  const int64_t n_struct = n_ctree + 2LL * s->n_extra_pairs + s->n_extra + s->n_pendant + n_path_edges +
                           n_tree_edges + 2LL * s->n_two_edge;
  const int64_t V = Vc + s->n_pendant + n_path_edges + n_tree_edges + s->n_two_edge;
  L->V = V;
  L->n_struct = n_struct;
  if (V > INT32_MAX) {
    free(rowcl);
    free(path_len);
    free(tree_sz);
    free(L);
    return NULL;
  }

  int32_t* su = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_struct + 1));
  int32_t* sv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_struct + 1));
  uint8_t* splanted = (uint8_t*)calloc((size_t)(n_struct + 1), 1);
  int32_t* cpar = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc);
  int32_t* cdepth = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc);
  uint8_t* covered = (uint8_t*)calloc((size_t)nc, 1); /* covered[c]: tree edge (c, parent c) covered */
  int64_t k = 0;
  int64_t next_vertex = Vc;

#define CORE_IN(c) (cluster_start(s, (c)) + (int32_t)seq_below(&R, (uint64_t)(cluster_start(s, (c) + 1) - cluster_start(s, (c)))))
#define ANY_CORE() ((int32_t)seq_below(&R, (uint64_t)Vc))

  /* random recursive tree over clusters: cluster c >= 1 hangs under a uniform earlier cluster */
  cpar[0] = -1;
  cdepth[0] = 0;
  for (int64_t c = 1; c < nc; c++) {
    cpar[c] = (int32_t)seq_below(&R, (uint64_t)c);
    cdepth[c] = cdepth[cpar[c]] + 1;
  }
  int64_t ctree_base = k;
  for (int64_t c = 1; c < nc; c++) {
    su[k] = CORE_IN(c);
    sv[k] = CORE_IN(cpar[c]);
    k++;
  }
  /* an extra connection between clusters a and b covers every tree edge on the cluster-tree path a..b */
#define COVER(a_, b_)                         \
  do {                                        \
    int32_t x_ = (a_), y_ = (b_);             \
    while (x_ != y_) {                        \
      if (cdepth[x_] >= cdepth[y_]) {         \
        covered[x_] = 1;                      \
        x_ = cpar[x_];                        \
      } else {                                \
        covered[y_] = 1;                      \
        y_ = cpar[y_];                        \
      }                                       \
    }                                         \
  } while (0)
  for (int i = 0; i < s->n_extra_pairs; i++) {
    int32_t a = (int32_t)seq_below(&R, (uint64_t)nc);
    int32_t b = (int32_t)seq_below(&R, (uint64_t)(nc - 1));
    if (b >= a) b++;
    for (int j = 0; j < 2; j++) {
      su[k] = CORE_IN(a);
      sv[k] = CORE_IN(b);
      k++;
    }
    COVER(a, b);
  }
  for (int i = 0; i < s->n_extra; i++) {
    int32_t a = (int32_t)seq_below(&R, (uint64_t)nc);
    int32_t b = (int32_t)seq_below(&R, (uint64_t)(nc - 1));
    if (b >= a) b++;
    su[k] = CORE_IN(a);
    sv[k] = CORE_IN(b);
    k++;
    COVER(a, b);
  }
  for (int i = 0; i < s->n_pendant; i++) {
    su[k] = ANY_CORE();
    sv[k] = (int32_t)next_vertex++;
    splanted[k] = 1;
    k++;
  }
  for (int i = 0; i < s->n_paths; i++) {
    int32_t prev = ANY_CORE();
    for (int j = 0; j < path_len[i]; j++) {
      int32_t w = (int32_t)next_vertex++;
      su[k] = prev;
      sv[k] = w;
      splanted[k] = 1;
      k++;
      prev = w;
    }
  }
  for (int i = 0; i < s->n_trees; i++) {
    int32_t base = (int32_t)next_vertex;
    next_vertex += tree_sz[i];
    su[k] = ANY_CORE();
    sv[k] = base;
    splanted[k] = 1;
    k++;
    for (int j = 1; j < tree_sz[i]; j++) {
      su[k] = base + (int32_t)seq_below(&R, (uint64_t)j);
      sv[k] = base + j;
      splanted[k] = 1;
      k++;
    }
  }
  for (int i = 0; i < s->n_two_edge; i++) {
    int32_t w = (int32_t)next_vertex++;
    int32_t c1 = ANY_CORE();
    int32_t c2 = (int32_t)seq_below(&R, (uint64_t)(Vc - 1));
    if (c2 >= c1) c2++;
    su[k] = w;
    sv[k] = c1;
    k++;
    su[k] = w;
    sv[k] = c2;
    k++;
    if (rowcl[c1] != rowcl[c2]) COVER(rowcl[c1], rowcl[c2]);
  }
#undef CORE_IN
#undef ANY_CORE
#undef COVER
  /* uncovered cluster-tree edges are bridges whatever the clusters' insides look like */
  for (int64_t c = 1; c < nc; c++)
    if (!covered[c]) splanted[ctree_base + (c - 1)] = 1;

  /* the vertex relabelling and the planted bridges in final ids */
  perm_init(&L->PV, (uint64_t)(V > 0 ? V : 1), s->seed, ST_VPERM);
  int64_t np = 0;
  for (int64_t i = 0; i < n_struct; i++) np += splanted[i];
  L->n_planted = np;
  L->planted = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * np + 2));
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(np + 1));
  int64_t q = 0;
  for (int64_t i = 0; i < n_struct; i++) {
    if (!splanted[i]) continue;
    const int64_t ra = gg_relabel(L, su[i]), rb = gg_relabel(L, sv[i]);
    const int64_t lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
    keys[q++] = ((uint64_t)lo << 32) | (uint64_t)hi;
  }
  qsort(keys, (size_t)np, sizeof(uint64_t), cmp_u64);
  for (int64_t i = 0; i < np; i++) {
    L->planted[2 * i] = (int32_t)(keys[i] >> 32);
    L->planted[2 * i + 1] = (int32_t)(keys[i] & 0xffffffffULL);
  }
  free(keys);
  L->su = su;
  L->sv = sv;
  L->rowcl = rowcl;
  free(path_len);
  free(tree_sz);
  free(splanted);
  free(cpar);
  free(cdepth);
  free(covered);
  return L;
}

void gg_layout_free(gg_layout* L) {
  if (!L) return;
  free(L->su);
  free(L->sv);
  free(L->planted);
  free(L->rowcl);
  free(L);
}

/* Final id of raw vertex x (the keyed bijection, or x itself without relabelling). */
int64_t gg_relabel(const gg_layout* L, int64_t x) {
  return L->s.relabel ? (int64_t)perm_apply(&L->PV, (uint64_t)x) : x;
}

/* The edge shuffle of a graph with E edges: the keyed bijection's parameters (perm_t). */
void gg_edge_perm(const gg_layout* L, int64_t E, gg_perm* out) {
  perm_init(out, (uint64_t)(E > 0 ? E : 1), L->s.seed, ST_EPERM);
}

/* Generates the graph described by *s.  Returns NULL on invalid spec or out of memory. */
gg_graph* gg_generate(const gg_spec* s_in) {
  gg_layout* L = gg_layout_make(s_in);
  if (!L) return NULL;
  const gg_spec* s = &L->s;
  const int64_t Vc = L->Vc;
  const uint64_t thr = L->thr;
  const uint64_t kER = L->kER;
  const int32_t* rowcl = L->rowcl;

  /* ---- pass 1: ER edge count per core row ---- */
  int64_t* rowoff = (int64_t*)malloc((size_t)(Vc + 1) * sizeof(int64_t));
  if (!rowoff) {
    gg_layout_free(L);
    return NULL;
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < Vc; a++) {
    int64_t c = rowcl[a];
    int64_t c0 = cluster_start(s, c), sz = cluster_start(s, c + 1) - c0;
    int64_t la = a - c0, cnt = 0;
    for (int64_t lb = la + 1; lb < sz; lb++) cnt += (draw(kER, er_ctr(c, sz, la, lb)) < thr);
    rowoff[a + 1] = cnt;
  }
  rowoff[0] = 0;
  for (int64_t a = 0; a < Vc; a++) rowoff[a + 1] += rowoff[a];
  const int64_t n_er = rowoff[Vc];
  const int64_t n_struct = L->n_struct;
  const int64_t V = L->V;
  const int64_t E = n_er + n_struct;

  /* ---- output with relabelling and shuffling ---- */
  gg_graph* g = (gg_graph*)calloc(1, sizeof(gg_graph));
  g->E = E;
  g->V = (int32_t)V;
  g->n_er = n_er;
  g->u = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  g->v = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  g->planted = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * L->n_planted + 2));
  if (!g->u || !g->v || !g->planted) {
    free(g->u);
    free(g->v);
    free(g->planted);
    free(g);
    g = NULL;
    goto done;
  }
  {
    perm_t PE;
    gg_edge_perm(L, E, &PE);
    const int shuffle = s->shuffle;
    int32_t* phi = (int32_t*)malloc(sizeof(int32_t) * (size_t)(V > 0 ? V : 1));
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < V; x++) phi[x] = (int32_t)gg_relabel(L, x);
    int32_t* ou = g->u;
    int32_t* ov = g->v;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < Vc; a++) {
      int64_t c = rowcl[a];
      int64_t c0 = cluster_start(s, c), sz = cluster_start(s, c + 1) - c0;
      int64_t la = a - c0, pos = rowoff[a];
      int64_t ra = phi[a];
      for (int64_t lb = la + 1; lb < sz; lb++) {
        if (draw(kER, er_ctr(c, sz, la, lb)) < thr) {
          int64_t b = c0 + lb;
          int64_t rb = phi[b];
          int64_t at = shuffle ? (int64_t)perm_apply(&PE, (uint64_t)pos) : pos;
          ou[at] = (int32_t)(ra < rb ? ra : rb);
          ov[at] = (int32_t)(ra < rb ? rb : ra);
          pos++;
        }
      }
    }
    for (int64_t i = 0; i < n_struct; i++) {
      int64_t ra = phi[L->su[i]];
      int64_t rb = phi[L->sv[i]];
      int64_t lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
      int64_t raw = n_er + i;
      int64_t at = shuffle ? (int64_t)perm_apply(&PE, (uint64_t)raw) : raw;
      ou[at] = (int32_t)lo;
      ov[at] = (int32_t)hi;
    }
    g->n_planted = L->n_planted;
    memcpy(g->planted, L->planted, sizeof(int32_t) * (size_t)(2 * L->n_planted));
    free(phi);
  }
done:
  free(rowoff);
  gg_layout_free(L);
  return g;
}

void gg_free(gg_graph* g) {
  if (!g) return;
  free(g->u);
  free(g->v);
  free(g->planted);
  free(g);
}

/* Per-graph parameters of the batched and served workloads, drawn from one sequential stream
 * keyed by (seed, index).  Sizes are log-uniform in [vmin, vmax] (vmax/vmin a power of two,
 * log2 ratio = lg_ratio), densities uniform in [dmin, dmax].
 *
 * kind 0 (batched): b ~ U{1..32} planted bridges, c ~ U{2..min(8, b+1)} clusters; the cluster
 *   tree gives c-1 bridges and b-(c-1) pendant vertices give the rest; core = V - pendants.
 * kind 1 (served): clusters of min(512, V) vertices, ceil(V*1000/32768) pendant paths of length
 *   1-8 and ceil(V*500/32768) extra inter-cluster edges (the mid-size plant mix scaled by V). */
int gg_workload_spec(int kind, uint64_t seed, int64_t index, int32_t vmin, int32_t lg_ratio, double dmin,
                     double dmax, gg_spec* out) {
  seq_rng R = {stream_key(seed ^ mix64((uint64_t)index + 1), ST_PARAM), 0};
  double u = seq_unit(&R);
  double vv = (double)vmin * exp2_det(u * (double)lg_ratio);
  int32_t V = (int32_t)(vv + 0.5);
  if (V < vmin) V = vmin;
  double d = dmin + (dmax - dmin) * seq_unit(&R);
  memset(out, 0, sizeof(*out));
  out->seed = mix64(seed * GOLDEN + (uint64_t)index);
  out->p = d;
  out->shuffle = 1;
  out->relabel = 1;
  if (kind == 0) {
    int32_t b = 1 + (int32_t)seq_below(&R, 32);
    int32_t cmax = b + 1 < 8 ? b + 1 : 8;
    int32_t c = 2 + (int32_t)seq_below(&R, (uint64_t)(cmax - 1));
    int32_t pend = b - (c - 1);
    out->n_clusters = c;
    out->core_vertices = V - pend;
    out->n_pendant = pend;
    return 0;
  }
  if (kind == 1) {
    int32_t cs = V < 512 ? V : 512;
    int32_t nclu = (V + cs - 1) / cs;
    int32_t npath = (int32_t)(((int64_t)V * 1000 + 32767) / 32768);
    int32_t nextra = (int32_t)(((int64_t)V * 500 + 32767) / 32768);
    out->n_clusters = nclu;
    out->core_vertices = V;
    out->n_paths = npath;
    out->path_min = 1;
    out->path_max = 8;
    out->n_extra = nclu >= 2 ? nextra : 0;
    return 0;
  }
  return -1;
}

/* Seeded random multigraph for tests: E edges with endpoints uniform in [0, V); self-loops and
 * duplicates are kept (the method must handle both).  No normalisation. */
void gg_random_multigraph(uint64_t seed, int32_t V, int64_t E, int32_t* u, int32_t* v) {
  uint64_t key = stream_key(seed, 77);
  for (int64_t i = 0; i < E; i++) {
    uint64_t r = draw(key, (uint64_t)i);
    u[i] = (int32_t)(((r & 0xffffffffULL) * (uint64_t)V) >> 32);
    v[i] = (int32_t)(((r >> 32) * (uint64_t)V) >> 32);
  }
}

/* R-MAT graph (Chakrabarti, Zhan & Faloutsos, SDM 2004): each of E edges picks one of the four
 * quadrants of the 2^scale x 2^scale adjacency matrix with probabilities a, b, c, 1-a-b-c, scale
 * times over; vertex ids are then relabelled by the keyed bijection (so hubs do not sit at small
 * ids).  Self-loops and repeated edges are kept.  Skewed degrees: a few hubs, many leaves. */
void gg_rmat(uint64_t seed, int32_t scale, int64_t E, double a, double b, double c, int32_t* u, int32_t* v) {
  const uint64_t ta = density_threshold(a), tb = density_threshold(a + b), tc = density_threshold(a + b + c);
  const uint64_t key = stream_key(seed, 91);
  perm_t P;
  perm_init(&P, (uint64_t)1 << scale, seed, 92);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < E; i++) {
    uint64_t x = 0, y = 0;
    for (int32_t k = 0; k < scale; k++) {
      const uint64_t r = draw(key, (uint64_t)i * (uint64_t)scale + (uint64_t)k);
      const uint64_t bx = r >= tb, by = (r >= ta && r < tb) || r >= tc;
      x = (x << 1) | bx;
      y = (y << 1) | by;
    }
    u[i] = (int32_t)perm_apply(&P, x);
    v[i] = (int32_t)perm_apply(&P, y);
  }
}

int gg_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
