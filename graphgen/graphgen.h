/*
 * graphgen.h -- types shared by the host generator (graphgen.c) and its device form
 * (graphgen_dev.cu).  Inputs only: nothing here belongs to the bridge method.
 */
#ifndef GRAPHGEN_H
#define GRAPHGEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* keyed bijection on [0, n): three rounds of (add, odd multiply, xor-shift) on ceil(log2 n)
 * bits, cycle-walked onto [0, n) */
typedef struct {
  uint64_t add[3], mul[3];
  int shift;
  uint64_t mask;
  uint64_t n;
} gg_perm;

typedef struct {
  uint64_t seed;
  int32_t n_clusters;    /* >= 1; core vertices are split into near-equal clusters */
  int32_t core_vertices; /* >= n_clusters */
  double p;              /* Erdos-Renyi density inside every cluster */
  int32_t n_pendant;     /* pendant vertices, one edge each to a random core vertex */
  int32_t n_paths;       /* pendant paths hung from random core vertices */
  int32_t path_min, path_max;
  int32_t n_extra_pairs; /* pairs of edges joining the same random pair of distinct clusters */
  int32_t n_extra;       /* single extra edges between random distinct clusters */
  int32_t n_trees;       /* pendant random recursive trees, each hung by one edge */
  int32_t tree_min, tree_max;
  int32_t n_two_edge; /* vertices joined to two distinct random core vertices */
  int32_t shuffle;    /* 1: random edge order */
  int32_t relabel;    /* 1: random vertex ids */
} gg_spec;

typedef struct {
  int64_t E;
  int32_t V;
  int64_t n_planted;
  int32_t* u;
  int32_t* v;
  int32_t* planted; /* 2 * n_planted, (a<b) pairs sorted ascending */
  int64_t n_er;     /* edges inside clusters */
} gg_graph;

/* A graph of a spec without its Erdos-Renyi edges (gg_layout_make).  Its ER edges are the
 * pairs (a, b), a < b in one cluster, whose draw(kER, counter of the pair) is below thr; they
 * take raw positions [0, n_er) in row order (row a, then b ascending), the structural edges
 * positions n_er + i; the final position of raw position r is the edge shuffle of r. */
typedef struct {
  gg_spec s;
  int64_t Vc, nc;     /* core vertices, clusters */
  int64_t V;          /* all vertices */
  int64_t n_struct;   /* structural edges */
  uint64_t thr, kER;  /* ER density threshold and key */
  int32_t* su;        /* structural edges in raw ids (before relabelling), n_struct each */
  int32_t* sv;
  int64_t n_planted;
  int32_t* planted;   /* 2 * n_planted: the planted bridges, final ids, sorted (a<b) pairs */
  int32_t* rowcl;     /* cluster of each core vertex */
  gg_perm PV;         /* vertex relabelling (used when s.relabel) */
} gg_layout;

gg_layout* gg_layout_make(const gg_spec* s);
void gg_layout_free(gg_layout* L);
int64_t gg_relabel(const gg_layout* L, int64_t x);
void gg_edge_perm(const gg_layout* L, int64_t E, gg_perm* out);

#ifdef __cplusplus
}
#endif

#endif
