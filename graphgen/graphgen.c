/*
 * Seeded synthetic graph generators and the CSR cleaner.
 *
 * This module only PRODUCES inputs (simple undirected graphs in CSR form with
 * id-sorted adjacency, Section 2.2 of the paper: "simple graphs", adjacency
 * lists). It holds none of the clustering method's arithmetic: no
 * intersections, similarities, orders or queries. Both the CPU oracle and the
 * CUDA library are fed from here; neither is imported by it.
 *
 * Random numbers come from one counter-based generator: output number `ctr` of
 * a SplitMix64 stream (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) whose state starts at `key`. Every draw is a pure
 * function of (key, ctr), so results do not depend on the thread count.
 *
 * Generators:
 *  - R-MAT (Chakrabarti, Zhan, Faloutsos 2004): each of edgefactor * 2^scale
 *    samples descends `scale` levels, choosing quadrant (src bit, dst bit) =
 *    (0,0),(0,1),(1,0),(1,1) with probabilities a, b, c, d = 1-a-b-c, no noise.
 *    Two levels are taken per 64-bit draw (32-bit uniforms). An optional seeded
 *    Fisher-Yates permutation relabels the vertices.
 *  - Stochastic block model: vertices split into `blocks` contiguous blocks whose
 *    sizes differ by at most one; each unordered pair is an edge independently
 *    with p_in (same block) or p_out (different blocks). Pairs are enumerated by
 *    geometric skipping (Batagelj and Brandes 2005), so work is O(n + m).
 *
 * Cleaning (every generator ends with it): drop self-loops, symmetrise, sort
 * each adjacency list by id and remove duplicates. Offsets are int64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

typedef struct gg_graph {
  int64_t n;
  int64_t arcs;
  int64_t* off; /* n+1 */
  int32_t* adj; /* arcs */
} gg_graph;

static inline uint64_t gg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Stream key for a user seed and a sub-stream tag. */
uint64_t gg_key(uint64_t seed, uint64_t tag) {
  return gg_mix64(gg_mix64(seed + GG_GAMMA) ^ (tag * 0xD1B54A32D192ED03ULL + 0x632BE59BD9B4E019ULL));
}

/* Output number ctr (0-based) of the SplitMix64 stream with initial state key. */
uint64_t gg_draw(uint64_t key, uint64_t ctr) { return gg_mix64(key + (ctr + 1) * GG_GAMMA); }

/* Uniform double in [0,1) from the top 53 bits of a draw. */
static inline double gg_unit(uint64_t key, uint64_t ctr) {
  return (double)(gg_draw(key, ctr) >> 11) * (1.0 / 9007199254740992.0);
}

double gg_uniform(uint64_t key, uint64_t ctr) { return gg_unit(key, ctr); }

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

void gg_free(gg_graph* g) {
  if (!g) return;
  free(g->off);
  free(g->adj);
  free(g);
}

/*
 * Clean a list of (src[i], dst[i]) pairs over vertices [0,n) into CSR.
 * Pairs with an endpoint outside [0,n) are dropped too. Returns NULL on OOM.
 */
gg_graph* gg_clean_pairs(int64_t n, int64_t npairs, const int32_t* src, const int32_t* dst) {
  gg_graph* g = (gg_graph*)calloc(1, sizeof(gg_graph));
  if (!g) return NULL;
  g->n = n;
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) { free(g); return NULL; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < npairs; ++i) {
    int32_t u = src[i], v = dst[i];
    if (u == v || u < 0 || v < 0 || u >= n || v >= n) continue;
#pragma omp atomic
    cnt[u]++;
#pragma omp atomic
    cnt[v]++;
  }
  int64_t* pos = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!pos) { free(cnt); free(g); return NULL; }
  int64_t s = 0;
  for (int64_t v = 0; v < n; ++v) { pos[v] = s; s += cnt[v]; }
  pos[n] = s;
  int32_t* tmp = (int32_t*)malloc((size_t)(s > 0 ? s : 1) * sizeof(int32_t));
  int64_t* fill = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!tmp || !fill) { free(cnt); free(pos); free(tmp); free(fill); free(g); return NULL; }
  memcpy(fill, pos, ((size_t)n + 1) * sizeof(int64_t));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < npairs; ++i) {
    int32_t u = src[i], v = dst[i];
    if (u == v || u < 0 || v < 0 || u >= n || v >= n) continue;
    int64_t pu, pv;
#pragma omp atomic capture
    pu = fill[u]++;
#pragma omp atomic capture
    pv = fill[v]++;
    tmp[pu] = v;
    tmp[pv] = u;
  }
  free(fill);
  /* sort and dedup each list in place; cnt[v] becomes the unique count */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < n; ++v) {
    int64_t b = pos[v], e = pos[v + 1];
    if (e - b > 1) qsort(tmp + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
    int64_t w = b;
    for (int64_t i = b; i < e; ++i)
      if (i == b || tmp[i] != tmp[i - 1]) tmp[w++] = tmp[i];
    cnt[v] = w - b;
  }
  g->off = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!g->off) { free(cnt); free(pos); free(tmp); free(g); return NULL; }
  s = 0;
  for (int64_t v = 0; v < n; ++v) { g->off[v] = s; s += cnt[v]; }
  g->off[n] = s;
  g->arcs = s;
  g->adj = (int32_t*)malloc((size_t)(s > 0 ? s : 1) * sizeof(int32_t));
  if (!g->adj) { free(cnt); free(pos); free(tmp); free(g->off); free(g); return NULL; }
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; ++v)
    memcpy(g->adj + g->off[v], tmp + pos[v], (size_t)cnt[v] * sizeof(int32_t));
  free(cnt);
  free(pos);
  free(tmp);
  return g;
}

/* Seeded Fisher-Yates permutation of [0,n): perm[old id] = new id. */
int gg_permutation(int64_t n, uint64_t seed, int32_t* perm) {
  uint64_t key = gg_key(seed, 0x7065726D); /* "perm" */
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    uint64_t j = gg_draw(key, (uint64_t)i) % (uint64_t)(i + 1);
    int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
  return 0;
}

/* Raw R-MAT samples (before cleaning); src/dst hold edgefactor << scale pairs. */
int gg_rmat_pairs(int scale, int64_t edgefactor, double a, double b, double c, uint64_t seed,
                  int permute, int32_t* src, int32_t* dst) {
  if (scale < 1 || scale > 30 || edgefactor < 1) return -1;
  if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
  const int64_t n = (int64_t)1 << scale;
  const int64_t ns = edgefactor << scale;
  const uint64_t key = gg_key(seed, 0x726D6174); /* "rmat" */
  const double two32 = 4294967296.0;
  const uint64_t ta = (uint64_t)(a * two32);
  const uint64_t tab = (uint64_t)((a + b) * two32);
  const uint64_t tabc = (uint64_t)((a + b + c) * two32);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < ns; ++i) {
    uint32_t u = 0, v = 0;
    uint64_t r = 0;
    for (int l = 0; l < scale; ++l) {
      uint64_t x;
      if ((l & 1) == 0) {
        r = gg_draw(key, (uint64_t)i * 16u + (uint64_t)(l >> 1));
        x = r >> 32;
      } else {
        x = r & 0xFFFFFFFFULL;
      }
      uint32_t sb, db;
      if (x < ta) { sb = 0; db = 0; }
      else if (x < tab) { sb = 0; db = 1; }
      else if (x < tabc) { sb = 1; db = 0; }
      else { sb = 1; db = 1; }
      u = (u << 1) | sb;
      v = (v << 1) | db;
    }
    src[i] = (int32_t)u;
    dst[i] = (int32_t)v;
  }
  if (permute) {
    int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!perm) return -2;
    gg_permutation(n, seed, perm);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ns; ++i) {
      src[i] = perm[src[i]];
      dst[i] = perm[dst[i]];
    }
    free(perm);
  }
  return 0;
}

gg_graph* gg_rmat(int scale, int64_t edgefactor, double a, double b, double c, uint64_t seed,
                  int permute) {
  if (scale < 1 || scale > 30 || edgefactor < 1) return NULL;
  const int64_t ns = edgefactor << scale;
  int32_t* src = (int32_t*)malloc((size_t)ns * sizeof(int32_t));
  int32_t* dst = (int32_t*)malloc((size_t)ns * sizeof(int32_t));
  if (!src || !dst) { free(src); free(dst); return NULL; }
  if (gg_rmat_pairs(scale, edgefactor, a, b, c, seed, permute, src, dst) != 0) {
    free(src); free(dst); return NULL;
  }
  gg_graph* g = gg_clean_pairs((int64_t)1 << scale, ns, src, dst);
  free(src);
  free(dst);
  return g;
}

/* Pairs of one SBM region by geometric skipping. Region (bi,bj), bi<=bj. */
typedef struct { int32_t* u; int32_t* v; int64_t len, cap; } gg_pairbuf;

static int pb_push(gg_pairbuf* p, int32_t u, int32_t v) {
  if (p->len == p->cap) {
    int64_t nc = p->cap ? p->cap * 2 : 256;
    int32_t* nu = (int32_t*)realloc(p->u, (size_t)nc * sizeof(int32_t));
    if (!nu) return -1;
    p->u = nu;
    int32_t* nv = (int32_t*)realloc(p->v, (size_t)nc * sizeof(int32_t));
    if (!nv) return -1;
    p->v = nv;
    p->cap = nc;
  }
  p->u[p->len] = u;
  p->v[p->len] = v;
  p->len++;
  return 0;
}

/* Number of failures before the next success of a Bernoulli(p) sequence. */
static inline int64_t geo_skip(uint64_t key, uint64_t ctr, double log1mp) {
  double U = gg_unit(key, ctr);
  double k = floor(log1p(-U) / log1mp);
  if (!(k < 9.0e18)) return INT64_MAX / 4;
  return (int64_t)k;
}

static int sbm_region(int64_t s0, int64_t s1, int64_t t0, int64_t t1, int same, double p,
                      uint64_t key, gg_pairbuf* out) {
  if (p <= 0.0) return 0;
  int64_t rows = s1 - s0, cols = t1 - t0;
  if (rows <= 0 || cols <= 0) return 0;
  if (p >= 1.0) {
    for (int64_t x = 0; x < rows; ++x)
      for (int64_t y = same ? x + 1 : 0; y < cols; ++y)
        if (pb_push(out, (int32_t)(s0 + x), (int32_t)(t0 + y))) return -1;
    return 0;
  }
  const double log1mp = log1p(-p);
  uint64_t ctr = 0;
  if (!same) {
    const int64_t total = rows * cols;
    int64_t k = geo_skip(key, ctr++, log1mp);
    while (k < total) {
      if (pb_push(out, (int32_t)(s0 + k / cols), (int32_t)(t0 + k % cols))) return -1;
      k += 1 + geo_skip(key, ctr++, log1mp);
    }
  } else {
    /* upper triangle, row by row: row x has columns x+1 .. rows-1 */
    int64_t x = 0, y = 1;
    int64_t skip = geo_skip(key, ctr++, log1mp);
    while (x < rows - 1) {
      int64_t left = rows - y; /* columns remaining in row x from y */
      if (skip >= left) { skip -= left; ++x; y = x + 1; continue; }
      y += skip;
      if (pb_push(out, (int32_t)(s0 + x), (int32_t)(s0 + y))) return -1;
      ++y;
      if (y >= rows) { ++x; y = x + 1; }
      skip = geo_skip(key, ctr++, log1mp);
    }
  }
  return 0;
}

gg_graph* gg_sbm(int64_t n, int64_t blocks, double p_in, double p_out, uint64_t seed) {
  if (n < 0 || n > 0x7FFFFFFF || blocks < 1 || blocks > n) return NULL;
  const int64_t B = blocks;
  const int64_t R = B * (B + 1) / 2;
  gg_pairbuf* bufs = (gg_pairbuf*)calloc((size_t)R, sizeof(gg_pairbuf));
  if (!bufs) return NULL;
  const uint64_t key = gg_key(seed, 0x73626D); /* "sbm" */
  int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
  for (int64_t r = 0; r < R; ++r) {
    /* region r -> (bi, bj), bi <= bj, row-major over the upper triangle */
    int64_t bi = 0, rem = r;
    while (rem >= B - bi) { rem -= B - bi; ++bi; }
    int64_t bj = bi + rem;
    int64_t s0 = bi * n / B, s1 = (bi + 1) * n / B;
    int64_t t0 = bj * n / B, t1 = (bj + 1) * n / B;
    uint64_t rkey = gg_mix64(key ^ ((uint64_t)r * GG_GAMMA + 0x51ED2701ULL));
    fail |= sbm_region(s0, s1, t0, t1, bi == bj, bi == bj ? p_in : p_out, rkey, &bufs[r]) != 0;
  }
  gg_graph* g = NULL;
  if (!fail) {
    int64_t tot = 0;
    for (int64_t r = 0; r < R; ++r) tot += bufs[r].len;
    int32_t* su = (int32_t*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
    int32_t* sv = (int32_t*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
    if (su && sv) {
      int64_t w = 0;
      for (int64_t r = 0; r < R; ++r) {
        memcpy(su + w, bufs[r].u, (size_t)bufs[r].len * sizeof(int32_t));
        memcpy(sv + w, bufs[r].v, (size_t)bufs[r].len * sizeof(int32_t));
        w += bufs[r].len;
      }
      g = gg_clean_pairs(n, tot, su, sv);
    }
    free(su);
    free(sv);
  }
  for (int64_t r = 0; r < R; ++r) { free(bufs[r].u); free(bufs[r].v); }
  free(bufs);
  return g;
}

/* Accessors for ctypes. */
int64_t gg_n(const gg_graph* g) { return g ? g->n : -1; }
int64_t gg_arcs(const gg_graph* g) { return g ? g->arcs : -1; }
int gg_copy_out(const gg_graph* g, int64_t* off, int32_t* adj) {
  if (!g) return -1;
  memcpy(off, g->off, ((size_t)g->n + 1) * sizeof(int64_t));
  if (g->arcs) memcpy(adj, g->adj, (size_t)g->arcs * sizeof(int32_t));
  return 0;
}

int gg_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
  return omp_get_max_threads();
#else
  (void)t;
  return 1;
#endif
}
