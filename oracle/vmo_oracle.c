/*
 * Plain CPU oracle for visual matrix ordering (VMO), Fagginger Auer and
 * Bisseling, "A Geometric Approach to Matrix Ordering".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent, slow, obviously
 * correct restatement of the method that the GPU library is checked against.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it; the product path never does.  It shares no code, header
 * or constant table with the CUDA library.
 *
 * Precision: floating point state is FP64 (the paper fixes none), except where
 * a floating point value decides an integer (a grid cell, a 2-means label, a
 * separator choice).  There the decision is taken in IEEE binary32 with a fixed
 * operation order and no fused multiply-add, the precision of the paper's own
 * float4 implementation (Sec. 5), so that both implementations take the same
 * decision from the same fp32 inputs.  Compile with -ffp-contract=off.
 *
 * Every function cites the passage of the paper it follows.  Readings of
 * passages the paper leaves open are stated where they are used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_EXPORT __attribute__((visibility("default")))

/* Threads of the per-vertex loops (OpenMP when built with it).  Every vertex's
 * sums are taken by one thread in a fixed order, so results do not depend on
 * the thread count. */
ORA_EXPORT void ora_set_threads(int32_t n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

ORA_EXPORT int32_t ora_get_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Random numbers: the SplitMix64 output function (Steele, Lea, Flood 2014),  */
/* used as a counter-based generator keyed by (seed, a, b).                   */
/* ------------------------------------------------------------------------- */
static const uint64_t ORA_GOLDEN = 0x9E3779B97F4A7C15ull;
static const uint64_t ORA_TAG_COORD = 0x636f6f7264000000ull; /* initial layout */
static const uint64_t ORA_TAG_KMEANS = 0x6b6d65616e730000ull; /* k-means++ draws */

static uint64_t ora_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

ORA_EXPORT uint64_t ora_rand64(uint64_t seed, uint64_t a, uint64_t b) {
  return ora_mix64(ora_mix64(seed + ORA_GOLDEN * (a + 1)) + ORA_GOLDEN * (b + 1));
}

/* floor(n * r / 2^64): a uniform index in [0, n) from a 64-bit draw r. */
static uint64_t ora_scale_draw(uint64_t n, uint64_t r) {
  return (uint64_t)(((unsigned __int128)n * (unsigned __int128)r) >> 64);
}

ORA_EXPORT void ora_free(void* p) { free(p); }

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------- */
/* Hypergraph models of a sparse matrix (Table 1, Sec. 1.1).                  */
/*                                                                            */
/* Every model is returned as nets (net_ptr/pins, pins of a net ascending)    */
/* and the vertex-to-net incidence (vtx_ptr/vnets, nets of a vertex           */
/* ascending).  Graph models (symmetric, bipartite) also return the vertex    */
/* adjacency (adj_ptr/adj, neighbours ascending); their nets are the edges,   */
/* listed in lexicographic order of (smaller end, larger end).                */
/*                                                                            */
/* Readings: a collection of nets is a set, so a pair {i,j} given by a_ij and */
/* a_ji (or by duplicate entries) is one net; in the symmetric model the      */
/* diagonal gives singleton nets {i}, which exert no force (x_i = z_j) and    */
/* are dropped.  Unit vertex weights and net costs.                           */
/*   model 0 symmetric : V = {0..m-1}, E = {{i,j} : a_ij != 0, i != j}        */
/*   model 1 bipartite : V = rows 0..m-1, columns m..m+n-1, E = {{r_i,c_j}}   */
/*   model 2 row-net   : V = columns, net i = {c_j : a_ij != 0}               */
/*   model 3 col-net   : V = rows, net j = {r_i : a_ij != 0}                  */
/*   model 4 finegrain : V = the distinct entries v_ij in row-major order,    */
/*                       net i = {v_ij : j} (rows), net m+j = {v_ij : i}      */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t model, k, l; /* vertices, nets */
  int32_t* net_ptr;    /* l+1 */
  int32_t* pins;       /* net_ptr[l] */
  int32_t* vtx_ptr;    /* k+1 */
  int32_t* vnets;      /* vtx_ptr[k] */
  int32_t* adj_ptr;    /* k+1, graph models only (else NULL) */
  int32_t* adj;        /* adj_ptr[k] */
} ora_hg;

ORA_EXPORT void ora_hg_free(ora_hg* h) {
  free(h->net_ptr); free(h->pins); free(h->vtx_ptr); free(h->vnets);
  free(h->adj_ptr); free(h->adj);
  memset(h, 0, sizeof(*h));
}

/* Transposes a list of (a, b) pairs given as sorted 64-bit keys a*nb+b into
 * CSR of b -> a (a ascending within each b).  */
static void ora_incidence(int32_t na, int32_t nb, const int64_t* keys, int64_t nkeys,
                          int32_t** ptr_out, int32_t** idx_out) {
  int32_t* ptr = (int32_t*)calloc((size_t)nb + 1, sizeof(int32_t));
  int32_t* idx = (int32_t*)malloc((size_t)(nkeys > 0 ? nkeys : 1) * sizeof(int32_t));
  int32_t* fill = (int32_t*)calloc((size_t)nb + 1, sizeof(int32_t));
  for (int64_t t = 0; t < nkeys; ++t) ptr[keys[t] % nb + 1]++;
  for (int32_t b = 0; b < nb; ++b) ptr[b + 1] += ptr[b];
  for (int64_t t = 0; t < nkeys; ++t) { /* keys ascending => a ascending per b */
    int32_t a = (int32_t)(keys[t] / nb), b = (int32_t)(keys[t] % nb);
    idx[ptr[b] + fill[b]++] = a;
  }
  (void)na;
  free(fill);
  *ptr_out = ptr; *idx_out = idx;
}

/* Builds CSR a -> b from sorted keys a*nb+b. */
static void ora_rows(int32_t na, int32_t nb, const int64_t* keys, int64_t nkeys,
                     int32_t** ptr_out, int32_t** idx_out) {
  int32_t* ptr = (int32_t*)calloc((size_t)na + 1, sizeof(int32_t));
  int32_t* idx = (int32_t*)malloc((size_t)(nkeys > 0 ? nkeys : 1) * sizeof(int32_t));
  for (int64_t t = 0; t < nkeys; ++t) {
    ptr[keys[t] / nb + 1]++;
    idx[t] = (int32_t)(keys[t] % nb);
  }
  for (int32_t a = 0; a < na; ++a) ptr[a + 1] += ptr[a];
  *ptr_out = ptr; *idx_out = idx;
}

static int64_t ora_sort_unique(int64_t* keys, int64_t n) {
  if (n == 0) return 0;
  qsort(keys, (size_t)n, sizeof(int64_t), cmp_i64);
  int64_t u = 1;
  for (int64_t t = 1; t < n; ++t)
    if (keys[t] != keys[u - 1]) keys[u++] = keys[t];
  return u;
}

ORA_EXPORT int ora_build(int32_t model, int32_t m, int32_t n, const int32_t* rowptr,
                         const int32_t* colidx, ora_hg* out) {
  memset(out, 0, sizeof(*out));
  out->model = model;
  int64_t nnz = rowptr[m];
  if (model == 0 || model == 1) {
    /* Graph models: the edge set as sorted unique keys lo*k+hi. */
    int32_t k = (model == 0) ? m : m + n;
    int64_t* e = (int64_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    int64_t ne = 0;
    for (int32_t i = 0; i < m; ++i)
      for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
        int32_t j = colidx[t];
        int64_t u = i, v = (model == 0) ? j : (int64_t)m + j;
        if (u == v) continue; /* singleton net of the diagonal */
        int64_t lo = u < v ? u : v, hi = u < v ? v : u;
        e[ne++] = lo * k + hi;
      }
    ne = ora_sort_unique(e, ne);
    out->k = k; out->l = (int32_t)ne;
    out->net_ptr = (int32_t*)malloc((size_t)(ne + 1) * sizeof(int32_t));
    out->pins = (int32_t*)malloc((size_t)(2 * ne > 0 ? 2 * ne : 1) * sizeof(int32_t));
    for (int64_t t = 0; t < ne; ++t) {
      out->net_ptr[t] = (int32_t)(2 * t);
      out->pins[2 * t] = (int32_t)(e[t] / k);
      out->pins[2 * t + 1] = (int32_t)(e[t] % k);
    }
    out->net_ptr[ne] = (int32_t)(2 * ne);
    /* vertex -> nets: keys (vertex, net) */
    int64_t* vn = (int64_t*)malloc((size_t)(2 * ne > 0 ? 2 * ne : 1) * sizeof(int64_t));
    int64_t* aj = (int64_t*)malloc((size_t)(2 * ne > 0 ? 2 * ne : 1) * sizeof(int64_t));
    for (int64_t t = 0; t < ne; ++t) {
      int64_t a = e[t] / k, b = e[t] % k;
      vn[2 * t] = a * (ne > 0 ? ne : 1) + t;
      vn[2 * t + 1] = b * (ne > 0 ? ne : 1) + t;
      aj[2 * t] = a * k + b;
      aj[2 * t + 1] = b * k + a;
    }
    qsort(vn, (size_t)(2 * ne), sizeof(int64_t), cmp_i64);
    qsort(aj, (size_t)(2 * ne), sizeof(int64_t), cmp_i64);
    ora_rows(k, (int32_t)(ne > 0 ? ne : 1), vn, 2 * ne, &out->vtx_ptr, &out->vnets);
    ora_rows(k, k, aj, 2 * ne, &out->adj_ptr, &out->adj);
    free(vn); free(aj); free(e);
    return 0;
  }
  if (model == 2 || model == 3) {
    /* Sorted unique (row, col) keys. */
    int64_t* key = (int64_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    for (int32_t i = 0; i < m; ++i)
      for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) key[t] = (int64_t)i * n + colidx[t];
    int64_t u = ora_sort_unique(key, nnz);
    if (model == 2) { /* vertices = columns, nets = rows */
      out->k = n; out->l = m;
      ora_rows(m, n, key, u, &out->net_ptr, &out->pins);
      ora_incidence(m, n, key, u, &out->vtx_ptr, &out->vnets);
    } else { /* vertices = rows, nets = columns */
      out->k = m; out->l = n;
      ora_rows(m, n, key, u, &out->vtx_ptr, &out->vnets);
      ora_incidence(m, n, key, u, &out->net_ptr, &out->pins);
    }
    free(key);
    return 0;
  }
  if (model == 4) {
    int64_t* key = (int64_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    for (int32_t i = 0; i < m; ++i)
      for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) key[t] = (int64_t)i * n + colidx[t];
    int64_t u = ora_sort_unique(key, nnz); /* vertex t = the t-th distinct entry */
    out->k = (int32_t)u; out->l = m + n;
    /* (net, vertex) pairs: v_ij lies on row net i and column net m + j */
    int64_t* nv = (int64_t*)malloc((size_t)(2 * u > 0 ? 2 * u : 1) * sizeof(int64_t));
    for (int64_t t = 0; t < u; ++t) {
      int64_t i = key[t] / n, j = key[t] % n;
      nv[2 * t] = i * (u > 0 ? u : 1) + t;
      nv[2 * t + 1] = ((int64_t)m + j) * (u > 0 ? u : 1) + t;
    }
    qsort(nv, (size_t)(2 * u), sizeof(int64_t), cmp_i64);
    ora_rows(m + n, (int32_t)(u > 0 ? u : 1), nv, 2 * u, &out->net_ptr, &out->pins);
    ora_incidence(m + n, (int32_t)(u > 0 ? u : 1), nv, 2 * u, &out->vtx_ptr, &out->vnets);
    free(nv); free(key);
    return 0;
  }
  return 1;
}

/* Finegrain coordinates from the bipartite layout (Sec. 4.2): the dual of the
 * finegrain hypergraph is the bipartite graph, and every entry a_ij is placed
 * at the mean of the points of its row r_i and its column c_j.  fg: the
 * finegrain model; xb: bipartite coordinates (rows 0..m-1, columns m..),
 * 4 floats per vertex; xf: 4 doubles per entry. */
ORA_EXPORT void ora_finegrain_coords(const ora_hg* fg, const float* xb, double* xf) {
  for (int32_t t = 0; t < fg->k; ++t) {
    int32_t r = fg->vnets[fg->vtx_ptr[t]], c = fg->vnets[fg->vtx_ptr[t] + 1];
    for (int q = 0; q < 4; ++q)
      xf[4 * (int64_t)t + q] = 0.5 * ((double)xb[4 * (int64_t)r + q] + (double)xb[4 * (int64_t)c + q]);
  }
}

/* Dual hypergraph (Definition 1.2): V* = E and E* = {{e : e contains v} : v in V}.
 * Input nets (k vertices, l nets); output nets of G* (l vertices, k nets). */
ORA_EXPORT void ora_dual(int32_t k, int32_t l, const int32_t* net_ptr, const int32_t* pins,
                         int32_t** dptr, int32_t** dpins) {
  int64_t np_ = net_ptr[l];
  int32_t* ptr = (int32_t*)calloc((size_t)k + 1, sizeof(int32_t));
  int32_t* out = (int32_t*)malloc((size_t)(np_ > 0 ? np_ : 1) * sizeof(int32_t));
  for (int32_t v = 0; v < k; ++v) {          /* net of G* belonging to vertex v */
    ptr[v + 1] = ptr[v];
    for (int32_t e = 0; e < l; ++e)          /* every net of G that contains v */
      for (int32_t t = net_ptr[e]; t < net_ptr[e + 1]; ++t)
        if (pins[t] == v) { out[ptr[v + 1]++] = e; break; }
  }
  *dptr = ptr; *dpins = out;
}

/* ------------------------------------------------------------------------- */
/* Connected components, Algorithm 1 (Sec. 2.3), written as the paper gives   */
/* it: a forest of parent pointers, trees of all pins of a net merged under   */
/* the smallest root, then every vertex attached directly to its root.  The   */
/* label of a component is its smallest vertex id.                            */
/* ------------------------------------------------------------------------- */
ORA_EXPORT void ora_components(int32_t k, int32_t l, const int32_t* net_ptr, const int32_t* pins,
                               int32_t* p) {
  for (int32_t v = 0; v < k; ++v) p[v] = v;
  for (int32_t e = 0; e < l; ++e) {
    for (int32_t t = net_ptr[e]; t < net_ptr[e + 1]; ++t) {
      int32_t v = pins[t];
      while (p[v] != p[p[v]]) p[v] = p[p[v]];
    }
    if (net_ptr[e] == net_ptr[e + 1]) continue;
    int32_t pm = p[pins[net_ptr[e]]];
    for (int32_t t = net_ptr[e]; t < net_ptr[e + 1]; ++t)
      if (p[pins[t]] < pm) pm = p[pins[t]];
    for (int32_t t = net_ptr[e]; t < net_ptr[e + 1]; ++t) p[p[pins[t]]] = pm;
  }
  for (int32_t v = 0; v < k; ++v)
    while (p[v] != p[p[v]]) p[v] = p[p[v]];
}

/* ------------------------------------------------------------------------- */
/* Random initial layout (Algorithm 3, lines on the coarsest level): every    */
/* coordinate uniform in [0, s) with s the smallest integer with s^d >= k     */
/* (reading: unit point density).  u = (r >> 40) * 2^-24 is exact in fp32 and */
/* the coordinate is the fp32 product u * s.                                  */
/* ------------------------------------------------------------------------- */
ORA_EXPORT int32_t ora_init_side(int32_t k, int32_t d) {
  int64_t s = 1;
  for (;;) {
    int64_t p = 1;
    for (int i = 0; i < d; ++i) p *= s;
    if (p >= k) return (int32_t)s;
    ++s;
  }
}

ORA_EXPORT void ora_init_coords(int32_t k, int32_t d, uint64_t seed, float* x /* k*4 */) {
  float side = (float)ora_init_side(k, d);
  for (int32_t v = 0; v < k; ++v)
    for (int m = 0; m < 4; ++m) {
      if (m >= d) { x[4 * v + m] = 0.0f; continue; }
      uint64_t r = ora_rand64(seed ^ ORA_TAG_COORD, (uint64_t)v, (uint64_t)m);
      float u = (float)(r >> 40) * 0x1p-24f;
      x[4 * v + m] = u * side;
    }
}

/* ------------------------------------------------------------------------- */
/* Energy (eq. graphenergysimple, Sec. 2.1, alpha = beta = 1, gamma = 2,      */
/* delta = d - 2), used by the descent and finite-difference checks.          */
/* Reading for d = 2 (the paper requires d >= 3): the repulsion term is the   */
/* harmonic kernel of the plane, -1/2 sum_{i != j} w_i w_j log||x_i - x_j||,  */
/* the limit of (r^-(d-2) - 1)/(d-2) as d -> 2; its gradient has the same     */
/* form as eq. graphenergygradientsimple with the factor (d-2) replaced by 1. */
/* ------------------------------------------------------------------------- */
static double ora_kappa(int d) { return d == 2 ? 1.0 : (double)(d - 2); }

ORA_EXPORT double ora_energy(const ora_hg* h, int32_t d, const double* x /* k*4 */,
                             const double* w /* k or NULL */, const double* c /* l or NULL */) {
  double f = 0.0;
  for (int32_t j = 0; j < h->l; ++j) {
    int32_t a = h->net_ptr[j], b = h->net_ptr[j + 1];
    if (b == a) continue;
    double z[4] = {0, 0, 0, 0};
    for (int32_t t = a; t < b; ++t)
      for (int m = 0; m < d; ++m) z[m] += x[4 * h->pins[t] + m];
    for (int m = 0; m < d; ++m) z[m] /= (double)(b - a);
    double s = 0.0;
    for (int32_t t = a; t < b; ++t)
      for (int m = 0; m < d; ++m) {
        double q = x[4 * h->pins[t] + m] - z[m];
        s += q * q;
      }
    f += 0.5 * (c ? c[j] : 1.0) * s;
  }
  for (int32_t i = 0; i < h->k; ++i)
    for (int32_t j = 0; j < h->k; ++j) {
      if (i == j) continue;
      double r2 = 0.0;
      for (int m = 0; m < d; ++m) {
        double q = x[4 * i + m] - x[4 * j + m];
        r2 += q * q;
      }
      double ww = (w ? w[i] : 1.0) * (w ? w[j] : 1.0);
      if (d == 2) f -= 0.5 * ww * 0.5 * log(r2);
      else f += 0.5 * ww * pow(r2, -0.5 * (d - 2));
    }
  return f;
}

/* ------------------------------------------------------------------------- */
/* Grid pyramid standing in for the tree of Algorithm 4 (Sec. 2.3).           */
/*                                                                            */
/* Reading of "build tree T recursively clustering x" and "far away": a       */
/* uniform-grid pyramid over the bounding cube of the layout.  With the fp32  */
/* bounding box lo/hi and E = max extent, the finest level is the smallest    */
/* L >= 1 with occ * 2^(dL) >= k, capped at Lmax(d) = 15, 10, 7 for d = 2,3,4. */
/* The level-L cell of a point is c_m = min(2^L - 1, floor((x_m - lo_m) * s))  */
/* with s = 2^L / E, all in fp32 without FMA; the level-l cell is c >> (L-l). */
/* A cell's charge sits at the weighted mean of its points with their summed   */
/* weight (Sec. 2.3).  For a target point n the sources are:                  */
/*   near: every other point whose level-L cell is adjacent or equal          */
/*         (Chebyshev distance <= 1) to n's level-L cell, exactly;            */
/*   far:  at each level l = 2..L, every cell whose parent is adjacent or     */
/*         equal to n's level-(l-1) cell but which is not adjacent or equal   */
/*         to n's level-l cell, as one charge.                                */
/* The level-L cell index (row-major, coordinate 0 fastest) is the key of a  */
/* point.                                                                     */
/* Every other point is counted exactly once (in the coarsest level where its */
/* cell stops being adjacent to n's cell, or in the near field).              */
/* Pairs at distance 0 contribute nothing (they lie outside U of Def. 2.1).   */
/* ------------------------------------------------------------------------- */
static int ora_lmax(int d) { return d == 2 ? 15 : (d == 3 ? 10 : 7); }

ORA_EXPORT int32_t ora_levels(int32_t k, int32_t d, int32_t occ) {
  int L = 1;
  while (L < ora_lmax(d) && (int64_t)occ * (1ll << (d * L)) < (int64_t)k) ++L;
  return L;
}

/* Index of a level-`bits` cell: row-major with coordinate 0 fastest,
 * sum_m c_m 2^(bits m).  The level-L index is the sort key of a point. */
static uint32_t ora_cellidx(const int32_t* c, int d, int bits) {
  uint32_t key = 0;
  for (int m = d - 1; m >= 0; --m) key = (key << bits) | (uint32_t)c[m];
  return key;
}

/* Cell coordinates at the finest level, decided in fp32 (see above). */
static void ora_cells(int32_t k, int d, int L, const float* xf /* k*4 */, int32_t* cell /* k*4 */,
                      float* lo_out, float* hi_out) {
  float lo[4], hi[4];
  for (int m = 0; m < d; ++m) { lo[m] = INFINITY; hi[m] = -INFINITY; }
  for (int32_t v = 0; v < k; ++v)
    for (int m = 0; m < d; ++m) {
      float q = xf[4 * v + m];
      if (q < lo[m]) lo[m] = q;
      if (q > hi[m]) hi[m] = q;
    }
  float E = 0.0f;
  for (int m = 0; m < d; ++m) {
    float ext = hi[m] - lo[m];
    if (ext > E) E = ext;
  }
  float s = (E > 0.0f) ? (float)(1 << L) / E : 0.0f;
  int32_t cmax = (1 << L) - 1;
  for (int32_t v = 0; v < k; ++v)
    for (int m = 0; m < 4; ++m) {
      if (m >= d) { cell[4 * v + m] = 0; continue; }
      float t = (xf[4 * v + m] - lo[m]) * s;
      int32_t c = (int32_t)floorf(t);
      cell[4 * v + m] = c < cmax ? c : cmax;
    }
  for (int m = 0; m < d; ++m) { lo_out[m] = lo[m]; hi_out[m] = hi[m]; }
}

/* Diagnostics of one gradient evaluation, for the checks on the interaction
 * lists: number of sources (points plus charges) and their summed weight. */
typedef struct {
  int64_t* n_inter;   /* k or NULL */
  double* w_seen;     /* k or NULL */
} ora_diag;

/* Gradient y = df/dx of eq. graphenergygradientsimple with the repulsion sum
 * approximated on the grid pyramid.  Also returns the level-L Morton key of
 * every vertex (the GPU must reproduce these bit for bit). */
/* |r|^(-d) from r2 = |r|^2, the kernel of the repulsion term of eq.
 * graphenergygradientsimple (d = 2: the planar reading 1/r^2). */
static double ora_rpow(double r2, int d) {
  if (d == 2) return 1.0 / r2;
  if (d == 3) return 1.0 / (r2 * sqrt(r2));
  return 1.0 / (r2 * r2);
}

ORA_EXPORT int ora_gradient(const ora_hg* h, int32_t d, int32_t occ, const double* x /* k*4 */,
                            const double* w, const double* c, double* y /* k*4 */,
                            uint32_t* keys /* k or NULL */, int32_t* L_out, ora_diag* diag) {
  int32_t k = h->k;
  for (int64_t t = 0; t < 4 * (int64_t)k; ++t) y[t] = 0.0;
  /* Rubber bands (Algorithm 4, net centres then per-vertex sums). */
  for (int32_t j = 0; j < h->l; ++j) {
    int32_t a = h->net_ptr[j], b = h->net_ptr[j + 1];
    if (b == a) continue;
    double z[4] = {0, 0, 0, 0};
    for (int32_t t = a; t < b; ++t)
      for (int m = 0; m < d; ++m) z[m] += x[4 * h->pins[t] + m];
    for (int m = 0; m < d; ++m) z[m] /= (double)(b - a);
    double cj = c ? c[j] : 1.0;
    for (int32_t t = a; t < b; ++t)
      for (int m = 0; m < d; ++m) y[4 * h->pins[t] + m] += cj * (x[4 * h->pins[t] + m] - z[m]);
  }
  if (k == 0) { *L_out = 1; return 0; }
  /* Grid pyramid. */
  int L = ora_levels(k, d, occ);
  *L_out = L;
  float* xf = (float*)malloc((size_t)k * 4 * sizeof(float));
  int32_t* cell = (int32_t*)malloc((size_t)k * 4 * sizeof(int32_t));
  for (int64_t t = 0; t < 4 * (int64_t)k; ++t) xf[t] = (float)x[t];
  float lo[4], hi[4];
  ora_cells(k, d, L, xf, cell, lo, hi);
  if (keys)
    for (int32_t v = 0; v < k; ++v) keys[v] = ora_cellidx(&cell[4 * v], d, L);
  /* Dense per-level tables of (sum w, sum w x), FP64. */
  int64_t* off = (int64_t*)malloc((size_t)(L + 2) * sizeof(int64_t));
  off[0] = 0;
  for (int l = 0; l <= L; ++l) off[l + 1] = off[l] + (1ll << (d * l));
  double* W = (double*)calloc((size_t)off[L + 1], sizeof(double));
  double* S = (double*)calloc((size_t)off[L + 1] * 4, sizeof(double));
  for (int32_t v = 0; v < k; ++v) {
    double wv = w ? w[v] : 1.0;
    for (int l = 0; l <= L; ++l) {
      int32_t cl[4];
      for (int m = 0; m < d; ++m) cl[m] = cell[4 * v + m] >> (L - l);
      int64_t id = off[l] + ora_cellidx(cl, d, l);
      W[id] += wv;
      for (int m = 0; m < d; ++m) S[4 * id + m] += wv * x[4 * v + m];
    }
  }
  /* Members of each finest cell, ascending vertex id. */
  int64_t ncell = 1ll << (d * L);
  int32_t* head = (int32_t*)calloc((size_t)ncell + 1, sizeof(int32_t));
  int32_t* mem = (int32_t*)malloc((size_t)k * sizeof(int32_t));
  int32_t* fill = (int32_t*)calloc((size_t)ncell, sizeof(int32_t));
  for (int32_t v = 0; v < k; ++v) head[ora_cellidx(&cell[4 * v], d, L) + 1]++;
  for (int64_t q = 0; q < ncell; ++q) head[q + 1] += head[q];
  for (int32_t v = 0; v < k; ++v) {
    uint32_t q = ora_cellidx(&cell[4 * v], d, L);
    mem[head[q] + fill[q]++] = v;
  }
  double kap = ora_kappa(d);
  int nb = 1;
  for (int m = 0; m < d; ++m) nb *= 3;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
  for (int32_t n = 0; n < k; ++n) {
    double wn = w ? w[n] : 1.0;
    double F[4] = {0, 0, 0, 0};
    int64_t cnt = 0;
    double wseen = 0.0;
    /* near field: the 3^d cells around n's finest cell */
    for (int o = 0; o < nb; ++o) {
      int32_t cc[4];
      int oo = o, inside = 1;
      for (int m = 0; m < d; ++m) {
        cc[m] = cell[4 * n + m] + (oo % 3) - 1;
        oo /= 3;
        if (cc[m] < 0 || cc[m] >= (1 << L)) inside = 0;
      }
      if (!inside) continue;
      uint32_t q = ora_cellidx(cc, d, L);
      for (int32_t t = head[q]; t < head[q + 1]; ++t) {
        int32_t i = mem[t];
        if (i == n) continue;
        double dx[4], r2 = 0.0;
        for (int m = 0; m < d; ++m) { dx[m] = x[4 * i + m] - x[4 * n + m]; r2 += dx[m] * dx[m]; }
        double wi = w ? w[i] : 1.0;
        cnt++; wseen += wi;
        if (r2 == 0.0) continue;
        double g = wi * wn * ora_rpow(r2, d);
        for (int m = 0; m < d; ++m) F[m] += g * dx[m];
      }
    }
    /* far field: level l = 2..L, children of the cells around the parent cell */
    for (int l = 2; l <= L; ++l) {
      int32_t me[4], par[4];
      for (int m = 0; m < d; ++m) { me[m] = cell[4 * n + m] >> (L - l); par[m] = me[m] >> 1; }
      int nchild = 1 << d;
      for (int o = 0; o < nb; ++o) {
        int32_t pc[4];
        int oo = o, inside = 1;
        for (int m = 0; m < d; ++m) {
          pc[m] = par[m] + (oo % 3) - 1;
          oo /= 3;
          if (pc[m] < 0 || pc[m] >= (1 << (l - 1))) inside = 0;
        }
        if (!inside) continue;
        for (int ch = 0; ch < nchild; ++ch) {
          int32_t cc[4];
          int adjacent = 1;
          for (int m = 0; m < d; ++m) {
            cc[m] = 2 * pc[m] + ((ch >> m) & 1);
            int32_t diff = cc[m] - me[m];
            if (diff < -1 || diff > 1) adjacent = 0;
          }
          if (adjacent) continue;
          int64_t id = off[l] + ora_cellidx(cc, d, l);
          if (W[id] <= 0.0) continue;
          double dx[4], r2 = 0.0;
          for (int m = 0; m < d; ++m) {
            dx[m] = S[4 * id + m] / W[id] - x[4 * n + m];
            r2 += dx[m] * dx[m];
          }
          cnt++; wseen += W[id];
          if (r2 == 0.0) continue;
          double g = W[id] * wn * ora_rpow(r2, d);
          for (int m = 0; m < d; ++m) F[m] += g * dx[m];
        }
      }
    }
    for (int m = 0; m < d; ++m) y[4 * n + m] += kap * F[m];
    if (diag && diag->n_inter) diag->n_inter[n] = cnt;
    if (diag && diag->w_seen) diag->w_seen[n] = wseen;
  }
  free(xf); free(cell); free(off); free(W); free(S); free(head); free(mem); free(fill);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* One steepest-descent step of Algorithm 4 (Sec. 2.3).                       */
/*                                                                            */
/* Reading of the step-size rule ("compare the bounding box volume to the     */
/* individual gradients ... to prevent blowup ... then decrease the found     */
/* stepsize by multiplying it by 0.9", after Hu 2005): a step length s_t is   */
/* fixed from the bounding box when a level starts,                           */
/*   s_0 = sigma * Lbox / k^(1/d),  Lbox = (prod_m extent_m)^(1/d)             */
/* (the largest extent if one is zero), i.e. sigma times the mean point       */
/* spacing, and decays as s_{t+1} = 0.9 s_t.  Each vertex moves s_t along its */
/* own descent direction: x_n <- x_n - (s_t / ||y_n||) y_n (no move when      */
/* y_n = 0), so one large gradient cannot blow the layout up.                 */
/* ------------------------------------------------------------------------- */
ORA_EXPORT double ora_step0(int32_t k, int32_t d, double sigma, const double* x /* k*4 */) {
  if (k <= 0) return 0.0;
  double lo[4], hi[4];
  for (int m = 0; m < d; ++m) { lo[m] = INFINITY; hi[m] = -INFINITY; }
  for (int32_t v = 0; v < k; ++v)
    for (int m = 0; m < d; ++m) {
      if (x[4 * v + m] < lo[m]) lo[m] = x[4 * v + m];
      if (x[4 * v + m] > hi[m]) hi[m] = x[4 * v + m];
    }
  double vol = 1.0, emax = 0.0;
  int degenerate = 0;
  for (int m = 0; m < d; ++m) {
    double e = hi[m] - lo[m];
    if (e > emax) emax = e;
    if (e <= 0.0) degenerate = 1;
    vol *= e;
  }
  double Lbox = degenerate ? emax : pow(vol, 1.0 / d);
  return sigma * Lbox / pow((double)k, 1.0 / d);
}

ORA_EXPORT int ora_layout_step(const ora_hg* h, int32_t d, int32_t occ, const double* w, const double* c,
                               double* x /* k*4, updated */, double step, double* y /* k*4 */,
                               uint32_t* keys, int32_t* L_out) {
  int32_t k = h->k;
  ora_gradient(h, d, occ, x, w, c, y, keys, L_out, NULL);
  for (int32_t v = 0; v < k; ++v) {
    double s = 0.0;
    for (int m = 0; m < d; ++m) s += y[4 * v + m] * y[4 * v + m];
    if (s <= 0.0) continue;
    double a = step / sqrt(s);
    for (int m = 0; m < d; ++m) x[4 * v + m] -= a * y[4 * v + m];
  }
  return 0;
}

/* T steps of Algorithm 4 on one level (reading: "while we are not satisfied"
 * = a fixed number T of steps). */
ORA_EXPORT int ora_layout(const ora_hg* h, int32_t d, int32_t occ, double sigma, double decay,
                          int32_t iters, const double* w, const double* c, double* x) {
  double* y = (double*)malloc((size_t)(h->k > 0 ? h->k : 1) * 4 * sizeof(double));
  double s = ora_step0(h->k, d, sigma, x);
  int32_t L;
  for (int32_t t = 0; t < iters; ++t) {
    ora_layout_step(h, d, occ, w, c, x, s, y, NULL, &L);
    s *= decay;
  }
  free(y);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Multilevel layout, Algorithm 3 (Sec. 2.3), for graph models.               */
/*                                                                            */
/* Coarsening (reading of "a maximal matching constructed greedily from heavy */
/* hyperedges" in a form that does not depend on visiting order): R = 4       */
/* handshake rounds; in round r every unmatched vertex v proposes to the      */
/* unmatched neighbour u with the largest edge cost, ties broken by the       */
/* smaller h = rand(seed^MATCH, min(u,v)*2^32 + max(u,v), 256*level + r) and  */
/* then the smaller id; mutual proposals are matched.  Then every unmatched   */
/* vertex with exactly one neighbour joins that neighbour's group (the        */
/* paper's rule against stars).  Groups become coarse vertices, numbered in   */
/* ascending order of their anchor (the smaller id of a matched pair, else    */
/* the vertex itself); weights add, parallel edges merge with added costs,    */
/* edges inside a group vanish.  Coarsening stops when k <= 64, when a level  */
/* keeps more than 95% of the vertices (that level is dropped), or after 40   */
/* levels.                                                                    */
/*                                                                            */
/* Prolongation: x_{j-1}(v) = f * x_j(pi(v)) + jitter, f = (k_{j-1}/k_j)^(1/d) */
/* (keeps unit point density), jitter_m = 0.1 * (u - 1/2) with                */
/* u = (rand(seed^JITTER, v, 4*(j-1) + m) >> 40) * 2^-24.  The coarsest level */
/* starts from the random layout above.  Every level runs T steps.            */
/* ------------------------------------------------------------------------- */
static const uint64_t ORA_TAG_MATCH = 0x6d61746368000000ull;
static const uint64_t ORA_TAG_JITTER = 0x6a69747465720000ull;

typedef struct {
  int32_t k;
  int32_t* adj_ptr; int32_t* adj; double* acost; /* symmetric adjacency with edge costs */
  double* w;                                       /* vertex weights */
} ora_graph;

static void ora_graph_free(ora_graph* g) {
  free(g->adj_ptr); free(g->adj); free(g->acost); free(g->w);
  memset(g, 0, sizeof(*g));
}

/* Matching and grouping of one level; returns the coarse vertex count and
 * fills pi (fine vertex -> coarse vertex). */
ORA_EXPORT int32_t ora_match(int32_t k, const int32_t* adj_ptr, const int32_t* adj, const double* acost,
                             uint64_t seed, int32_t level, int32_t rounds, int32_t* mate, int32_t* pi) {
  int32_t* prop = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  for (int32_t v = 0; v < k; ++v) mate[v] = -1;
  for (int32_t r = 0; r < rounds; ++r) {
    for (int32_t v = 0; v < k; ++v) {
      prop[v] = -1;
      if (mate[v] >= 0) continue;
      double bc = 0.0;
      uint64_t bh = 0;
      for (int32_t t = adj_ptr[v]; t < adj_ptr[v + 1]; ++t) {
        int32_t u = adj[t];
        if (u == v || mate[u] >= 0) continue;
        uint64_t lo = (uint64_t)(u < v ? u : v), hi = (uint64_t)(u < v ? v : u);
        uint64_t h = ora_rand64(seed ^ ORA_TAG_MATCH, (lo << 32) | hi, (uint64_t)level * 256 + (uint64_t)r);
        int better = 0;
        if (prop[v] < 0) better = 1;
        else if (acost[t] > bc) better = 1;
        else if (acost[t] == bc && (h < bh || (h == bh && u < prop[v]))) better = 1;
        if (better) { prop[v] = u; bc = acost[t]; bh = h; }
      }
    }
    for (int32_t v = 0; v < k; ++v)
      if (prop[v] >= 0 && prop[prop[v]] == v) mate[v] = prop[v];
  }
  /* anchors: matched pair -> smaller id; unmatched single-neighbour vertex ->
   * anchor of its neighbour; other unmatched vertex -> itself */
  int32_t* anchor = prop; /* reuse */
  for (int32_t v = 0; v < k; ++v)
    anchor[v] = (mate[v] >= 0) ? (mate[v] < v ? mate[v] : v) : v;
  for (int32_t v = 0; v < k; ++v) {
    if (mate[v] >= 0) continue;
    if (adj_ptr[v + 1] - adj_ptr[v] != 1) continue;
    int32_t u = adj[adj_ptr[v]];
    if (u == v) continue;
    anchor[v] = (mate[u] >= 0) ? (mate[u] < u ? mate[u] : u) : u;
  }
  /* coarse ids in ascending anchor order */
  int32_t* id = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  int32_t kc = 0;
  for (int32_t v = 0; v < k; ++v) id[v] = -1;
  for (int32_t v = 0; v < k; ++v) id[anchor[v]] = 0;
  for (int32_t v = 0; v < k; ++v)
    if (id[v] == 0) id[v] = kc++ + 1; /* 1-based while marking */
  for (int32_t v = 0; v < k; ++v) pi[v] = id[anchor[v]] - 1;
  free(id); free(prop);
  return kc;
}

typedef struct { int64_t key; double cost; } ora_kc;
static int cmp_kc(const void* a, const void* b) {
  int64_t x = ((const ora_kc*)a)->key, y = ((const ora_kc*)b)->key;
  return (x > y) - (x < y);
}

/* Coarse graph of a grouping pi (weights and parallel edge costs added). */
static void ora_contract(const ora_graph* g, const int32_t* pi, int32_t kc, ora_graph* out) {
  memset(out, 0, sizeof(*out));
  out->k = kc;
  out->w = (double*)calloc((size_t)(kc > 0 ? kc : 1), sizeof(double));
  for (int32_t v = 0; v < g->k; ++v) out->w[pi[v]] += g->w[v];
  int64_t ne = g->adj_ptr[g->k];
  ora_kc* e = (ora_kc*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(ora_kc));
  int64_t n = 0;
  for (int32_t v = 0; v < g->k; ++v)
    for (int32_t t = g->adj_ptr[v]; t < g->adj_ptr[v + 1]; ++t) {
      int32_t a = pi[v], b = pi[g->adj[t]];
      if (a == b) continue;
      e[n].key = (int64_t)a * kc + b;
      e[n].cost = g->acost[t];
      ++n;
    }
  qsort(e, (size_t)n, sizeof(ora_kc), cmp_kc);
  out->adj_ptr = (int32_t*)calloc((size_t)kc + 1, sizeof(int32_t));
  out->adj = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  out->acost = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  int64_t u = 0;
  for (int64_t t = 0; t < n; ++t) {
    if (t > 0 && e[t].key == e[t - 1].key) { out->acost[u - 1] += e[t].cost; continue; }
    out->adj[u] = (int32_t)(e[t].key % kc);
    out->acost[u] = e[t].cost;
    out->adj_ptr[e[t].key / kc + 1]++;
    ++u;
  }
  for (int32_t a = 0; a < kc; ++a) out->adj_ptr[a + 1] += out->adj_ptr[a];
  free(e);
}

/* Hypergraph (nets = edges u < v, lexicographic) with per-net costs. */
static void ora_graph_hg(const ora_graph* g, ora_hg* h, double** cost_out) {
  memset(h, 0, sizeof(*h));
  h->model = 0; h->k = g->k;
  int64_t ne = 0;
  for (int32_t v = 0; v < g->k; ++v)
    for (int32_t t = g->adj_ptr[v]; t < g->adj_ptr[v + 1]; ++t)
      if (g->adj[t] > v) ne++;
  h->l = (int32_t)ne;
  h->net_ptr = (int32_t*)malloc((size_t)(ne + 1) * sizeof(int32_t));
  h->pins = (int32_t*)malloc((size_t)(2 * ne > 0 ? 2 * ne : 1) * sizeof(int32_t));
  double* c = (double*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(double));
  ne = 0;
  for (int32_t v = 0; v < g->k; ++v)
    for (int32_t t = g->adj_ptr[v]; t < g->adj_ptr[v + 1]; ++t)
      if (g->adj[t] > v) {
        h->net_ptr[ne] = (int32_t)(2 * ne);
        h->pins[2 * ne] = v; h->pins[2 * ne + 1] = g->adj[t];
        c[ne] = g->acost[t];
        ++ne;
      }
  h->net_ptr[ne] = (int32_t)(2 * ne);
  *cost_out = c;
}

/* Coarsening hierarchy only (for checks): returns the number of levels and
 * writes the vertex count of each level into ks (capacity 41). */
ORA_EXPORT int32_t ora_hierarchy(const ora_hg* h, uint64_t seed, int32_t rounds, int32_t kmin, int32_t* ks);

static int32_t ora_build_hierarchy(const ora_hg* h, const double* w, uint64_t seed, int32_t rounds, int32_t kmin,
                                   ora_graph* G, int32_t** PI) {
  ora_graph* g0 = &G[0];
  g0->k = h->k;
  g0->adj_ptr = (int32_t*)malloc((size_t)(h->k + 1) * sizeof(int32_t));
  memcpy(g0->adj_ptr, h->adj_ptr, (size_t)(h->k + 1) * sizeof(int32_t));
  int64_t na = h->adj_ptr[h->k];
  g0->adj = (int32_t*)malloc((size_t)(na > 0 ? na : 1) * sizeof(int32_t));
  memcpy(g0->adj, h->adj, (size_t)na * sizeof(int32_t));
  g0->acost = (double*)malloc((size_t)(na > 0 ? na : 1) * sizeof(double));
  for (int64_t t = 0; t < na; ++t) g0->acost[t] = 1.0;
  g0->w = (double*)malloc((size_t)(h->k > 0 ? h->k : 1) * sizeof(double));
  for (int32_t v = 0; v < h->k; ++v) g0->w[v] = w ? w[v] : 1.0;
  int32_t nl = 1;
  while (nl < 41 && G[nl - 1].k > kmin) {
    ora_graph* g = &G[nl - 1];
    int32_t* mate = (int32_t*)malloc((size_t)(g->k > 0 ? g->k : 1) * sizeof(int32_t));
    int32_t* pi = (int32_t*)malloc((size_t)(g->k > 0 ? g->k : 1) * sizeof(int32_t));
    int32_t kc = ora_match(g->k, g->adj_ptr, g->adj, g->acost, seed, nl - 1, rounds, mate, pi);
    free(mate);
    if ((double)kc > 0.95 * (double)g->k) { free(pi); break; }
    PI[nl - 1] = pi;
    ora_contract(g, pi, kc, &G[nl]);
    ++nl;
  }
  return nl;
}

ORA_EXPORT int32_t ora_hierarchy(const ora_hg* h, uint64_t seed, int32_t rounds, int32_t kmin, int32_t* ks) {
  ora_graph G[41];
  int32_t* PI[41];
  memset(G, 0, sizeof(G)); memset(PI, 0, sizeof(PI));
  int32_t nl = ora_build_hierarchy(h, NULL, seed, rounds, kmin, G, PI);
  for (int32_t j = 0; j < nl; ++j) { ks[j] = G[j].k; ora_graph_free(&G[j]); free(PI[j]); }
  return nl;
}

/* One level of the coarsening hierarchy of a graph (for checks): the graph of
 * level j (vertex count, adjacency with summed edge costs, summed vertex
 * weights; w = NULL for unit weights at level 0) and, for j >= 1, the grouping
 * pi of level j-1 into level j.  Outputs are malloc'd (release with ora_free);
 * pi_out receives NULL for j = 0.  Returns the number of levels, or -1 (and
 * nothing allocated) when j is not a level. */
ORA_EXPORT int32_t ora_hierarchy_level(const ora_hg* h, const double* w, uint64_t seed, int32_t rounds, int32_t kmin,
                                       int32_t j, int32_t* k_out, int64_t* nadj_out, int32_t** adj_ptr_out,
                                       int32_t** adj_out, double** acost_out, double** w_out, int32_t** pi_out) {
  ora_graph G[41];
  int32_t* PI[41];
  memset(G, 0, sizeof(G)); memset(PI, 0, sizeof(PI));
  int32_t nl = ora_build_hierarchy(h, w, seed, rounds, kmin, G, PI);
  int32_t ret = (j >= 0 && j < nl) ? nl : -1;
  if (ret > 0) {
    *k_out = G[j].k;
    *nadj_out = G[j].adj_ptr[G[j].k];
    *adj_ptr_out = G[j].adj_ptr; *adj_out = G[j].adj; *acost_out = G[j].acost; *w_out = G[j].w;
    memset(&G[j], 0, sizeof(G[j]));
    *pi_out = j > 0 ? PI[j - 1] : NULL;
    if (j > 0) PI[j - 1] = NULL;
  }
  for (int32_t i = 0; i < nl; ++i) { ora_graph_free(&G[i]); free(PI[i]); }
  return ret;
}

/* Prolongation of Algorithm 3 from level j (kc vertices) to level j-1 (kf
 * vertices, grouping pi): x_{j-1}(v) = f * x_j(pi(v)) + jitter(v), with
 * f = (kf/kc)^(1/d), which keeps the number of points per unit volume, and
 * jitter_m = 0.1 * (u - 1/2), u = (rand(seed^JITTER, v, 4*(j-1) + m) >> 40) * 2^-24
 * uniform in [0, 1), so that the members of a group start apart. */
ORA_EXPORT void ora_prolong(int32_t kf, int32_t kc, int32_t d, uint64_t seed, int32_t j, const int32_t* pi,
                            const double* xc /* kc*4 */, double* xf /* kf*4, out */) {
  double f = pow((double)kf / (double)kc, 1.0 / d);
  for (int32_t v = 0; v < kf; ++v)
    for (int m = 0; m < 4; ++m) {
      if (m >= d) { xf[4 * v + m] = 0.0; continue; }
      uint64_t r = ora_rand64(seed ^ ORA_TAG_JITTER, (uint64_t)v, (uint64_t)(4 * (j - 1) + m));
      double u = (double)(r >> 40) * 0x1p-24;
      xf[4 * v + m] = f * xc[4 * pi[v] + m] + 0.1 * (u - 0.5);
    }
}

static int ora_layout_connected(const ora_hg* h, int32_t d, int32_t occ, double sigma, double decay,
                                int32_t iters, uint64_t seed, int32_t rounds, int32_t kmin, const double* w,
                                double* x /* out, k*4 */) {
  ora_graph G[41];
  int32_t* PI[41];
  memset(G, 0, sizeof(G)); memset(PI, 0, sizeof(PI));
  int32_t nl = ora_build_hierarchy(h, w, seed, rounds, kmin, G, PI);
  int32_t kc = G[nl - 1].k;
  double* xc = (double*)calloc((size_t)(kc > 0 ? kc : 1) * 4, sizeof(double));
  float* xf = (float*)malloc((size_t)(kc > 0 ? kc : 1) * 4 * sizeof(float));
  ora_init_coords(kc, d, seed, xf);
  for (int64_t t = 0; t < 4 * (int64_t)kc; ++t) xc[t] = xf[t];
  free(xf);
  for (int32_t j = nl - 1; j >= 0; --j) {
    ora_hg hj;
    double* cj;
    ora_graph_hg(&G[j], &hj, &cj);
    ora_layout(&hj, d, occ, sigma, decay, iters, G[j].w, cj, xc);
    free(cj);
    ora_hg_free(&hj);
    if (j > 0) { /* prolong to level j-1 */
      int32_t kf = G[j - 1].k;
      double* xn = (double*)calloc((size_t)kf * 4, sizeof(double));
      ora_prolong(kf, G[j].k, d, seed, j, PI[j - 1], xc, xn);
      free(xc);
      xc = xn;
    }
  }
  memcpy(x, xc, (size_t)h->k * 4 * sizeof(double));
  free(xc);
  for (int32_t j = 0; j < nl; ++j) { ora_graph_free(&G[j]); free(PI[j]); }
  return nl;
}

/* Component grouping used by the layout and the ordering (Sec. 2.2: no
 * minimiser exists for a disconnected hypergraph, so every connected
 * component is treated separately).  Components are numbered in ascending
 * order of their smallest vertex (the label of Algorithm 1); cperm lists the
 * vertices component by component, ascending within a component; cbase[c]
 * is the first position of component c (ncomp+1 entries).  Returns ncomp. */
static int32_t ora_group_components(const ora_hg* h, int32_t* cperm, int32_t** cbase_out) {
  int32_t k = h->k;
  int32_t* lab = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  ora_components(k, h->l, h->net_ptr, h->pins, lab);
  int32_t* cid = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  int32_t nc = 0;
  for (int32_t v = 0; v < k; ++v) cid[v] = (lab[v] == v) ? nc++ : -1;
  int32_t* cbase = (int32_t*)calloc((size_t)nc + 1, sizeof(int32_t));
  for (int32_t v = 0; v < k; ++v) cbase[cid[lab[v]] + 1]++;
  for (int32_t c = 0; c < nc; ++c) cbase[c + 1] += cbase[c];
  int32_t* fill = (int32_t*)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int32_t));
  for (int32_t v = 0; v < k; ++v) {
    int32_t c = cid[lab[v]];
    cperm[cbase[c] + fill[c]++] = v;
  }
  free(lab); free(cid); free(fill);
  *cbase_out = cbase;
  return nc;
}

/* Induced subgraph of the vertices cperm[a..b) with local ids 0..b-a-1
 * (adjacency only, neighbours ascending since local ids follow global ids). */
static void ora_subgraph(const ora_hg* h, const int32_t* cperm, int32_t a, int32_t b, const int32_t* local,
                         ora_hg* out) {
  memset(out, 0, sizeof(*out));
  int32_t k = b - a;
  out->model = 0; out->k = k;
  out->adj_ptr = (int32_t*)calloc((size_t)k + 1, sizeof(int32_t));
  for (int32_t i = 0; i < k; ++i) {
    int32_t v = cperm[a + i];
    out->adj_ptr[i + 1] = out->adj_ptr[i] + (h->adj_ptr[v + 1] - h->adj_ptr[v]);
  }
  out->adj = (int32_t*)malloc((size_t)(out->adj_ptr[k] > 0 ? out->adj_ptr[k] : 1) * sizeof(int32_t));
  for (int32_t i = 0; i < k; ++i) {
    int32_t v = cperm[a + i];
    int32_t o = out->adj_ptr[i];
    for (int32_t t = h->adj_ptr[v]; t < h->adj_ptr[v + 1]; ++t) out->adj[o++] = local[h->adj[t]];
  }
}

/* Multilevel layout (Algorithm 3) of a graph model, each connected component
 * laid out on its own with local vertex ids (the paper applies Algorithm 3 to
 * each component), all with the same seed. */
ORA_EXPORT int ora_layout_multilevel(const ora_hg* h, int32_t d, int32_t occ, double sigma, double decay,
                                     int32_t iters, uint64_t seed, int32_t rounds, int32_t kmin, const double* w,
                                     double* x /* out, k*4 */) {
  int32_t k = h->k;
  int32_t* cperm = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  int32_t* cbase;
  int32_t nc = ora_group_components(h, cperm, &cbase);
  int32_t* local = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  for (int32_t c = 0; c < nc; ++c)
    for (int32_t i = cbase[c]; i < cbase[c + 1]; ++i) local[cperm[i]] = i - cbase[c];
  for (int32_t c = 0; c < nc; ++c) {
    int32_t a = cbase[c], b = cbase[c + 1], kc = b - a;
    ora_hg sub;
    ora_subgraph(h, cperm, a, b, local, &sub);
    double* wc = NULL;
    if (w) {
      wc = (double*)malloc((size_t)kc * sizeof(double));
      for (int32_t i = 0; i < kc; ++i) wc[i] = w[cperm[a + i]];
    }
    double* xc = (double*)calloc((size_t)kc * 4, sizeof(double));
    ora_layout_connected(&sub, d, occ, sigma, decay, iters, seed, rounds, kmin, wc, xc);
    for (int32_t i = 0; i < kc; ++i)
      for (int m = 0; m < 4; ++m) x[4 * (int64_t)cperm[a + i] + m] = xc[4 * (int64_t)i + m];
    free(xc); free(wc); free(sub.adj_ptr); free(sub.adj);
  }
  free(cperm); free(cbase); free(local);
  return nc;
}

/* ------------------------------------------------------------------------- */
/* 2-means by k-means++ (Algorithm 5, Sec. 3, with m = 2).                    */
/*                                                                            */
/* Points are the fp32 coordinates of the node's vertices, in the node's      */
/* current order.  Readings:                                                  */
/*  * z1 is point floor(|S| * r0 / 2^64) with r0 = rand(seed^KM, key, 0),     */
/*    key = the node's heap number (root 1, children 2h and 2h+1).            */
/*  * z2 is drawn with probability d_i / sum d (Algorithm 5): d_i is the fp32 */
/*    squared distance to z1, weighted as D_i = floor(d_i * 2^Q) with         */
/*    Q = 34 - 2e and 2^e > max |coordinate| of the node, so the prefix sums  */
/*    are exact integers; z2 is the first point whose inclusive prefix        */
/*    exceeds floor(sum D * r1 / 2^64), r1 = rand(seed^KM, key, 1).  If the   */
/*    sum is 0 (all points on z1) the node is not split.                      */
/*  * A label is 1 iff ||x - z1||^2 <= ||x - z2||^2 (Algorithm 7), both       */
/*    squared distances in fp32, summed over m = 0..d-1, no FMA.              */
/*  * "A fixed number of iterations": assign, stop if no label changed,       */
/*    otherwise move each non-empty cluster's centre to its mean; at most     */
/*    km_iters rounds; final labels from the final centres.                   */
/*  * A centre is the mean of its points computed exactly on the grid 2^-P,   */
/*    P = 30 - e: q(x) = round-half-even(x * 2^P) summed in 64-bit integers,  */
/*    z = fp32((double(sum) / count) * 2^-P).                                 */
/* ------------------------------------------------------------------------- */
static float ora_sqdist32(const float* a, const float* b, int d) {
  float s = 0.0f;
  for (int m = 0; m < d; ++m) {
    float q = a[m] - b[m];
    float qq = q * q;
    s = s + qq;
  }
  return s;
}

static int ora_exponent(const float* x4, const int32_t* verts, int32_t nv, int d) {
  float mx = 0.0f;
  for (int32_t i = 0; i < nv; ++i)
    for (int m = 0; m < d; ++m) {
      float a = fabsf(x4[4 * (int64_t)verts[i] + m]);
      if (a > mx) mx = a;
    }
  if (mx == 0.0f) return 0;
  int e;
  frexpf(mx, &e); /* mx = f * 2^e, 0.5 <= f < 1, so mx < 2^e */
  return e;
}

/* Returns 1 if the node was split into two non-empty sides, 0 otherwise.
 * labels[i] in {1, 2} refers to verts[i]; z1/z2 receive the final centres. */
ORA_EXPORT int ora_bisect(int32_t d, const float* x4 /* coordinates, 4 per vertex */,
                          const int32_t* verts, int32_t nv, uint64_t seed, uint64_t key,
                          int32_t km_iters, uint8_t* labels, float* z1, float* z2) {
  for (int m = 0; m < 4; ++m) { z1[m] = 0.0f; z2[m] = 0.0f; }
  for (int32_t i = 0; i < nv; ++i) labels[i] = 1;
  if (nv < 2) return 0;
  int e = ora_exponent(x4, verts, nv, d);
  int P = 30 - e, Q = 34 - 2 * e;
  uint64_t r0 = ora_rand64(seed ^ ORA_TAG_KMEANS, key, 0);
  uint64_t r1 = ora_rand64(seed ^ ORA_TAG_KMEANS, key, 1);
  int32_t i0 = (int32_t)ora_scale_draw((uint64_t)nv, r0);
  for (int m = 0; m < d; ++m) z1[m] = x4[4 * (int64_t)verts[i0] + m];
  /* D^2 weighting */
  uint64_t total = 0;
  for (int32_t i = 0; i < nv; ++i) {
    float di = ora_sqdist32(&x4[4 * (int64_t)verts[i]], z1, d);
    total += (uint64_t)floor(ldexp((double)di, Q));
  }
  if (total == 0) return 0;
  uint64_t thr = ora_scale_draw(total, r1), pre = 0;
  int32_t i1 = nv - 1;
  for (int32_t i = 0; i < nv; ++i) {
    float di = ora_sqdist32(&x4[4 * (int64_t)verts[i]], z1, d);
    pre += (uint64_t)floor(ldexp((double)di, Q));
    if (pre > thr) { i1 = i; break; }
  }
  for (int m = 0; m < d; ++m) z2[m] = x4[4 * (int64_t)verts[i1] + m];
  /* Lloyd rounds */
  uint8_t* prev = (uint8_t*)malloc((size_t)nv);
  int have_prev = 0;
  for (int32_t it = 0; it < km_iters; ++it) {
    int changed = 0;
    int64_t S1[4] = {0, 0, 0, 0}, S2[4] = {0, 0, 0, 0};
    int64_t n1 = 0, n2 = 0;
    for (int32_t i = 0; i < nv; ++i) {
      const float* p = &x4[4 * (int64_t)verts[i]];
      uint8_t lab = (ora_sqdist32(p, z1, d) <= ora_sqdist32(p, z2, d)) ? 1 : 2;
      if (!have_prev || lab != prev[i]) changed = 1;
      prev[i] = lab;
      for (int m = 0; m < d; ++m) {
        int64_t q = llrint(ldexp((double)p[m], P));
        if (lab == 1) S1[m] += q; else S2[m] += q;
      }
      if (lab == 1) n1++; else n2++;
    }
    if (have_prev && !changed) break;
    have_prev = 1;
    for (int m = 0; m < d; ++m) {
      if (n1 > 0) z1[m] = (float)(((double)S1[m] / (double)n1) * ldexp(1.0, -P));
      if (n2 > 0) z2[m] = (float)(((double)S2[m] / (double)n2) * ldexp(1.0, -P));
    }
  }
  free(prev);
  int32_t n1 = 0, n2 = 0;
  for (int32_t i = 0; i < nv; ++i) {
    const float* p = &x4[4 * (int64_t)verts[i]];
    labels[i] = (ora_sqdist32(p, z1, d) <= ora_sqdist32(p, z2, d)) ? 1 : 2;
    if (labels[i] == 1) n1++; else n2++;
  }
  return (n1 > 0 && n2 > 0) ? 1 : 0;
}

/* ------------------------------------------------------------------------- */
/* m-way k-means++ (Algorithm 5 with m centres; the partition C_1..C_m of     */
/* Sec. 3), in the readings of the 2-means above:                             */
/*  * z_1 = point floor(nv * r_0 / 2^64); for n = 2..m, D_i =                 */
/*    floor(min_{j<n} ||x_i - z_j||^2 * 2^(34 - 2e)) (distances fp32, no      */
/*    FMA) and z_n = the first point whose inclusive prefix of D exceeds      */
/*    floor(sum D * r_(n-1) / 2^64), r_j = rand(seed ^ KMEANS, key, j).  If   */
/*    the sum is 0 (every point on a chosen centre) the remaining centres     */
/*    are copies of z_1 and never win a point.                                */
/*  * Lloyd: label argmin_j ||x - z_j||^2, ties to the smaller j; stop when   */
/*    no label changes, at most km_iters rounds; exact fixed-point means of   */
/*    non-empty clusters; final labels from the final centres.                */
/* For m = 2 this is ora_bisect with labels 0 / 1 instead of 1 / 2.          */
/* labels[i] in [0, m) refers to verts[i]; z: m x 4 floats.  Returns the      */
/* number of non-empty clusters.                                              */
/* ------------------------------------------------------------------------- */
static int32_t ora_nearest(const float* p, const float* z, int32_t m, int d) {
  int32_t best = 0;
  float bd = ora_sqdist32(p, z, d);
  for (int32_t j = 1; j < m; ++j) {
    float dj = ora_sqdist32(p, z + 4 * (int64_t)j, d);
    if (dj < bd) { bd = dj; best = j; }
  }
  return best;
}

ORA_EXPORT int32_t ora_kmeans(int32_t d, const float* x4, const int32_t* verts, int32_t nv, int32_t m,
                              uint64_t seed, uint64_t key, int32_t km_iters, int32_t* labels, float* z) {
  for (int64_t j = 0; j < 4 * (int64_t)m; ++j) z[j] = 0.0f;
  for (int32_t i = 0; i < nv; ++i) labels[i] = 0;
  if (nv < 1 || m < 1) return 0;
  int e = ora_exponent(x4, verts, nv, d);
  int P = 30 - e, Q = 34 - 2 * e;
  int32_t i0 = (int32_t)ora_scale_draw((uint64_t)nv, ora_rand64(seed ^ ORA_TAG_KMEANS, key, 0));
  for (int mm = 0; mm < d; ++mm) z[mm] = x4[4 * (int64_t)verts[i0] + mm];
  float* dmin = (float*)malloc((size_t)nv * sizeof(float));
  for (int32_t i = 0; i < nv; ++i) dmin[i] = ora_sqdist32(&x4[4 * (int64_t)verts[i]], z, d);
  int32_t chosen = 1;
  for (int32_t n = 1; n < m; ++n) { /* centre index n (the (n+1)-th) */
    uint64_t total = 0;
    for (int32_t i = 0; i < nv; ++i) total += (uint64_t)floor(ldexp((double)dmin[i], Q));
    if (total == 0) break;
    uint64_t thr = ora_scale_draw(total, ora_rand64(seed ^ ORA_TAG_KMEANS, key, (uint64_t)n)), pre = 0;
    int32_t pick = nv - 1;
    for (int32_t i = 0; i < nv; ++i) {
      pre += (uint64_t)floor(ldexp((double)dmin[i], Q));
      if (pre > thr) { pick = i; break; }
    }
    for (int mm = 0; mm < d; ++mm) z[4 * (int64_t)n + mm] = x4[4 * (int64_t)verts[pick] + mm];
    chosen = n + 1;
    for (int32_t i = 0; i < nv; ++i) {
      float dn = ora_sqdist32(&x4[4 * (int64_t)verts[i]], z + 4 * (int64_t)n, d);
      if (dn < dmin[i]) dmin[i] = dn;
    }
  }
  for (int32_t n = chosen; n < m; ++n)
    for (int mm = 0; mm < 4; ++mm) z[4 * (int64_t)n + mm] = z[mm];
  free(dmin);
  int64_t* S = (int64_t*)malloc((size_t)m * 4 * sizeof(int64_t));
  int64_t* cnt = (int64_t*)malloc((size_t)m * sizeof(int64_t));
  int32_t* prev = (int32_t*)malloc((size_t)nv * sizeof(int32_t));
  int have_prev = 0;
  for (int32_t it = 0; it < km_iters; ++it) {
    int changed = 0;
    memset(S, 0, (size_t)m * 4 * sizeof(int64_t));
    memset(cnt, 0, (size_t)m * sizeof(int64_t));
    for (int32_t i = 0; i < nv; ++i) {
      const float* p = &x4[4 * (int64_t)verts[i]];
      int32_t lab = ora_nearest(p, z, m, d);
      if (!have_prev || lab != prev[i]) changed = 1;
      prev[i] = lab;
      for (int mm = 0; mm < d; ++mm) S[4 * (int64_t)lab + mm] += llrint(ldexp((double)p[mm], P));
      cnt[lab]++;
    }
    if (have_prev && !changed) break;
    have_prev = 1;
    for (int32_t j = 0; j < m; ++j)
      if (cnt[j] > 0)
        for (int mm = 0; mm < d; ++mm)
          z[4 * (int64_t)j + mm] = (float)(((double)S[4 * (int64_t)j + mm] / (double)cnt[j]) * ldexp(1.0, -P));
  }
  memset(cnt, 0, (size_t)m * sizeof(int64_t));
  for (int32_t i = 0; i < nv; ++i) {
    labels[i] = ora_nearest(&x4[4 * (int64_t)verts[i]], z, m, d);
    cnt[labels[i]]++;
  }
  int32_t nonempty = 0;
  for (int32_t j = 0; j < m; ++j) nonempty += cnt[j] > 0;
  free(S); free(cnt); free(prev);
  return nonempty;
}

/* ------------------------------------------------------------------------- */
/* Vertex separator (Algorithm 7, Sec. 4.2) with mu = identity (no            */
/* strengthened diagonal).                                                    */
/*                                                                            */
/* Plane: r = z2 - z1, delta = sum_m (0.5 (z1_m + z2_m)) r_m, and             */
/* s(v) = |sum_m x_m(v) r_m - delta|, all fp32, left to right, no FMA.        */
/* The paper's edge loop is sequential and its result depends on the edge     */
/* order.  Reading: edges are visited in ascending order of the key           */
/* (s, vertex id) of their smaller-key end; an edge whose ends still carry    */
/* labels {1, 2} moves its smaller-key end into the separator (label 3).      */
/* This equals the order-free rule "v goes to 3 iff some neighbour w in the   */
/* node has the other label and (s(v), v) < (s(w), w)".                       */
/* ------------------------------------------------------------------------- */
static float ora_plane(const float* x, const float* r, float delta, int d) {
  float acc = 0.0f;
  for (int m = 0; m < d; ++m) {
    float t = x[m] * r[m];
    acc = acc + t;
  }
  return fabsf(acc - delta);
}

typedef struct { float s; int32_t v, w; } ora_cut_edge;

static int cmp_cut_edge(const void* a, const void* b) {
  const ora_cut_edge* p = (const ora_cut_edge*)a;
  const ora_cut_edge* q = (const ora_cut_edge*)b;
  if (p->s < q->s) return -1;
  if (p->s > q->s) return 1;
  if (p->v != q->v) return (p->v > q->v) - (p->v < q->v);
  return (p->w > q->w) - (p->w < q->w);
}

/* lab[v] (indexed by vertex id) holds the 2-means labels of the node's
 * vertices on entry and {1, 2, 3} on exit; innode[v] marks the node's
 * vertices.  mu: NULL (no strengthened diagonal: mu is the identity) or the
 * partner of every vertex under the matching M.  Returns the separator size.
 *
 * With a matching, the loop of Algorithm 7 moves both v and mu(v) into V3,
 * and a partner moved early turns later edges at it into uncut ones, so the
 * outcome depends on the edge order, which the paper does not fix.  Reading
 * (mu_rule 0, the default): the loop itself, over the cut edges in the
 * canonical order above; an edge whose ends no longer carry labels 1 and 2
 * (one of them, or its partner, moved already) is skipped.  mu_rule 1: the
 * order-free form, every edge cut by the 2-means labels (before any move)
 * selects its end with the smaller (|x.r - delta|, id), and the selected
 * vertices and their partners form V3 (a superset of the loop's separator).
 * With mu = identity both are the loop below. */
static int32_t ora_separate(const ora_hg* h, int d, const float* x4, const int32_t* verts, int32_t nv,
                            const uint8_t* innode, uint8_t* lab, const float* z1, const float* z2,
                            const int32_t* mu, int32_t mu_rule) {
  float r[4], delta = 0.0f;
  for (int m = 0; m < d; ++m) r[m] = z2[m] - z1[m];
  for (int m = 0; m < d; ++m) {
    float mid = 0.5f * (z1[m] + z2[m]);
    float t = mid * r[m];
    delta = delta + t;
  }
  int64_t ne = 0;
  for (int32_t i = 0; i < nv; ++i) {
    int32_t v = verts[i];
    for (int32_t t = h->adj_ptr[v]; t < h->adj_ptr[v + 1]; ++t) {
      int32_t w = h->adj[t];
      if (w > v && innode[w] && lab[v] != lab[w]) ne++;
    }
  }
  ora_cut_edge* E = (ora_cut_edge*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(ora_cut_edge));
  ne = 0;
  for (int32_t i = 0; i < nv; ++i) {
    int32_t v = verts[i];
    for (int32_t t = h->adj_ptr[v]; t < h->adj_ptr[v + 1]; ++t) {
      int32_t w = h->adj[t];
      if (!(w > v && innode[w] && lab[v] != lab[w])) continue;
      float sv = ora_plane(&x4[4 * (int64_t)v], r, delta, d);
      float sw = ora_plane(&x4[4 * (int64_t)w], r, delta, d);
      /* orient so that (s, id) of the first end is the smaller one */
      if (sw < sv || (sw == sv && w < v)) E[ne++] = (ora_cut_edge){sw, w, v};
      else E[ne++] = (ora_cut_edge){sv, v, w};
    }
  }
  qsort(E, (size_t)ne, sizeof(ora_cut_edge), cmp_cut_edge);
  int32_t nsep = 0;
  if (mu) {
    for (int64_t t = 0; t < ne; ++t) {
      if (!innode[mu[E[t].v]]) abort(); /* partners always share a node */
    }
  }
  if (mu && mu_rule == 1) {
    /* all selections are taken against the 2-means labels, then applied */
    for (int64_t t = 0; t < ne; ++t) {
      if (lab[E[t].v] != 3) { lab[E[t].v] = 3; nsep++; }
      if (lab[mu[E[t].v]] != 3) { lab[mu[E[t].v]] = 3; nsep++; }
    }
    free(E);
    return nsep;
  }
  for (int64_t t = 0; t < ne; ++t) {
    uint8_t pv = lab[E[t].v], pw = lab[E[t].w];
    if (!((pv == 1 && pw == 2) || (pv == 2 && pw == 1))) continue;
    lab[E[t].v] = 3; /* |x(v).r - delta| <= |x(w).r - delta|: v joins the separator */
    nsep++;
    if (mu && lab[mu[E[t].v]] != 3) { lab[mu[E[t].v]] = 3; nsep++; } /* and its partner */
  }
  free(E);
  return nsep;
}

/* ------------------------------------------------------------------------- */
/* Recursive BBD / SBD ordering (Algorithm 7 applied recursively, Sec. 4.2;   */
/* SBD places the separator between the two parts, Sec. 5).                  */
/*                                                                            */
/* Nodes are processed breadth first.  A node is a leaf if |V| <= min_part,   */
/* its depth equals max_depth, or 2-means leaves a side empty.  Otherwise its */
/* vertices are stably reordered to [V1, V2, V3] (BBD) or [V1, V3, V2] (SBD)  */
/* and V1, V2 become children (when non-empty) with heap numbers 2h, 2h+1.    */
/* The separator keeps its inherited order (it is not recursed into), unless  */
/* sep_rec is set: then V3 is a child as well (the additional freedom of      */
/* Sec. 4.2: V3 bisected recursively over the edges inside it, the Schur      */
/* complement in BBD form), the children of h are 3h-1, 3h, 3h+1 (V1, V2, V3) */
/* and nodes at depth min(max_depth, 39) are leaves (keys stay in 64 bits).  */
/* perm[new] = old.  Tree records: heap, offset, n1, n2, nsep, depth, comp  */
/* (a leaf has n1 = |V|, n2 = nsep = 0).                                      */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t count;
  uint64_t* heap;
  int32_t *offset, *n1, *n2, *nsep, *depth, *comp;
} ora_tree;

ORA_EXPORT void ora_tree_free(ora_tree* t) {
  free(t->heap); free(t->offset); free(t->n1); free(t->n2); free(t->nsep); free(t->depth); free(t->comp);
  memset(t, 0, sizeof(*t));
}

typedef struct { uint64_t heap; int32_t offset, size, depth, comp; } ora_node;

typedef struct { int32_t comp; uint64_t heap; int32_t rec; } ora_rec_key;
static int cmp_rec_key(const void* a, const void* b) {
  const ora_rec_key* p = (const ora_rec_key*)a;
  const ora_rec_key* q = (const ora_rec_key*)b;
  if (p->comp != q->comp) return (p->comp > q->comp) - (p->comp < q->comp);
  return (p->heap > q->heap) - (p->heap < q->heap);
}

/* Cut-row/column ordering (Sec. 4.2, the other use of the freedom in V3):    */
/* every vertex w of the separator V3 of a split node gets a two-bit number:  */
/* the first bit (value 1) if w has a neighbour in the first part of the     */
/* split of V1 or of V2 (V11 or V21), the second bit (value 2) if it has one  */
/* in their second parts (V12 or V22).  V3 is then stably sorted by the       */
/* number: ascending for BBD (00, 01, 10, 11); for SBD, whose separator sits  */
/* between the parts, as 01, 00, 11, 10 (cut rows of the first parts first,  */
/* of the second parts last).  Expanded to b two-bit pairs: pair l describes  */
/* the links into the first and second parts of the splits of the node's     */
/* descendants l levels down (l = 1: its children), and V3 is sorted by the   */
/* pairs in turn (pair 1 first), which brings the cut rows and columns into   */
/* recursive form down to the b-th level.  Part membership is by position     */
/* range, so the result does not depend on the order in which the nodes are   */
/* treated.  With a strengthened diagonal (mu) a row and its matched column   */
/* hold one position of the row and column orders, so a vertex is sorted by   */
/* the number of its pair: its own bits or its partner's.                     */
typedef struct { int32_t comp; uint64_t heap; int32_t rec; } ora_key;
static int cmp_key(const void* a, const void* b) {
  const ora_key* p = (const ora_key*)a;
  const ora_key* q = (const ora_key*)b;
  if (p->comp != q->comp) return (p->comp > q->comp) - (p->comp < q->comp);
  return (p->heap > q->heap) - (p->heap < q->heap);
}

static int32_t ora_find_rec(const ora_key* ks, int32_t n, int32_t comp, uint64_t heap) {
  int32_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    int32_t mid = (lo + hi) / 2;
    if (ks[mid].comp == comp && ks[mid].heap == heap) return ks[mid].rec;
    if (ks[mid].comp < comp || (ks[mid].comp == comp && ks[mid].heap < heap)) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

typedef struct { uint64_t key; int32_t i; } ora_cut_key;
static int cmp_cut_key(const void* a, const void* b) {
  const ora_cut_key* p = (const ora_cut_key*)a;
  const ora_cut_key* q = (const ora_cut_key*)b;
  if (p->key != q->key) return (p->key > q->key) - (p->key < q->key);
  return (p->i > q->i) - (p->i < q->i);
}

static void ora_cut_order(const ora_hg* h, int32_t sbd, int32_t b, const int32_t* mu, int32_t* perm,
                          const ora_tree* tree) {
  int32_t k = h->k, nrec = tree->count;
  int32_t* pos = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  for (int32_t i = 0; i < k; ++i) pos[perm[i]] = i;
  ora_key* ks = (ora_key*)malloc((size_t)(nrec > 0 ? nrec : 1) * sizeof(ora_key));
  for (int32_t r = 0; r < nrec; ++r) ks[r] = (ora_key){tree->comp[r], tree->heap[r], r};
  qsort(ks, (size_t)nrec, sizeof(ora_key), cmp_key);
  static const int rank_bbd[4] = {0, 1, 2, 3}, rank_sbd[4] = {1, 0, 3, 2};
  const int* rank = sbd ? rank_sbd : rank_bbd;
  int32_t* tmp = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  uint32_t* vcode = (uint32_t*)calloc((size_t)(k > 0 ? k : 1), sizeof(uint32_t));
  int32_t maxr = 2 << b; /* at most 2^b split descendants l <= b levels down, two parts each */
  int32_t* lo = (int32_t*)malloc((size_t)maxr * sizeof(int32_t));
  int32_t* hi = (int32_t*)malloc((size_t)maxr * sizeof(int32_t));
  uint8_t* bit = (uint8_t*)malloc((size_t)maxr);
  for (int32_t r = 0; r < nrec; ++r) {
    int32_t o = tree->offset[r], n1 = tree->n1[r], n2 = tree->n2[r], ns = tree->nsep[r];
    if (ns == 0) continue;
    int32_t a = sbd ? o + n1 : o + n1 + n2;
    for (int32_t i = 0; i < ns; ++i) vcode[perm[a + i]] = 0;
    for (int32_t l = 1; l <= b && tree->depth[r] + l <= 62; ++l) {
      /* first / second part ranges of the splits of the descendants l levels down */
      int32_t nr = 0;
      for (uint64_t j = 0; j < (1ull << l); ++j) {
        int32_t cr = ora_find_rec(ks, nrec, tree->comp[r], (tree->heap[r] << l) + j);
        if (cr < 0) continue;
        int32_t co = tree->offset[cr], c1 = tree->n1[cr], c2 = tree->n2[cr], cs = tree->nsep[cr];
        if (c2 == 0 && cs == 0) continue; /* a leaf has no parts */
        lo[nr] = co; hi[nr] = co + c1; bit[nr++] = 1;
        lo[nr] = sbd ? co + c1 + cs : co + c1; hi[nr] = lo[nr] + c2; bit[nr++] = 2;
      }
      for (int32_t i = 0; i < ns; ++i) {
        int32_t w = perm[a + i];
        uint32_t cw = 0;
        for (int32_t t = h->adj_ptr[w]; t < h->adj_ptr[w + 1]; ++t) {
          int32_t p = pos[h->adj[t]];
          for (int32_t q = 0; q < nr; ++q)
            if (p >= lo[q] && p < hi[q]) cw |= bit[q];
        }
        vcode[w] |= cw << (2 * (b - l));
      }
    }
    ora_cut_key* key = (ora_cut_key*)malloc((size_t)ns * sizeof(ora_cut_key));
    for (int32_t i = 0; i < ns; ++i) {
      int32_t w = perm[a + i];
      uint32_t c = mu ? (vcode[w] | vcode[mu[w]]) : vcode[w];
      uint64_t kk = 0;
      for (int32_t l = 1; l <= b; ++l) kk = 4 * kk + (uint64_t)rank[(c >> (2 * (b - l))) & 3];
      key[i] = (ora_cut_key){kk, i};
    }
    qsort(key, (size_t)ns, sizeof(ora_cut_key), cmp_cut_key);
    for (int32_t i = 0; i < ns; ++i) tmp[i] = perm[a + key[i].i];
    memcpy(perm + a, tmp, (size_t)ns * sizeof(int32_t));
    free(key);
  }
  free(pos); free(ks); free(tmp); free(vcode); free(lo); free(hi); free(bit);
}

/* Ordering of a graph model from fp32 coordinates.  A disconnected graph is
 * block diagonal: its components (grouped as in the layout) are ordered one
 * after the other, each by its own recursion (root heap number 1).  Tree
 * records carry the component index; offsets are absolute positions in perm;
 * records are sorted by (component, heap number). */
ORA_EXPORT int ora_order(const ora_hg* h, int32_t d, const float* x4, uint64_t seed, int32_t km_iters,
                         int32_t min_part, int32_t max_depth, int32_t sbd, int32_t sep_rec, int32_t cut_order,
                         const int32_t* mu, int32_t mu_rule, int32_t* perm, ora_tree* tree) {
  int32_t k = h->k;
  if (sep_rec && max_depth > 39) max_depth = 39;
  int32_t* cbase;
  int32_t nc = ora_group_components(h, perm, &cbase);
  memset(tree, 0, sizeof(*tree));
  int32_t cap = 2 * k + 8;
  ora_node* queue = (ora_node*)malloc((size_t)cap * sizeof(ora_node));
  tree->heap = (uint64_t*)malloc((size_t)cap * sizeof(uint64_t));
  tree->offset = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  tree->n1 = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  tree->n2 = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  tree->nsep = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  tree->depth = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  tree->comp = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  uint8_t* lab = (uint8_t*)calloc((size_t)(k > 0 ? k : 1), 1);
  uint8_t* innode = (uint8_t*)calloc((size_t)(k > 0 ? k : 1), 1);
  uint8_t* nlab = (uint8_t*)malloc((size_t)(k > 0 ? k : 1));
  int32_t* tmp = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  int32_t qh = 0, qt = 0;
  for (int32_t c = 0; c < nc; ++c) queue[qt++] = (ora_node){1ull, cbase[c], cbase[c + 1] - cbase[c], 0, c};
  while (qh < qt) {
    ora_node nd = queue[qh++];
    int32_t* verts = perm + nd.offset;
    int32_t rec = tree->count++;
    tree->heap[rec] = nd.heap; tree->offset[rec] = nd.offset; tree->depth[rec] = nd.depth;
    tree->comp[rec] = nd.comp;
    tree->n1[rec] = nd.size; tree->n2[rec] = 0; tree->nsep[rec] = 0;
    if (nd.size <= min_part || nd.depth >= max_depth) continue;
    float z1[4], z2[4];
    if (!ora_bisect(d, x4, verts, nd.size, seed, nd.heap, km_iters, nlab, z1, z2)) continue;
    for (int32_t i = 0; i < nd.size; ++i) { lab[verts[i]] = nlab[i]; innode[verts[i]] = 1; }
    ora_separate(h, d, x4, verts, nd.size, innode, lab, z1, z2, mu, mu_rule);
    int32_t c1 = 0, c2 = 0, c3 = 0;
    for (int32_t i = 0; i < nd.size; ++i) {
      uint8_t l = lab[verts[i]];
      c1 += (l == 1); c2 += (l == 2); c3 += (l == 3);
    }
    /* stable partition */
    int32_t p1 = 0, p2 = sbd ? c1 + c3 : c1, p3 = sbd ? c1 : c1 + c2;
    for (int32_t i = 0; i < nd.size; ++i) {
      int32_t v = verts[i];
      uint8_t l = lab[v];
      if (l == 1) tmp[p1++] = v; else if (l == 2) tmp[p2++] = v; else tmp[p3++] = v;
    }
    for (int32_t i = 0; i < nd.size; ++i) { verts[i] = tmp[i]; innode[tmp[i]] = 0; lab[tmp[i]] = 0; }
    tree->n1[rec] = c1; tree->n2[rec] = c2; tree->nsep[rec] = c3;
    if (!sep_rec) {
      if (c1 > 0) queue[qt++] = (ora_node){2 * nd.heap, nd.offset, c1, nd.depth + 1, nd.comp};
      if (c2 > 0) queue[qt++] = (ora_node){2 * nd.heap + 1, nd.offset + (sbd ? c1 + c3 : c1), c2, nd.depth + 1, nd.comp};
    } else {
      if (c1 > 0) queue[qt++] = (ora_node){3 * nd.heap - 1, nd.offset, c1, nd.depth + 1, nd.comp};
      if (c2 > 0) queue[qt++] = (ora_node){3 * nd.heap, nd.offset + (sbd ? c1 + c3 : c1), c2, nd.depth + 1, nd.comp};
      if (c3 > 0) queue[qt++] = (ora_node){3 * nd.heap + 1, nd.offset + (sbd ? c1 : c1 + c2), c3, nd.depth + 1, nd.comp};
    }
  }
  if (cut_order > 0 && !sep_rec) ora_cut_order(h, sbd, cut_order, mu, perm, tree);
  /* sort records by (component, heap number) */
  int32_t nrec = tree->count;
  ora_rec_key* rk = (ora_rec_key*)malloc((size_t)(nrec > 0 ? nrec : 1) * sizeof(ora_rec_key));
  for (int32_t r = 0; r < nrec; ++r) rk[r] = (ora_rec_key){tree->comp[r], tree->heap[r], r};
  qsort(rk, (size_t)nrec, sizeof(ora_rec_key), cmp_rec_key);
  int32_t* fields[6] = {tree->offset, tree->n1, tree->n2, tree->nsep, tree->depth, tree->comp};
  int32_t* t32 = (int32_t*)malloc((size_t)(nrec > 0 ? nrec : 1) * sizeof(int32_t));
  uint64_t* t64 = (uint64_t*)malloc((size_t)(nrec > 0 ? nrec : 1) * sizeof(uint64_t));
  for (int f = 0; f < 6; ++f) {
    for (int32_t r = 0; r < nrec; ++r) t32[r] = fields[f][rk[r].rec];
    memcpy(fields[f], t32, (size_t)nrec * sizeof(int32_t));
  }
  for (int32_t r = 0; r < nrec; ++r) t64[r] = tree->heap[rk[r].rec];
  memcpy(tree->heap, t64, (size_t)nrec * sizeof(uint64_t));
  free(rk); free(t32); free(t64);
  free(queue); free(lab); free(innode); free(nlab); free(tmp); free(cbase);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Cut metrics (Sec. 4.1 footnote on the cut-net and (lambda - 1) metrics,    */
/* Sec. 5): lambda_e = number of distinct parts among the pins of net e;      */
/* cut-net = #{e : lambda_e > 1}; lambda-1 = sum_e (lambda_e - 1).            */
/* ------------------------------------------------------------------------- */
ORA_EXPORT void ora_cut_size(int32_t l, const int32_t* net_ptr, const int32_t* pins, const int32_t* part,
                             int64_t* cutnet, int64_t* lambda1) {
  int64_t cn = 0, l1 = 0;
  for (int32_t e = 0; e < l; ++e) {
    int64_t lam = 0;
    for (int32_t t = net_ptr[e]; t < net_ptr[e + 1]; ++t) {
      int seen = 0;
      for (int32_t u = net_ptr[e]; u < t; ++u)
        if (part[pins[u]] == part[pins[t]]) { seen = 1; break; }
      if (!seen) lam++;
    }
    if (lam > 1) { cn++; l1 += lam - 1; }
  }
  *cutnet = cn; *lambda1 = l1;
}

/* ------------------------------------------------------------------------- */
/* Fill-in of the ordered matrix (Table 2 caption): (nz(L) + nz(U) - n)/nz(A) */
/* for A = LU without pivoting.  For a structurally symmetric pattern, L and  */
/* U^T share the pattern of the Cholesky factor of the symmetrically permuted */
/* matrix, counted here by the elimination-tree row-subtree walk (for each    */
/* row i, climb from every k < i with a_ik != 0 until reaching a node already */
/* visited for row i; every visited node is a nonzero of row i of L).         */
/* Returns nz(L) including the diagonal.  perm[new] = old; the pattern is     */
/* symmetrised (A + A^T) and given the full diagonal.                         */
/* ------------------------------------------------------------------------- */
ORA_EXPORT int64_t ora_cholesky_nnz(int32_t n, const int32_t* rowptr, const int32_t* colidx,
                                    const int32_t* perm) {
  int32_t* inv = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  for (int32_t i = 0; i < n; ++i) inv[perm[i]] = i;
  /* lower-triangular pattern of P(A + A^T)P^T: keys (row, col) with col < row */
  int64_t nnz = rowptr[n];
  int64_t* key = (int64_t*)malloc((size_t)(2 * nnz > 0 ? 2 * nnz : 1) * sizeof(int64_t));
  int64_t nk = 0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
      int64_t a = inv[i], b = inv[colidx[t]];
      if (a == b) continue;
      int64_t hi = a > b ? a : b, lo = a > b ? b : a;
      key[nk++] = hi * n + lo;
    }
  nk = ora_sort_unique(key, nk);
  int32_t* parent = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t* flag = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int64_t nzl = n;
  int64_t t = 0;
  for (int32_t i = 0; i < n; ++i) {
    parent[i] = -1; flag[i] = i;
    for (; t < nk && key[t] / n == i; ++t) {
      int32_t j = (int32_t)(key[t] % n);
      while (flag[j] != i) {
        if (parent[j] == -1) parent[j] = i;
        nzl++;
        flag[j] = i;
        j = parent[j];
      }
    }
  }
  free(inv); free(key); free(parent); free(flag);
  return nzl;
}
