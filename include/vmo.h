/*
 * vmo.h — C-ABI of the GB300 library for visual matrix ordering (VMO),
 * the geometric method of Fagginger Auer and Bisseling, "A Geometric
 * Approach to Matrix Ordering".
 *
 * Pipeline: sparse pattern -> hypergraph model (Table 1) -> geometry by
 * multilevel force-directed layout (Algorithms 3 and 4, eq.
 * graphenergygradientsimple) -> recursive 2-means bisection (Algorithm 5)
 * turned into vertex separators (Algorithm 7) -> recursive BBD / SBD row and
 * column permutations (Sec. 4.2, Sec. 5).
 *
 * Conventions shared by every entry point:
 *  - All array arguments are DEVICE pointers unless the comment says "host".
 *    The caller owns every input and output buffer; a handle (vmo_hg) owns
 *    only the device arrays of its hypergraph model.
 *  - Coordinates are float[4] per vertex (16-byte aligned, components >= d
 *    are zero and ignored); the layout dimension d is 2, 3 or 4.
 *  - Permutations are perm[new] = old, 0-based.
 *  - Labels: 1 and 2 are the two sides of a split (Algorithm 7), 3 the
 *    separator.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls that return sizes or counts to
 *    the host synchronise that stream before returning.
 *  - Every call returns a vmo_status; nothing throws, exits or traps.  Inputs
 *    are validated before any launch (VMO_ERR_INVALID / VMO_ERR_UNSUPPORTED).
 *    CUDA failures return VMO_ERR_CUDA; vmo_last_error() gives the message of
 *    the calling thread's last failure.  There is no CPU fallback: without a
 *    usable GPU every compute call returns VMO_ERR_CUDA.
 *  - Random draws come from a counter-based SplitMix64 generator keyed by
 *    params.seed, so results are deterministic for a given input and seed.
 */
#ifndef VMO_H
#define VMO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VMO_OK = 0,
  VMO_ERR_INVALID = 1,     /* malformed argument (null, negative size, bad CSR) */
  VMO_ERR_OOM = 2,         /* device allocation failed */
  VMO_ERR_CUDA = 3,        /* CUDA runtime or kernel failure, or no GPU */
  VMO_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out */
  VMO_ERR_BUDGET = 5,      /* request does not fit the admission budget */
  VMO_ERR_UNSUPPORTED = 6  /* valid but unsupported combination (e.g. d = 5) */
} vmo_status;

/* Hypergraph models of an m x n sparsity pattern (Table 1, Sec. 1.1).
 *  SYMMETRIC: vertices 0..m-1 (m == n), nets {i, j} for a_ij != 0, i != j
 *             (a set: a_ij and a_ji give one net; the diagonal is dropped).
 *  BIPARTITE: vertices rows 0..m-1 then columns m..m+n-1, nets {r_i, c_j}.
 *  ROWNET:    vertices = columns, net i = {c_j : a_ij != 0}.
 *  COLNET:    vertices = rows, net j = {r_i : a_ij != 0}.
 *  FINEGRAIN: vertices = the distinct entries v_ij in row-major order, nets
 *             = the m rows {v_ij : j} then the n columns {v_ij : i}
 *             (m + n nets; every vertex on two).
 * SYMMETRIC and BIPARTITE are graphs; only they can be ordered
 * (Algorithm 7 is stated for graphs). */
typedef enum { VMO_SYMMETRIC = 0, VMO_BIPARTITE = 1, VMO_ROWNET = 2, VMO_COLNET = 3, VMO_FINEGRAIN = 4 } vmo_model;

typedef struct vmo_hg_s* vmo_hg;

/* Sparsity pattern in CSR form: device rowptr[m+1] and colidx[nnz] (int32,
 * 0-based; columns may be unsorted and repeated — duplicates are merged).
 * Values are not used (Sec. 4.2: value-weighted costs were not used). */
typedef struct {
  int32_t m, n;
  int64_t nnz;
  const int32_t* rowptr;
  const int32_t* colidx;
} vmo_csr;

/* Method parameters; vmo_default_params() fills the defaults shown. */
typedef struct {
  int32_t d;            /* layout dimension, 2..4 (default 3) */
  int32_t iters;        /* steepest-descent steps per level, Algorithm 4 (100) */
  float sigma;          /* first step length in units of the mean point spacing (1.0) */
  float decay;          /* step-length decay per step, Sec. 2.3 (0.9) */
  int32_t occupancy;    /* target points per finest grid cell (8) */
  int32_t multilevel;   /* 1: Algorithm 3 coarsening/prolongation; 0: one level (1) */
  int32_t match_rounds; /* handshake matching rounds per coarsening level (4) */
  int32_t coarse_min;   /* stop coarsening at this many vertices (64) */
  int32_t km_iters;     /* Lloyd rounds of 2-means, Algorithm 5 (20) */
  int32_t min_part;     /* a node with <= min_part vertices is a leaf (64) */
  int32_t max_depth;    /* nodes at this depth are leaves, <= 62 (62) */
  int32_t sep_recursion; /* 1: the separator V3 of a split node is ordered recursively as well, by the
                            same bisection over the edges inside V3 (the Schur complement brought into
                            BBD form, Sec. 4.2); child keys then 3h-1, 3h, 3h+1 for V1, V2, V3 and
                            nodes at depth min(max_depth, 39) are leaves.  0: V3 keeps its inherited
                            order (0) */
  int32_t cut_order;    /* b in [0, 8] (with sep_recursion = 0): after the recursion every separator V3
                            is stably sorted by b two-bit numbers per vertex; pair l describes its
                            links into the first / second parts of the splits of the node's
                            descendants l levels down (first bit, value 1: a neighbour in a first part
                            such as V11 or V21; second bit, value 2: in a second part such as V12 or
                            V22); pair 1 sorts first, each pair ascending for BBD and in the order 01,
                            00, 11, 10 for SBD: the cut rows and columns brought into recursive form
                            down to the b-th level (Sec. 4.2) (0: off) */
  int32_t sep_order_free; /* with a strengthened diagonal (vmo_order_matched) only: 0 runs Algorithm 7's
                            loop over the cut edges in canonical order (ascending |x.r - delta|, id of
                            the end it moves, then the other end), where a partner moved early leaves
                            later edges at it uncut; 1 takes the order-free reading (every cut edge's
                            moved end and its partner; a superset) (0) */
  uint64_t seed;        /* seed of every random draw (1) */
} vmo_params;

/* Tree of the recursive ordering, one record per node.  A disconnected graph
 * is ordered component by component (Sec. 2.2: each connected component is
 * treated separately; the matrix is block diagonal), components in order of
 * their smallest vertex id, each with its own recursion whose root has heap
 * number 1 (children of h are 2h (V1) and 2h+1 (V2)).  Records are sorted by
 * (component, heap number), i.e. breadth first within a component.  A leaf
 * has n1 = |V|, n2 = nsep = 0.  An internal node's vertices occupy
 * [offset, offset + n1 + n2 + nsep) of the vertex permutation (absolute
 * positions) as [V1, V2, V3] (BBD) or [V1, V3, V2] (SBD).  Device arrays of
 * `capacity` entries each (component may be NULL); `count` is written (host)
 * on return.  A tree never has more than 2k records. */
typedef struct {
  int32_t capacity;
  int32_t count;
  uint64_t* heap;
  int32_t* offset;
  int32_t* n1;
  int32_t* n2;
  int32_t* nsep;
  int32_t* depth;
  int32_t* component;
} vmo_tree;

/* Counters of the library's own device work since the last vmo_stats_reset
 * (process-wide, all threads): kernels launched; and, when enabled, the
 * device time of the layout step kernel (repulsion + update, timed with CUDA
 * events on the launching stream), its launch count, the target points and the
 * source interactions (near-field pairs plus far-field cell charges) it
 * evaluated; and the device memory allocations the library has made (stream-
 * ordered pool and plain cudaMalloc alike; counted whether or not timing is
 * enabled). */
typedef struct {
  uint64_t launches;
  uint64_t step_launches;
  double step_ms;
  uint64_t step_points;
  uint64_t step_interactions;
  uint64_t device_allocations;
} vmo_stats;

/* Fills *p with the defaults listed above. */
void vmo_default_params(vmo_params* p);

/* Builds the hypergraph model of the pattern `a` on the device (Table 1).
 * vertex_weight: optional device float[k] (NULL = unit weights, Def. 1.1).
 * On success *out owns device copies of the model; free with vmo_destroy.
 * Errors: VMO_ERR_INVALID for null pointers, negative sizes, nnz not equal
 * to rowptr[m], column indices out of range, SYMMETRIC with m != n. */
vmo_status vmo_build_hypergraph(const vmo_csr* a, vmo_model model, const float* vertex_weight,
                                void* stream, vmo_hg* out);

/* Number of vertices k and nets l of the model (host values). */
int32_t vmo_hg_vertices(vmo_hg hg);
int64_t vmo_hg_nets(vmo_hg hg);

/* Device views of the model owned by the handle (valid until vmo_destroy).
 * Graph models: adjacency CSR adj_ptr[k+1], adj[adj_ptr[k]] (neighbours
 * ascending).  Every model: nets CSR net_ptr[l+1], pins (pins ascending;
 * graph models list the edges u < v lexicographically) and the incidence
 * vtx_ptr[k+1], vnets (nets of a vertex ascending).  *count_* receive the
 * lengths of adj / pins / vnets (host).  Pointers may be NULL to skip. */
vmo_status vmo_hg_arrays(vmo_hg hg, const int32_t** adj_ptr, const int32_t** adj, int64_t* count_adj,
                         const int32_t** net_ptr, const int32_t** pins, int64_t* count_pins,
                         const int32_t** vtx_ptr, const int32_t** vnets, int64_t* count_vnets);

/* Connected components (Algorithm 1): labels[v] = smallest vertex id of v's
 * component.  labels: device int32[k]. */
vmo_status vmo_components(vmo_hg hg, int32_t* labels, void* stream);

/* Random initial layout of Algorithm 3: coordinates uniform in [0, s)^d with
 * s the smallest integer with s^d >= k (fp32, exactly reproducible).
 * coords: device float[4k]. */
vmo_status vmo_init_coords(int32_t k, int32_t d, uint64_t seed, float* coords, void* stream);

/* Geometry (Sec. 2): multilevel layout of a graph model (Algorithm 3, with
 * Algorithm 4 on every level), or a single level from the random layout when
 * params->multilevel == 0 or the model is a hypergraph model.  If
 * use_given_init != 0 the single-level layout starts from `coords` instead.
 * coords: device float[4k], written on return. */
vmo_status vmo_layout(vmo_hg hg, const vmo_params* params, float* coords, int32_t use_given_init,
                      void* stream);

/* One steepest-descent step of Algorithm 4 on the finest level with step
 * length `step`: y = gradient of eq. graphenergygradientsimple (repulsion on
 * the grid pyramid), then x_n <- x_n - step * y_n / ||y_n||.
 * coords (in/out) device float[4k]; y_out device float[4k] or NULL;
 * keys_out device uint32[k] or NULL (row-major index of every vertex's
 * level-L grid cell, coordinate 0 fastest);
 * levels_out host int32 or NULL (finest grid level L). */
vmo_status vmo_layout_step(vmo_hg hg, const vmo_params* params, float* coords, float step, float* y_out,
                           uint32_t* keys_out, int32_t* levels_out, void* stream);

/* Coarsening of Algorithm 3 on the handle's graph: level 0 matching into
 * mate (device int32[k], -1 = unmatched) and grouping pi (device int32[k],
 * fine vertex -> coarse vertex), and the vertex counts of every level of the
 * hierarchy (host int32 level_sizes[41]; *nlevels host).  Any output may be
 * NULL.  Graph models only. */
vmo_status vmo_coarsen(vmo_hg hg, const vmo_params* params, int32_t* mate, int32_t* pi, int32_t* kc_out,
                       int32_t* level_sizes, int32_t* nlevels, void* stream);

/* One level of the coarsening hierarchy of Algorithm 3 (Sec. 2.3) built from
 * the handle's whole graph as one problem (the hierarchy whose sizes
 * vmo_coarsen reports; the layout of a connected graph uses the same one).
 * Level 0 is the handle's graph (unit costs; the handle's vertex weights, or
 * 1); level j >= 1 is the graph of the groups of level j-1: a coarse vertex
 * weighs what its group weighs, the fine edges between two groups merge into
 * one edge whose cost is the sum of theirs, edges inside a group vanish.
 * Outputs (device, any may be NULL): adj_ptr int32[k+1] and adj int32[nadj]
 * (neighbours ascending), acost float[nadj] (edge costs), weight float[k]
 * (vertex weights), pi int32[k_{j-1}] (vertex of level j-1 -> its group at
 * level j; untouched for level 0).  *k_out, *nadj_out: host sizes of the
 * level (call once with NULL arrays to size them).
 * Errors: VMO_ERR_INVALID for a level outside [0, levels), VMO_ERR_UNSUPPORTED
 * for hypergraph models. */
vmo_status vmo_hierarchy_level(vmo_hg hg, const vmo_params* params, int32_t level, int32_t* k_out, int64_t* nadj_out,
                               int32_t* adj_ptr, int32_t* adj, float* acost, float* weight, int32_t* pi,
                               void* stream);

/* Prolongation of Algorithm 3 from level `level` (>= 1) of that hierarchy to
 * level-1: fine[v] = f * coarse[pi(v)] + jitter(v) per coordinate m < d, with
 * f = (k_{level-1} / k_level)^(1/d) (the same number of points per unit
 * volume) and jitter(v)_m = 0.1 (u - 1/2), u uniform in [0, 1) from the keyed
 * draw (seed, v, 4 (level-1) + m); coordinates >= d are 0.  coarse: device
 * float[4 k_level], fine: device float[4 k_{level-1}] out, both 16-byte
 * aligned.  Errors: VMO_ERR_INVALID for level 0 or outside the hierarchy. */
vmo_status vmo_hierarchy_prolong(vmo_hg hg, const vmo_params* params, int32_t level, const float* coarse, float* fine,
                                 void* stream);

/* One steepest-descent step of Algorithm 4 on level `level` of that
 * hierarchy, with its vertex weights and edge costs (y = gradient of eq.
 * graphenergygradientsimple, x_n <- x_n - step * y_n / ||y_n||), as
 * vmo_layout_step does on the finest level.  coords: device float[4 k_level]
 * in/out; y_out: device float[4 k_level] or NULL. */
vmo_status vmo_hierarchy_step(vmo_hg hg, const vmo_params* params, int32_t level, float* coords, float step,
                              float* y_out, void* stream);

/* 2-means of the points coords[verts[i]] in dimension d (Algorithm 5 with
 * m = 2, in the exact arithmetic of the ordering): verts device int32[nverts]
 * (vertex ids of hg, in the order the node lists them), labels device
 * uint8[nverts] in {1, 2},
 * centres z device float[8] (z1 then z2), *split host 1 iff both sides are
 * non-empty.  `key` keys the k-means++ draws (the heap number of a node). */
vmo_status vmo_bisect(vmo_hg hg, int32_t d, const float* coords, const int32_t* verts, int32_t nverts,
                      uint64_t seed, uint64_t key, int32_t km_iters, uint8_t* labels, float* z, int32_t* split,
                      void* stream);

/* vmo_bisect for callers that must not allocate device memory (for example
 * when another allocator or a fixed budget owns all device memory, or inside a
 * latency-critical loop where an allocation could block).  The paper has no
 * counterpart: this is a deployment variant of vmo_bisect, without the handle.
 * Same arguments, results and rules as vmo_bisect (verts must be valid rows of
 * coords), but every intermediate lives in one fixed device array that the
 * library reserves on each GPU that loads it (about 5.3 MB, kept until the
 * process exits) instead of in freshly allocated memory; no cudaMalloc or
 * other allocation is made.  Limit: nverts <= 131072, larger inputs return
 * VMO_ERR_INVALID.  Every call looks up the array's device address
 * (cudaGetSymbolAddress, which allocates nothing); the first call on a device
 * also loads the library's device code there, so make that first call before
 * any stream capture.  All calls share the array and it keeps the last call's contents:
 * calls that overlap on the GPU (other streams or threads) race and must be
 * serialised by the caller. */
vmo_status vmo_bisect_noalloc(int32_t d, const float* coords, const int32_t* verts, int32_t nverts, uint64_t seed,
                              uint64_t key, int32_t km_iters, uint8_t* labels, float* z, int32_t* split,
                              void* stream);

/* m-way k-means++ (Algorithm 5 with m centres): the m-way partition C_1..C_m
 * of the points coords[verts[i]] that the paper describes as a one-shot
 * partitioner, in the readings of vmo_bisect (the same draws keyed by
 * (seed, key, centre index), integer D^2 weights, fp32 distances without FMA,
 * ties to the smaller centre, at most km_iters Lloyd rounds ending at the
 * first round without a change, exact fixed-point means); for m = 2 it equals
 * vmo_bisect with labels 0 / 1 for 1 / 2.  If the D^2 weights vanish before m
 * centres are drawn (points on the chosen centres), the remaining centres are
 * copies of the first and stay empty.
 * coords: device float[4] per vertex (16-byte aligned); verts: device int32[nverts];
 * labels: device int32[nverts] out, in [0, m); centres: device float[4 * m] out
 * (16-byte aligned); nonempty: host int32 out, the number of non-empty clusters.
 * Errors: VMO_ERR_INVALID for m outside [1, 256], negative sizes, null or
 * unaligned pointers; VMO_ERR_UNSUPPORTED for d outside 2..4. */
vmo_status vmo_kmeans(int32_t d, const float* coords, const int32_t* verts, int32_t nverts, int32_t m, uint64_t seed,
                      uint64_t key, int32_t km_iters, int32_t* labels, float* centres, int32_t* nonempty,
                      void* stream);

/* Recursive BBD ordering (Sec. 4.2): layout (when coords == NULL) and then
 * recursive bisection with vertex separators placed last.  Symmetric model:
 * row_perm and col_perm (device int32[m]) receive the same permutation.
 * Bipartite model: rows and columns are permuted separately (row_perm[m],
 * col_perm[n]).  tree: optional (NULL), see vmo_tree. */
vmo_status vmo_order_bbd(vmo_hg hg, const float* coords, const vmo_params* params, int32_t* row_perm,
                         int32_t* col_perm, vmo_tree* tree, void* stream);

/* Recursive SBD ordering (Sec. 5): as vmo_order_bbd, with the separator
 * placed between the two parts at every split. */
vmo_status vmo_order_sbd(vmo_hg hg, const float* coords, const vmo_params* params, int32_t* row_perm,
                         int32_t* col_perm, vmo_tree* tree, void* stream);

/* Vertex order of the last ordering step before the row/column split:
 * identical to vmo_order_bbd/sbd but writes the single vertex permutation
 * (device int32[k]) — for the bipartite model rows and columns interleaved
 * as they lie in the recursive partition. */
vmo_status vmo_order_vertices(vmo_hg hg, const float* coords, const vmo_params* params, int32_t sbd,
                              int32_t* perm, vmo_tree* tree, void* stream);

/* Recursive BBD (or SBD) ordering of a square, generally unsymmetric matrix
 * that keeps a strengthened diagonal (Sec. 4.2 and Algorithm 7: a perfect
 * matching M of the bipartite model, seen as the map mu; whenever a vertex
 * joins a separator its partner mu(v) joins too, so no edge of M leaves the
 * diagonal blocks and every block on the diagonal is square).
 * The paper's edge loop gives an order-dependent result once partners move
 * and fixes no order; this entry point runs the loop over the edges cut by
 * the 2-means labels in canonical order (ascending (|x.r - delta|, vertex id)
 * of the end the loop moves, then the other end): an edge still cut when
 * reached moves that end and its partner into V3.  With
 * params->sep_order_free = 1 it takes the order-free reading instead (every
 * cut edge's moved end and its partner; a superset).  With mu the identity
 * both are the separator of vmo_order_bbd.
 * With params->cut_order = b a separator is sorted by the b two-bit numbers
 * of each pair (the row's bits or its matched column's, level by level).
 * hg: bipartite model (VMO_BIPARTITE) of an m x m pattern.
 * match: device int32[m], match[i] = the column matched to row i: a
 * permutation of [0, m) with (i, match[i]) an entry of the pattern.
 * row_perm, col_perm: device int32[m] out; row_perm[t] = the row at position
 * t, col_perm[t] = match[row_perm[t]], so the matched entries form the
 * diagonal of the permuted matrix.  vperm: optional device int32[2m] out, the
 * vertex order (rows 0..m-1, columns m..2m-1, interleaved as they lie in the
 * recursive partition).  tree: optional, in positions of the vertex order
 * (every range holds whole pairs, so halving gives row positions).
 * sbd: 0 BBD [V1, V2, V3], 1 SBD [V1, V3, V2].  coords: NULL (the layout is
 * computed) or device float[4 * 2m].
 * Errors: VMO_ERR_INVALID for a model other than bipartite, a non-square
 * pattern, a null match or output, and a match that is not a perfect
 * matching of the pattern (index out of range, a column used twice, or a
 * pair that is not an entry). */
vmo_status vmo_order_matched(vmo_hg hg, const float* coords, const vmo_params* params, int32_t sbd,
                             const int32_t* match, int32_t* row_perm, int32_t* col_perm, int32_t* vperm,
                             vmo_tree* tree, void* stream);

/* ------------------------------------------------------------------------
 * Matrix Market files (host I/O; no counterpart in the paper, whose test
 * matrices come in this format).  A host CSR: row-major, columns sorted
 * within a row, duplicate entries summed; arrays allocated with malloc by
 * vmo_read_matrix_market and released with vmo_free_host_csr.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t m, n;
  int64_t nnz;
  int32_t* rowptr; /* m + 1 */
  int32_t* colidx; /* nnz */
  float* values;   /* nnz (pattern files: 1; complex files: the modulus) */
} vmo_host_csr;

/* Reads a coordinate Matrix Market file (fields real, integer, complex,
 * pattern; symmetry general, symmetric, skew-symmetric, hermitian).
 * expand_symmetric: 1 stores both triangles of symmetric storage (a_ji =
 * a_ij, -a_ij for skew-symmetric), 0 keeps the stored triangle.
 * Errors: VMO_ERR_INVALID for a missing file or a malformed header, size
 * line or entry (index outside the matrix); VMO_ERR_UNSUPPORTED for array
 * (dense) files and sizes beyond 2^30; VMO_ERR_OOM. *out is zeroed on
 * error. */
vmo_status vmo_read_matrix_market(const char* path, int32_t expand_symmetric, vmo_host_csr* out);

/* Writes a host CSR as a general coordinate file (pattern = 1: no values).
 * Errors: VMO_ERR_INVALID for null arguments or a file that cannot be
 * written. */
vmo_status vmo_write_matrix_market(const char* path, const vmo_host_csr* csr, int32_t pattern);

/* Releases the arrays of a CSR filled by vmo_read_matrix_market (NULL-safe). */
void vmo_free_host_csr(vmo_host_csr* csr);

/* Strengthened diagonal for vmo_order_matched, computed on the host: a
 * perfect matching of the bipartite model of the square pattern (rows to
 * columns), as the paper obtains it for its LU experiments (Sec. 5): a
 * heavy-edge matching (entries by decreasing |value|, ties by row then
 * column, each taken when its row and column are both free; without values,
 * every row in order takes its first free column) augmented by the
 * Hopcroft-Karp algorithm to a maximum matching.  Host preprocessing of the
 * input, outside the ordering's GPU path; it touches no device memory.
 * rowptr, colidx: HOST arrays of an m x m pattern (int32[m + 1], int32[nnz]);
 * values: optional host float[nnz] (NULL: pattern only); match: host
 * int32[m] out, match[i] = the column matched to row i (-1 if unmatched);
 * matched: optional host out, the size of the maximum matching.
 * Errors: VMO_ERR_INVALID for a malformed pattern or a NaN value;
 * VMO_ERR_UNSUPPORTED when the pattern is structurally singular (no perfect
 * matching exists: match then holds a maximum matching). */
vmo_status vmo_perfect_matching_host(int32_t m, const int32_t* rowptr, const int32_t* colidx, const float* values,
                                     int32_t* match, int32_t* matched);

/* Batched recursive ordering of `count` independent square patterns in one
 * launch sequence (symmetric model).  The matrices are joined
 * block-diagonally on the device and every connected component of every
 * matrix is laid out and ordered as one problem of a single batch; the result
 * for each matrix is identical, bit for bit, to vmo_order_vertices on that
 * matrix alone with the same params (no arithmetic depends on the batch).
 * mats: host array of `count` vmo_csr (device pointers inside).
 * coords: NULL (the layout is computed) or device float[4 sum_i m_i], the
 * matrices' coordinates one after the other (ordering only, Sec. 5 "O").
 * perm: device int32[sum_i m_i]; matrix i's permutation (perm[new] = old, local
 * row indices) starts at offset sum_{j<i} m_j.  sbd: 0 BBD, 1 SBD.
 * Errors: VMO_ERR_INVALID for count < 0, a null list, a non-square or
 * malformed matrix; VMO_ERR_UNSUPPORTED beyond 2^30 rows or 2^31 nonzeros in
 * total. */
vmo_status vmo_batch_order(const vmo_csr* mats, int32_t count, const float* coords, const vmo_params* params,
                           int32_t sbd, int32_t* perm, void* stream);

/* Batched geometry only (multilevel layout of every connected component of
 * every matrix as one batch, symmetric model): coords device float[4 sum_i m_i],
 * matrix i's coordinates at row offset sum_{j<i} m_j; identical, bit for bit,
 * to vmo_layout of each matrix alone.  Errors as vmo_batch_order. */
vmo_status vmo_batch_layout(const vmo_csr* mats, int32_t count, const vmo_params* params, float* coords,
                            void* stream);

/* Finegrain layout from the bipartite one (Sec. 4.2: the finegrain model's
 * dual is the bipartite graph; laying that out and placing every entry a_ij
 * at the mean of the points of row r_i and column c_j gives a finegrain
 * layout at the cost of a 2m-vertex layout instead of an nnz-vertex one).
 * hg: a FINEGRAIN handle of the pattern; bipartite_coords: device
 * float[4 (m + n)] (16-byte aligned), the coordinates of the BIPARTITE model
 * of the same pattern (rows, then columns), e.g. from vmo_layout;
 * coords: device float[4 k] out (k = distinct entries), entry t at
 * 0.5 (x(row) + x(column)) in fp32 per coordinate.  The result feeds
 * vmo_bisect / vmo_kmeans (a partition of the entries) and vmo_cut_size on
 * the finegrain handle (cut rows and columns of that partition).
 * Errors: VMO_ERR_INVALID for a handle of another model, null or unaligned
 * pointers. */
vmo_status vmo_finegrain_coords(vmo_hg hg, const float* bipartite_coords, float* coords, void* stream);

/* ------------------------------------------------------------------------
 * Launch-shape tuning (no counterpart in the paper: choices of this GPU
 * implementation).  None of these settings changes any result, bit for bit;
 * they only change how the work is split into launches:
 *   small_step_threads: layout step launches of at most this many threads
 *     use the step-kernel variant with two far-field rows in flight per lane
 *     (latency hiding for small levels); default 19,456 (4 warps per SM);
 *   radix_max_bits: widest digit of the binning sort's LSD passes, 8, 9 or
 *     10 (default 10: fewest passes);
 *   assign_items: positions per thread of the Lloyd assignment, 1, 2, 4 or
 *     8 (default 4; fewer are used when the blocks would not fill the GPU);
 *   small_bin_points: a layout level whose problems all have at most this
 *     many vertices (0 ... 2,048) is binned by one block per problem (keys,
 *     sort, gather and cell charges in one launch) instead of the device-wide
 *     sequence; 0 turns it off (default 2,048).
 * The setting is process-wide and read at every launch.
 * ------------------------------------------------------------------------ */
typedef struct {
  int64_t small_step_threads;
  int32_t radix_max_bits;
  int32_t assign_items;
  int32_t small_bin_points;
} vmo_tuning;

/* Current setting (host struct out). */
void vmo_get_tuning(vmo_tuning* out);

/* Sets all four choices.  Errors: VMO_ERR_INVALID for a null pointer or a
 * value outside the ranges above (nothing is changed then).  Not to be called
 * while another thread is inside a library call. */
vmo_status vmo_set_tuning(const vmo_tuning* tuning);

/* Timed search for the setting that orders the given matrices fastest: from
 * the current setting, each choice in turn over its candidates
 * (small_step_threads 0 ... 155,648; radix_max_bits 8, 9, 10; assign_items
 * 1, 2, 4, 8; small_bin_points 0, 512, 2,048), every candidate timed as the median of `reps` calls of
 * vmo_batch_order(mats, count, NULL, params, BBD) after one untimed call, with
 * CUDA events on `stream`.  The fastest becomes the process-wide setting.
 * mats: host array of `count` vmo_csr (device pointers inside), as for
 * vmo_batch_order; best (host, optional): the chosen setting; best_ms /
 * default_ms (host, optional): its time and the starting setting's time.
 * Allocates one device permutation buffer for the duration of the call.
 * Errors: those of vmo_batch_order (the setting is restored then);
 * VMO_ERR_INVALID for count <= 0 or reps outside [1, 100]. */
vmo_status vmo_autotune(const vmo_csr* mats, int32_t count, const vmo_params* params, int32_t reps,
                        vmo_tuning* best, double* best_ms, double* default_ms, void* stream);

/* Cut metrics of a vertex partition (Sec. 4.1 footnote, Sec. 5): over the
 * nets of the model, lambda_e = number of distinct parts among the pins;
 * cutnet = #{e : lambda_e > 1}, lambda1 = sum_e (lambda_e - 1).
 * part: device int32[k] in [0, nparts).  cutnet, lambda1: host int64.
 * Errors: VMO_ERR_INVALID for nparts < 1. */
vmo_status vmo_cut_size(vmo_hg hg, const int32_t* part, int32_t nparts, int64_t* cutnet, int64_t* lambda1,
                        void* stream);

/* ------------------------------------------------------------------------
 * Request server: continuous batching of ordering requests.
 *
 * The paper orders one matrix at a time; the server serves a stream of
 * ordering requests of mixed sizes on one GPU.  A request is a square
 * pattern in HOST memory; the result is the recursive BBD (or SBD)
 * permutation of the symmetric model, bit-identical to vmo_batch_order /
 * vmo_order_bbd of that matrix alone with the same parameters.
 *
 * Scheduling: `slots` host workers, each with its own non-blocking CUDA
 * stream.  A free slot takes the oldest queued requests (at most max_batch,
 * at most max_batch_nnz nonzeros unless a single request is larger) whose
 * estimated device memory (vmo_server_estimate_bytes) fits what is left of
 * budget_bytes, copies their patterns to the device, orders them as one batch
 * (vmo_batch_order) and copies each permutation to its host buffer.  Requests
 * that arrive while others run are admitted as soon as a slot and budget are
 * free, and their work overlaps on the device with the running batches.
 * Coordinates, recursion trees and scratch stay on the device until the batch
 * completes.  Times are seconds since vmo_server_create (steady clock).
 * ------------------------------------------------------------------------ */
typedef struct vmo_server_s* vmo_server;

typedef struct {
  vmo_params params;      /* ordering parameters of every request */
  int32_t sbd;            /* 0: BBD [V1,V2,V3]; 1: SBD [V1,V3,V2] */
  int32_t slots;          /* concurrent batches (host workers + streams), 1..64 (default 4) */
  int32_t max_batch;      /* requests per batch, >= 1 (default 256) */
  int64_t max_batch_nnz;  /* nonzeros per batch (default 8,000,000) */
  int64_t budget_bytes;   /* device memory admitted requests may hold, by estimate;
                             0: half of the free device memory at creation */
} vmo_server_config;

typedef enum {
  VMO_REQ_QUEUED = 0,
  VMO_REQ_RUNNING = 1,
  VMO_REQ_DONE = 2,
  VMO_REQ_FAILED = 3,
  VMO_REQ_CANCELLED = 4
} vmo_request_state;

typedef struct {
  int32_t state;          /* vmo_request_state */
  int32_t status;         /* vmo_status of a failed request, else VMO_OK */
  int64_t n, nnz;
  int64_t bytes;          /* admission estimate */
  double t_submit, t_admit, t_done;  /* seconds; t_done - t_submit is the latency */
  int64_t batch;          /* sequence number of the batch that ran it (-1 before admission) */
  int32_t batch_size;     /* requests in that batch */
  int32_t slot;           /* slot that ran it */
} vmo_request_info;

typedef struct {
  int64_t submitted, completed, failed, cancelled, queued, running;
  int64_t batches;
  int64_t nnz_completed;
  int64_t budget_bytes, bytes_in_use, bytes_peak;  /* by estimate */
  int64_t pool_peak_bytes;  /* high-water mark of the device pool (measured) */
} vmo_server_stats;

/* Fills the defaults shown above (params = vmo_default_params()). */
void vmo_server_default_config(vmo_server_config* cfg);

/* Device-memory estimate used for admission of an n x n request with nnz
 * nonzeros: 512 n + 64 nnz + 1 MiB bytes (model, hierarchy, layout and
 * ordering scratch). */
int64_t vmo_server_estimate_bytes(int64_t n, int64_t nnz);

/* The admission rule of a free slot, exposed for inspection: given the
 * queue's estimates and nonzeros (host arrays, oldest first), the memory
 * still free in the budget and the batch limits, returns how many requests
 * from the head form the next batch (0: the head does not fit yet).  The head
 * is always taken if it fits, even above max_batch_nnz. */
int32_t vmo_server_plan(const int64_t* bytes, const int64_t* nnz, int32_t count, int64_t budget_free,
                        int32_t max_batch, int64_t max_batch_nnz);

/* Creates a server on the current device and starts its slots.
 * Errors: VMO_ERR_INVALID for a bad config, VMO_ERR_CUDA without a GPU. */
vmo_status vmo_server_create(const vmo_server_config* cfg, vmo_server* out);

/* Queues one request.  rowptr[n+1], colidx[nnz] and perm_out[n] are HOST
 * arrays that must stay valid until the request is terminal (done, failed or
 * cancelled); the pattern is validated here (square, rowptr monotone from 0
 * to nnz, columns in range).  *id receives the request id (> 0).
 * Errors: VMO_ERR_INVALID (malformed pattern or null), VMO_ERR_BUDGET (the
 * estimate alone exceeds the budget), VMO_ERR_INVALID after shutdown began. */
vmo_status vmo_server_submit(vmo_server srv, int32_t n, const int32_t* rowptr, const int32_t* colidx,
                             int32_t* perm_out, uint64_t* id);

/* State of a request (host).  Errors: VMO_ERR_INVALID for an unknown id. */
vmo_status vmo_server_poll(vmo_server srv, uint64_t id, vmo_request_info* info);

/* Blocks until the request is terminal or timeout_s seconds pass (< 0: no
 * limit); returns VMO_ERR_TIMEOUT in the latter case, info filled either way. */
vmo_status vmo_server_wait(vmo_server srv, uint64_t id, double timeout_s, vmo_request_info* info);

/* Cancels a request: a queued one never runs and is cancelled at once; a
 * running one stays VMO_REQ_RUNNING (its batch may still read its host
 * arrays) and becomes VMO_REQ_CANCELLED, with nothing written, when its batch
 * ends.  No effect on terminal ones. */
vmo_status vmo_server_cancel(vmo_server srv, uint64_t id);

/* Forgets a terminal request (done, failed or cancelled): its record is freed
 * and its id becomes unknown, so a long-running server does not grow by one
 * record per request.  Errors: VMO_ERR_INVALID for an unknown id or a request
 * that is still queued or running. */
vmo_status vmo_server_release(vmo_server srv, uint64_t id);

vmo_status vmo_server_get_stats(vmo_server srv, vmo_server_stats* out);

/* Stops admission, lets running batches finish, cancels what is still
 * queued and frees the server (NULL is ignored). */
void vmo_server_destroy(vmo_server srv);

/* Measured arithmetic throughput of the current GPU, the ceiling of the
 * layout step kernel (no counterpart in the paper; measurement support):
 * FP32 fused multiply-add, scalar (ffma) and packed two-lane (ffma2), in
 * TFLOP/s counting a multiply-add as 2 flops, and the special-function
 * unit's approximate reciprocal square root in T operations/s; sms receives
 * the number of SMs.  Each figure is the best of a few launches that fill
 * every SM with independent dependency chains (a few ms in all), at the
 * clock the GPU runs at.  Any output may be NULL (that kernel is skipped). */
vmo_status vmo_measure_alu_peaks(double* ffma_tflops, double* ffma2_tflops, double* rsqrt_tops, int32_t* sms,
                                 void* stream);

/* Resets the counters.  time_step_kernel != 0 records CUDA events around
 * every layout step kernel; count_interactions != 0 makes that kernel count
 * its interactions (an atomic per warp; same arithmetic otherwise). */
void vmo_stats_reset(int32_t time_step_kernel, int32_t count_interactions);

/* Reads the counters (synchronises the device when kernel timing is on). */
vmo_status vmo_stats_get(vmo_stats* out);

/* Frees the handle and its device arrays (NULL is ignored). */
void vmo_destroy(vmo_hg hg);

/* Static description of a status code. */
const char* vmo_status_string(vmo_status s);

/* Message of the calling thread's last failing call ("" if none). */
const char* vmo_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VMO_H */
