// Ordering engine (recursive 2-means bisection with vertex separators).
#pragma once

#include "vmo_internal.cuh"

namespace vmo {

// One node of the recursion (device).
struct NodeDev {
  uint64_t heap;        // heap number (root 1, children 2h, 2h+1; with separator recursion 3h-1, 3h, 3h+1)
  int64_t off;          // first position of the node
  int32_t size;
  int32_t depth;
  int32_t prob;         // problem of the batch
  int32_t e;            // fixed-point exponent: max |x| < 2^e
  uint32_t maxabs;      // float bits of max |x| (atomicMax)
  int32_t state;        // 0 iterating, 1 converged, 2 not splittable
  int32_t changed;
  int32_t c1, c2, c3;   // sizes after the separator
  int32_t child1, child2, child3;
  float4 z1, z2;
  long long S1[4], S2[4];
  long long n1, n2;
};

// Tree records (device arrays of capacity cap; count is a device counter).
struct TreeDev {
  uint64_t* heap = nullptr;
  int32_t* prob = nullptr;
  int32_t* offset = nullptr;
  int32_t* n1 = nullptr;
  int32_t* n2 = nullptr;
  int32_t* nsep = nullptr;
  int32_t* depth = nullptr;
  int32_t* count = nullptr;
  int cap = 0;
};

struct OrderParams {
  int d = 3;
  int km_iters = 20;
  int min_part = 64;
  int max_depth = 62;
  int sbd = 0;
  int sep_rec = 0;  // order V3 recursively too (ternary keys, depth <= kSepRecMaxDepth)
  int cut_order = 0;  // b: sort every separator by b two-bit link numbers (without sep_rec)
  int mu_order_free = 0;  // with a strengthened diagonal: 0 Algorithm 7's loop in canonical order, 1 order-free
};

// Deepest node with separator recursion: ternary keys (3^(d+1) - 1) / 2 fit 64 bits up to d = 39.
constexpr int kSepRecMaxDepth = 39;

// Working state of the ordering of a batch of problems (all device).
struct OrderState {
  int64_t n = 0;                      // positions (all problems)
  int32_t* ord = nullptr;             // vertex at each position
  float4* xo = nullptr;               // its coordinates
  int32_t* seg = nullptr;             // active node of each position, -1 if none
  uint8_t* lab = nullptr;             // 2-means label of each position
  uint64_t* vrec = nullptr;           // per vertex: (node << 2 | 2-means label, 0 if not in a split node) and
                                      // the plane distance, one word (written by the separator phase)
  int64_t* pbase = nullptr;           // first position of every problem (P+1)
  uint64_t* seeds = nullptr;          // seed of every problem
  const int32_t* adj_ptr = nullptr;   // graph (global vertex ids)
  const int32_t* adj = nullptr;
  const int32_t* mu = nullptr;        // matching partner of every vertex (strengthened diagonal) or null
  uint8_t* vpick = nullptr;           // separator selection of each vertex (with mu)
  NodeDev* nodes = nullptr;
  int node_cap = 0;
  int nroots = 0;
  TreeDev tree;
};

// Positions start as init_ord (vertex ids; null: identity), grouped by problem
// as pbase_host gives.  Tree offsets are absolute positions.
vmo_status order_setup(OrderState& st, const float4* x, const std::vector<int64_t>& pbase_host,
                       const std::vector<uint64_t>& seeds, const OrderParams& op, const uint32_t* init_ord,
                       cudaStream_t s, Scratch& sc);
vmo_status two_means(OrderState& st, int N, int d, int km_iters, cudaStream_t s, Scratch& sc);
// two_means with every buffer supplied by the caller (allocates nothing):
// dval, dpre hold st.n values, partial scan_partials_needed(st.n), cnt one int.
vmo_status two_means_into(OrderState& st, int N, int d, int km_iters, unsigned long long* dval,
                          unsigned long long* dpre, int* cnt, uint64_t* partial, cudaStream_t s);
vmo_status order_levels(OrderState& st, const OrderParams& op, cudaStream_t s, Scratch& sc);
// Separators stably sorted by b two-bit link numbers (after order_levels).
vmo_status cut_order_pass(OrderState& st, const OrderParams& op, cudaStream_t s, Scratch& sc);
// Indices of the tree records sorted by heap number (and by problem first when
// by_prob); *count_out receives the number of records (host).
vmo_status tree_sorted(OrderState& st, bool by_prob, int32_t* count_out, uint32_t** idx_out, cudaStream_t s,
                       Scratch& sc);
// xo[i] = x[ord[i]]
vmo_status gather_coords(const float4* x, const int32_t* ord, int64_t n, float4* xo, cudaStream_t s);
vmo_status tree_write(OrderState& st, const uint32_t* idx, int n, uint64_t* heap, int32_t* offset, int32_t* n1,
                      int32_t* n2, int32_t* nsep, int32_t* depth, int32_t* prob, cudaStream_t s);

}  // namespace vmo
