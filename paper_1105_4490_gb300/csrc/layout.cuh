// Layout engine shared by the plain, batched and served paths.
#pragma once

#include <memory>

#include "vmo_internal.cuh"

namespace vmo {

// Per-problem constants of one level of a batch (device copy in LevelBatch).
struct ProbDev {
  int64_t vbase;   // first vertex of the problem in the level
  int64_t cbase;   // first entry of its cell tables (all levels 0..L)
  int64_t fbase;   // first entry of its finest-level cell ranges
  int64_t tbase;   // first thread of its targets in the step kernel (multiple of 32)
  int32_t k;       // vertices
  int32_t L;       // finest grid level
  int32_t side;    // side of the random initial box
  int32_t group;   // lanes per target in the step kernel (power of two <= 32)
};

// One level of the multilevel hierarchy for a batch of independent problems
// (one problem in plain mode).  Vertex ids are global to the level; problems
// occupy consecutive vertex ranges.
struct LevelBatch {
  int64_t K = 0;                 // vertices
  int32_t P = 0;                 // problems in this level
  std::vector<int64_t> vbase;    // host, P+1
  std::vector<int32_t> src;      // host, P: index of the problem in the batch
  std::vector<int32_t> L;        // host, P
  std::vector<int64_t> cbase;    // host, P+1
  std::vector<int64_t> fbase;    // host, P+1
  // graph of the level (device)
  const int32_t* adj_ptr = nullptr;
  const int32_t* adj = nullptr;
  const float* acost = nullptr;  // null: unit costs
  const float* w = nullptr;      // null: unit weights
  int64_t nadj = 0;
  // hypergraph nets (rownet / colnet, single level only)
  const int32_t* net_ptr = nullptr;
  const int32_t* pins = nullptr;
  const int32_t* vtx_ptr = nullptr;
  const int32_t* vnets = nullptr;
  int64_t nnets = 0;
  // device tables
  DevArray<ProbDev> prob;
  DevArray<int32_t> vprob;       // K: problem index of every vertex
  DevArray<int64_t> aggoff;      // (maxL-1) x (P+1): prefix of coarse-level cell counts
  int32_t maxL = 1;
  DevArray<int64_t> tbase;       // P+1: thread bases of the step kernel
  DevArray<int64_t> fbase_dev;   // P+1: fbase on the device
  int64_t threads = 0;           // threads of the step kernel
  // vertices by degree class (graph models): medium and heavy rows get a warp
  // or a block each in the gather kernels
  DevArray<int32_t> mid_list, heavy_list;
  int64_t n_mid = 0, n_heavy = 0;
  // storage of coarse levels built by the coarsening
  DevArray<int32_t> own_adj_ptr, own_adj;
  DevArray<float> own_acost, own_w;
};

struct LayoutOptions {
  int d = 3;
  int iters = 100;
  float sigma = 1.0f;
  float decay = 0.9f;
  int occupancy = 8;
};

// Fills the per-problem tables of a level (L, cell bases, device copies).
vmo_status level_setup(LevelBatch& lb, int d, int occupancy, cudaStream_t s);

// Runs `iters` steps of Algorithm 4 on a level.  x: device float4[K] in/out.
// If step_override > 0 it is used as the step length of a single step and
// y_out / keys_out (vertex order, may be null) receive the gradient and keys.
vmo_status layout_level(LevelBatch& lb, const LayoutOptions& o, float4* x, int iters, float step_override,
                        float4* y_out, uint32_t* keys_out, cudaStream_t s, Scratch& sc);

// Random initial layout of the problems of a level (all, or those with
// start[p] != 0 when start_dev is given).  seeds_dev: device uint64[P].
vmo_status init_coords_level(LevelBatch& lb, int d, const uint64_t* seeds_dev, float4* x, const int32_t* start_dev,
                             cudaStream_t s);

// Multilevel layout (Algorithm 3) of a level-0 batch.  seeds: one seed per
// problem (host).  x: device float4[K] out.  Hypergraph models and
// multilevel == false run a single level from the random layout.
vmo_status layout_multilevel(LevelBatch& fine, const LayoutOptions& o, const std::vector<uint64_t>& seeds,
                             int match_rounds, int coarse_min, bool multilevel, float4* x, cudaStream_t s,
                             Scratch& sc);

// Matching and grouping of level j for the problems flagged in active_dev:
// mate, anchor and the exclusive rank of anchors; kc receives the coarse
// vertex count of every problem (host).
vmo_status coarsen_level(LevelBatch& lb, const uint64_t* seeds_dev, int j, int rounds, const int32_t* active_dev,
                         int32_t* mate, int32_t* anchor, int32_t* rank, std::vector<int64_t>& kc, cudaStream_t s,
                         Scratch& sc);

// Coarsening hierarchy of Algorithm 3: levels[0] is the fine batch,
// pis[j] maps level j to level j+1 (-1 for problems that stop at level j).
struct Hierarchy {
  std::vector<LevelBatch*> levels;
  std::vector<std::unique_ptr<LevelBatch>> owned;
  std::vector<int32_t*> pis;
  std::vector<std::vector<uint64_t>> seeds;
};

vmo_status build_hierarchy(LevelBatch& fine, const LayoutOptions& o, const std::vector<uint64_t>& seeds,
                           int match_rounds, int coarse_min, bool multilevel, Hierarchy& H, cudaStream_t s,
                           Scratch& sc);

// Start of level j of a hierarchy (the levels above it already laid out):
// problems that continue from level j+1 are prolonged from its coordinates xc
// (Algorithm 3: x = f x_c(pi(v)) + jitter, f = (k_j / k_{j+1})^(1/d)), the
// others (and every problem when xc is null) get the random initial layout.
vmo_status prolong_level(const Hierarchy& H, int j, int d, const float4* xc, float4* xj, cudaStream_t s,
                         Scratch& sc);

int grid_levels(int64_t k, int d, int occ);
int init_side(int64_t k, int d);

}  // namespace vmo
