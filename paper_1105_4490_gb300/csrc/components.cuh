// Grouping of a graph model by connected components.
#pragma once

#include "layout.cuh"
#include "order.cuh"

namespace vmo {

struct ComponentGroups {
  int64_t k = 0;
  std::vector<int64_t> base;   // host, ncomp+1: first position of each component
  uint32_t* cperm = nullptr;   // device, k: vertices component by component (ascending inside)
  int32_t* cinv = nullptr;     // device, k: position of every vertex
};

// Components (Algorithm 1) and the grouping permutation.
vmo_status group_components(const vmo_hg_s* h, ComponentGroups& g, cudaStream_t s, Scratch& sc);

// Level-0 batch of the graph relabelled by the grouping: one problem per
// component (block diagonal adjacency, weights permuted).
vmo_status relabel_graph(const vmo_hg_s* h, const ComponentGroups& g, LevelBatch& lb, cudaStream_t s, Scratch& sc);

// x[cperm[i]] = xp[i].
vmo_status unpermute_coords(const ComponentGroups& g, const float4* xp, float4* x, cudaStream_t s);

inline LayoutOptions options_of(const vmo_params* p) {
  LayoutOptions o;
  o.d = p->d;
  o.iters = p->iters;
  o.sigma = p->sigma;
  o.decay = p->decay;
  o.occupancy = p->occupancy;
  return o;
}

// Multilevel layout of a graph model, one problem per component (x in vertex
// order of the handle).
vmo_status layout_grouped(const vmo_hg_s* h, const ComponentGroups& g, const vmo_params* p, float4* x,
                          cudaStream_t s, Scratch& sc);

// Recursive ordering of a graph model from coordinates x: every component
// from its own root, components one after the other.  st.ord holds the
// vertex permutation on return.  mu: matching partner of every vertex
// (device int32[k], a strengthened diagonal) or null.
vmo_status order_grouped(const vmo_hg_s* h, const ComponentGroups& g, const float4* x, const vmo_params* p, int sbd,
                         OrderState& st, cudaStream_t s, Scratch& sc, const int32_t* mu = nullptr);

}  // namespace vmo
