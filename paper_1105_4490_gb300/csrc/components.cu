// Connected-component grouping (Sec. 2.2: a disconnected hypergraph has no
// minimum-energy layout, so every component is treated separately).
//
// Components are numbered by their smallest vertex (the label of
// Algorithm 1).  cperm lists the vertices component by component, ascending
// inside a component (a stable radix sort of the labels), so relabelling the
// graph by cinv = cperm^-1 keeps every adjacency list ascending and makes the
// graph block diagonal with one block per component: exactly the layout of a
// batch of independent problems.
#include <algorithm>

#include "components.cuh"

namespace vmo {

vmo_status components(const vmo_hg_s* h, int32_t* labels, cudaStream_t s);

namespace {

__global__ void k_iota_u32(uint32_t* a, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (uint32_t)i;
}

__global__ void k_run_starts(const uint32_t* __restrict__ slab, int64_t n, int32_t* __restrict__ flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (i == 0 || slab[i - 1] != slab[i]) ? 1 : 0;
}

__global__ void k_bases(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t n,
                        int64_t* __restrict__ base) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) base[pos[i]] = i;
}

__global__ void k_inverse(const uint32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ inv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) inv[perm[i]] = (int32_t)i;
}

__global__ void k_perm_degree(const uint32_t* __restrict__ perm, const int32_t* __restrict__ ptr, int64_t n,
                              int32_t* __restrict__ deg) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    uint32_t v = perm[i];
    deg[i] = ptr[v + 1] - ptr[v];
  }
}

__global__ void k_relabel_adj(const uint32_t* __restrict__ perm, const int32_t* __restrict__ inv,
                              const int32_t* __restrict__ ptr, const int32_t* __restrict__ adj, int64_t n,
                              const int32_t* __restrict__ nptr, int32_t* __restrict__ nadj) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t v = perm[i];
  int32_t o = nptr[i];
  for (int32_t t = ptr[v]; t < ptr[v + 1]; ++t) nadj[o++] = inv[adj[t]];
}

__global__ void k_perm_float(const uint32_t* __restrict__ perm, const float* __restrict__ a, int64_t n,
                             float* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[perm[i]];
}

__global__ void k_unpermute_coords(const uint32_t* __restrict__ perm, const float4* __restrict__ xp, int64_t n,
                                   float4* __restrict__ x) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[perm[i]] = xp[i];
}

__global__ void k_set_last(int32_t* ptr, int64_t n, const int32_t* total) { ptr[n] = *total; }

}  // namespace

vmo_status group_components(const vmo_hg_s* h, ComponentGroups& g, cudaStream_t s, Scratch& sc) {
  const int64_t k = h->k;
  g.k = k;
  int32_t* lab;
  uint32_t *ids, *slab;
  int32_t *flag, *pos, *total;
  VMO_TRY(sc.alloc(&lab, std::max<int64_t>(k, 1)));
  VMO_TRY(sc.alloc(&ids, std::max<int64_t>(k, 1)));
  VMO_TRY(sc.alloc(&slab, std::max<int64_t>(k, 1)));
  VMO_TRY(sc.alloc(&g.cperm, std::max<int64_t>(k, 1)));
  VMO_TRY(sc.alloc(&g.cinv, std::max<int64_t>(k, 1)));
  VMO_TRY(sc.alloc(&flag, std::max<int64_t>(k, 1)));
  VMO_TRY(sc.alloc(&pos, std::max<int64_t>(k, 1)));
  VMO_TRY(sc.alloc(&total, 1));
  g.base.assign(1, 0);
  if (k == 0) return VMO_OK;
  VMO_TRY(components(h, lab, s));
  launch(k_iota_u32, grid_for(k, 256), 256, 0, s, ids, k);
  VMO_TRY(radix_sort_u32((uint32_t*)lab, ids, slab, g.cperm, k, bits_for((uint64_t)k), nullptr, s, sc));
  launch(k_run_starts, grid_for(k, 256), 256, 0, s, slab, k, flag);
  VMO_LAUNCHED("run_starts");
  VMO_TRY(scan_exclusive<int32_t>(flag, pos, k, total, s, sc));
  int32_t P = 0;
  VMO_CUDA(cudaMemcpyAsync(&P, total, 4, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  int64_t* dbase;
  VMO_TRY(sc.alloc(&dbase, P + 1));
  launch(k_bases, grid_for(k, 256), 256, 0, s, flag, pos, k, dbase);
  launch(k_inverse, grid_for(k, 256), 256, 0, s, g.cperm, k, g.cinv);
  VMO_LAUNCHED("bases");
  g.base.resize(P + 1);
  VMO_CUDA(cudaMemcpyAsync(g.base.data(), dbase, P * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  g.base[P] = k;
  return VMO_OK;
}

vmo_status relabel_graph(const vmo_hg_s* h, const ComponentGroups& g, LevelBatch& lb, cudaStream_t s, Scratch& sc) {
  const int64_t k = g.k;
  const int P = (int)g.base.size() - 1;
  int32_t *deg, *total;
  VMO_TRY(lb.own_adj_ptr.resize((size_t)k + 1));
  VMO_TRY(lb.own_adj.resize((size_t)std::max<int64_t>(h->nadj, 1)));
  VMO_TRY(sc.alloc(&deg, std::max<int64_t>(k, 1)));
  VMO_TRY(sc.alloc(&total, 1));
  if (k > 0) {
    launch(k_perm_degree, grid_for(k, 256), 256, 0, s, g.cperm, h->adj_ptr.ptr, k, deg);
    VMO_LAUNCHED("perm_degree");
  }
  VMO_TRY(scan_exclusive<int32_t>(deg, lb.own_adj_ptr.ptr, k, total, s, sc));
  launch(k_set_last, 1, 1, 0, s, lb.own_adj_ptr.ptr, k, total);
  if (k > 0)
    launch(k_relabel_adj, grid_for(k, 256), 256, 0, s, g.cperm, g.cinv, h->adj_ptr.ptr, h->adj.ptr, k,
           lb.own_adj_ptr.ptr, lb.own_adj.ptr);
  VMO_LAUNCHED("relabel_adj");
  lb.K = k;
  lb.P = P;
  lb.vbase = g.base;
  lb.src.resize(P);
  for (int p = 0; p < P; ++p) lb.src[p] = p;
  lb.adj_ptr = lb.own_adj_ptr.ptr;
  lb.adj = lb.own_adj.ptr;
  lb.nadj = h->nadj;
  lb.acost = nullptr;
  lb.w = nullptr;
  if (h->has_weight) {
    VMO_TRY(lb.own_w.resize((size_t)std::max<int64_t>(k, 1)));
    if (k > 0) launch(k_perm_float, grid_for(k, 256), 256, 0, s, g.cperm, (const float*)h->weight.ptr, k, lb.own_w.ptr);
    VMO_LAUNCHED("perm_weight");
    lb.w = lb.own_w.ptr;
  }
  return VMO_OK;
}

vmo_status unpermute_coords(const ComponentGroups& g, const float4* xp, float4* x, cudaStream_t s) {
  if (g.k == 0) return VMO_OK;
  launch(k_unpermute_coords, grid_for(g.k, 256), 256, 0, s, g.cperm, xp, g.k, x);
  VMO_LAUNCHED("unpermute_coords");
  return VMO_OK;
}

vmo_status layout_grouped(const vmo_hg_s* h, const ComponentGroups& g, const vmo_params* p, float4* x,
                          cudaStream_t s, Scratch& sc) {
  LevelBatch lb;
  VMO_TRY(relabel_graph(h, g, lb, s, sc));
  VMO_TRY(level_setup(lb, p->d, p->occupancy, s));
  std::vector<uint64_t> seeds(lb.P, p->seed);
  float4* xp;
  VMO_TRY(sc.alloc(&xp, std::max<int64_t>(h->k, 1)));
  VMO_TRY(layout_multilevel(lb, options_of(p), seeds, p->match_rounds, p->coarse_min, p->multilevel != 0, xp, s, sc));
  return unpermute_coords(g, xp, x, s);
}

vmo_status order_grouped(const vmo_hg_s* h, const ComponentGroups& g, const float4* x, const vmo_params* p, int sbd,
                         OrderState& st, cudaStream_t s, Scratch& sc, const int32_t* mu) {
  OrderParams op;
  op.d = p->d;
  op.km_iters = p->km_iters;
  op.min_part = p->min_part;
  op.max_depth = p->max_depth;
  op.sbd = sbd;
  op.sep_rec = p->sep_recursion;
  op.cut_order = p->cut_order;
  op.mu_order_free = p->sep_order_free;
  st.adj_ptr = h->adj_ptr.ptr;
  st.adj = h->adj.ptr;
  st.mu = mu;
  std::vector<uint64_t> seeds(g.base.size() - 1, p->seed);
  VMO_TRY(order_setup(st, x, g.base, seeds, op, g.cperm, s, sc));
  VMO_TRY(order_levels(st, op, s, sc));
  if (op.cut_order > 0 && !op.sep_rec) VMO_TRY(cut_order_pass(st, op, s, sc));
  return VMO_OK;
}

}  // namespace vmo
