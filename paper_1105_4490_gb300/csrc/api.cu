// C-ABI entry points of the VMO library (declared in include/vmo.h).
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>

#include "components.cuh"
#include "layout.cuh"
#include "order.cuh"

namespace vmo {

static thread_local std::string g_last_error;
thread_local cudaStream_t g_devarray_stream = nullptr;
thread_local bool g_devarray_async = false;
thread_local bool g_pdl = false;

void set_error(const std::string& msg) { g_last_error = msg; }

vmo_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  set_error(buf);
  return VMO_ERR_CUDA;
}

vmo_status invalid(const std::string& msg) {
  set_error(msg);
  return VMO_ERR_INVALID;
}

vmo_status unsupported(const std::string& msg) {
  set_error(msg);
  return VMO_ERR_UNSUPPORTED;
}

// ------------------------------ instrumentation ----------------------------
std::atomic<uint64_t> g_launches{0};
// Device allocations made by the library (reported by vmo_stats_get).
std::atomic<uint64_t> g_device_allocs{0};
namespace {
std::mutex g_stats_mu;
bool g_time = false;
unsigned long long* g_icount = nullptr;  // device counter (counting mode)
struct TimedLaunch {
  cudaEvent_t a, b;
  uint64_t points;
};
std::vector<TimedLaunch> g_timed;
std::vector<cudaEvent_t> g_event_pool;
cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

bool stats_timing() { return g_time; }
unsigned long long* stats_interaction_counter() { return g_icount; }

void stats_time_begin(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_stats_mu);
  TimedLaunch t;
  t.a = take_event();
  t.b = take_event();
  t.points = 0;
  cudaEventRecord(t.a, s);
  g_timed.push_back(t);
}

void stats_time_end(cudaStream_t s, uint64_t points) {
  std::lock_guard<std::mutex> lk(g_stats_mu);
  if (g_timed.empty()) return;
  cudaEventRecord(g_timed.back().b, s);
  g_timed.back().points = points;
}

Scratch::~Scratch() { release_to(0); }

vmo_status Scratch::alloc_bytes(void** p, size_t bytes) {
  if (bytes < 16) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    (void)cudaGetLastError();
    set_error("device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    return VMO_ERR_OOM;
  }
  g_device_allocs.fetch_add(1, std::memory_order_relaxed);
  ptrs.push_back(*p);
  return VMO_OK;
}

void Scratch::release_to(size_t m) {
  while (ptrs.size() > m) {
    cudaFreeAsync(ptrs.back(), stream);
    ptrs.pop_back();
  }
}

vmo_status build_model(const vmo_csr* a, vmo_model model, vmo_hg_s* h, cudaStream_t s);
vmo_status components(const vmo_hg_s* h, int32_t* labels, cudaStream_t s);
vmo_status finegrain_coords(const vmo_hg_s* h, const float* xb, float* xf, cudaStream_t s);
vmo_status cut_size(const vmo_hg_s* h, const int32_t* part, int32_t nparts, int64_t* cutnet, int64_t* lambda1,
                    cudaStream_t s);

namespace {

std::once_flag g_pool_once;

// Device present; stream-ordered pool keeps freed scratch for reuse.
vmo_status ensure_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    (void)cudaGetLastError();
    set_error("no usable CUDA device (the library has no CPU fallback)");
    return VMO_ERR_CUDA;
  }
  std::call_once(g_pool_once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
  return VMO_OK;
}

vmo_status check_params(const vmo_params* p) {
  if (!p) return invalid("params is null");
  if (p->d < 2 || p->d > 4) return unsupported("layout dimension d must be 2, 3 or 4");
  if (p->iters < 0 || p->km_iters < 0 || p->min_part < 0 || p->occupancy < 1 || p->match_rounds < 0 ||
      p->coarse_min < 1)
    return invalid("negative or zero parameter");
  if (!(p->sigma > 0.0f) || !(p->decay > 0.0f) || p->decay > 1.0f) return invalid("sigma > 0 and 0 < decay <= 1");
  if (p->max_depth < 0 || p->max_depth > 62) return invalid("max_depth must be in [0, 62]");
  if (p->sep_recursion != 0 && p->sep_recursion != 1) return invalid("sep_recursion must be 0 or 1");
  if (p->cut_order < 0 || p->cut_order > 8) return invalid("cut_order must be in [0, 8]");
  if (p->sep_order_free != 0 && p->sep_order_free != 1) return invalid("sep_order_free must be 0 or 1");
  return VMO_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }


// Level-0 batch of one problem: the handle's model.
vmo_status single_batch(vmo_hg_s* h, int d, int occ, LevelBatch& lb, cudaStream_t s) {
  lb.K = h->k;
  lb.P = 1;
  lb.vbase = {0, (int64_t)h->k};
  lb.src = {0};
  if (h->model == VMO_SYMMETRIC || h->model == VMO_BIPARTITE) {
    lb.adj_ptr = h->adj_ptr.ptr;
    lb.adj = h->adj.ptr;
    lb.nadj = h->nadj;
  } else {
    lb.net_ptr = h->net_ptr.ptr;
    lb.pins = h->pins.ptr;
    lb.vtx_ptr = h->vtx_ptr.ptr;
    lb.vnets = h->vnets.ptr;
    lb.nnets = h->l;
  }
  lb.w = h->has_weight ? h->weight.ptr : nullptr;
  return level_setup(lb, d, occ, s);
}

// Geometry of a handle.  Graph models: every connected component is laid out
// as its own problem of one batch (Sec. 2.2), then the coordinates are put
// back in vertex order.  Hypergraph models and a given start: one problem.
vmo_status run_layout(vmo_hg_s* h, const vmo_params* p, float4* x, bool given, cudaStream_t s, Scratch& sc) {
  LayoutOptions o = options_of(p);
  const bool graph = h->model == VMO_SYMMETRIC || h->model == VMO_BIPARTITE;
  if (given || !graph) {
    LevelBatch lb;
    VMO_TRY(single_batch(h, p->d, p->occupancy, lb, s));
    if (given) return layout_level(lb, o, x, o.iters, -1.0f, nullptr, nullptr, s, sc);
    std::vector<uint64_t> seeds{p->seed};
    return layout_multilevel(lb, o, seeds, p->match_rounds, p->coarse_min, false, x, s, sc);
  }
  ComponentGroups g;
  VMO_TRY(group_components(h, g, s, sc));
  return layout_grouped(h, g, p, x, s, sc);
}

__global__ void k_split_rows(const int32_t* __restrict__ ord, int64_t n, int32_t m, const int32_t* __restrict__ rpos,
                             int32_t* __restrict__ row_perm, int32_t* __restrict__ col_perm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t v = ord[i];
  int32_t r = rpos[i];
  if (v < m) row_perm[r] = v;
  else col_perm[i - r] = v - m;
}

// Coarse vertex of every fine vertex: rank of its group's anchor.
__global__ void k_group_ids(const int32_t* __restrict__ anchor, const int32_t* __restrict__ rank, int64_t k,
                            int32_t* __restrict__ pi) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < k) pi[v] = rank[anchor[v]];
}

__global__ void k_is_row(const int32_t* __restrict__ ord, int64_t n, int32_t m, int32_t* __restrict__ flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = ord[i] < m ? 1 : 0;
}

// A strengthened diagonal: match[i] in [0, m), every column once, and the
// pattern holds (i, match[i]) (row vertex i is linked to column vertex m + match[i]).
__global__ void k_check_match(const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                              const int32_t* __restrict__ match, int32_t m, int32_t* __restrict__ seen,
                              int32_t* __restrict__ err) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int32_t c = match[i];
  if (c < 0 || c >= m) { atomicOr(err, 1); return; }
  if (atomicAdd(&seen[c], 1) != 0) atomicOr(err, 2);
  bool found = false;
  for (int32_t t = adj_ptr[i]; t < adj_ptr[i + 1] && !found; ++t) found = adj[t] == m + c;
  if (!found) atomicOr(err, 4);
}

__global__ void k_build_mu(const int32_t* __restrict__ match, int32_t m, int32_t* __restrict__ mu) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  mu[i] = m + match[i];
  mu[m + match[i]] = i;
}

__global__ void k_match_cols(const int32_t* __restrict__ row_perm, const int32_t* __restrict__ match, int32_t m,
                             int32_t* __restrict__ col_perm) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) col_perm[t] = match[row_perm[t]];
}

vmo_status run_order(vmo_hg_s* h, const float* coords, const vmo_params* p, int sbd, int32_t* vperm,
                     int32_t* row_perm, int32_t* col_perm, vmo_tree* tree, cudaStream_t s,
                     const int32_t* match = nullptr) {
  VMO_TRY(ensure_device());
  VMO_TRY(check_params(p));
  if (!h) return invalid("handle is null");
  if (h->model != VMO_SYMMETRIC && h->model != VMO_BIPARTITE)
    return unsupported("ordering needs a graph model (symmetric or bipartite, Algorithm 7)");
  if (coords && !aligned16(coords)) return invalid("coords must be 16-byte aligned");
  Scratch sc(s);
  const int64_t k = h->k;
  int32_t* mu = nullptr;
  if (match) {
    if (h->model != VMO_BIPARTITE || h->m != h->n)
      return invalid("a strengthened diagonal needs the bipartite model of a square pattern");
    const int32_t m = h->m;
    int32_t *seen, *err;
    VMO_TRY(sc.alloc(&mu, std::max<int64_t>(k, 1)));
    VMO_TRY(sc.alloc(&seen, std::max<int32_t>(m, 1)));
    VMO_TRY(sc.alloc(&err, 1));
    VMO_CUDA(cudaMemsetAsync(seen, 0, std::max<int32_t>(m, 1) * sizeof(int32_t), s));
    VMO_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    if (m > 0) {
      launch(k_check_match, grid_for(m, 256), 256, 0, s, h->adj_ptr.ptr, h->adj.ptr, match, m, seen, err);
      VMO_LAUNCHED("check_match");
    }
    int32_t herr = 0;
    VMO_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
    VMO_CUDA(cudaStreamSynchronize(s));
    if (herr & 1) return invalid("match: a column index outside [0, m)");
    if (herr & 2) return invalid("match: a column matched to two rows (not a permutation)");
    if (herr & 4) return invalid("match: a row not linked to its matched column (not an entry of the pattern)");
    if (m > 0) {
      launch(k_build_mu, grid_for(m, 256), 256, 0, s, match, m, mu);
      VMO_LAUNCHED("build_mu");
    }
  }
  ComponentGroups g;
  VMO_TRY(group_components(h, g, s, sc));
  float4* x = (float4*)coords;
  if (!x) {
    VMO_TRY(sc.alloc(&x, std::max<int64_t>(k, 1)));
    VMO_TRY(layout_grouped(h, g, p, x, s, sc));
  }
  OrderState st;
  VMO_TRY(order_grouped(h, g, x, p, sbd, st, s, sc, mu));
  if (vperm) VMO_CUDA(cudaMemcpyAsync(vperm, st.ord, k * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (row_perm || col_perm) {
    if (h->model == VMO_SYMMETRIC) {
      if (row_perm) VMO_CUDA(cudaMemcpyAsync(row_perm, st.ord, k * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      if (col_perm) VMO_CUDA(cudaMemcpyAsync(col_perm, st.ord, k * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    } else {
      if (!row_perm || !col_perm) return invalid("bipartite ordering needs both row_perm and col_perm");
      int32_t* flag;
      VMO_TRY(sc.alloc(&flag, std::max<int64_t>(k, 1)));
      if (k > 0) {
        launch(k_is_row, grid_for(k, 256), 256, 0, s, st.ord, k, h->m, flag);
        VMO_LAUNCHED("is_row");
      }
      VMO_TRY(scan_exclusive<int32_t>(flag, flag, k, nullptr, s, sc));
      if (k > 0) {
        launch(k_split_rows, grid_for(k, 256), 256, 0, s, st.ord, k, h->m, flag, row_perm, col_perm);
        VMO_LAUNCHED("split_rows");
      }
      if (match && h->m > 0) {  // every column at its matched row's position
        launch(k_match_cols, grid_for(h->m, 256), 256, 0, s, row_perm, match, h->m, col_perm);
        VMO_LAUNCHED("match_cols");
      }
    }
  }
  if (tree) {
    int32_t cnt = 0;
    uint32_t* idx;
    VMO_TRY(tree_sorted(st, true, &cnt, &idx, s, sc));
    tree->count = cnt;
    if (cnt > tree->capacity) {
      VMO_CUDA(cudaStreamSynchronize(s));
      return invalid("tree capacity " + std::to_string(tree->capacity) + " < " + std::to_string(cnt) + " records");
    }
    VMO_TRY(tree_write(st, idx, cnt, tree->heap, tree->offset, tree->n1, tree->n2, tree->nsep, tree->depth,
                       tree->component, s));
  }
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

// The coarsening hierarchy of the handle's graph as one problem (the one that
// vmo_coarsen counts) and a check that `level` is one of its levels.
vmo_status hierarchy_of(vmo_hg_s* h, const vmo_params* p, int32_t level, LevelBatch& lb, Hierarchy& H, cudaStream_t s,
                        Scratch& sc) {
  VMO_TRY(ensure_device());
  VMO_TRY(check_params(p));
  if (!h) return invalid("handle is null");
  if (h->model != VMO_SYMMETRIC && h->model != VMO_BIPARTITE) return unsupported("the hierarchy needs a graph model");
  VMO_TRY(single_batch(h, p->d, p->occupancy, lb, s));
  std::vector<uint64_t> seeds{p->seed};
  VMO_TRY(build_hierarchy(lb, options_of(p), seeds, p->match_rounds, p->coarse_min, p->multilevel != 0, H, s, sc));
  if (level < 0 || level >= (int32_t)H.levels.size())
    return invalid("level " + std::to_string(level) + " outside the hierarchy's " + std::to_string(H.levels.size()) +
                   " levels");
  return VMO_OK;
}

__global__ void k_fill_f32(float* __restrict__ a, int64_t n, float v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

}  // namespace

vmo_status ensure_device_public() { return ensure_device(); }
vmo_status check_params_public(const vmo_params* p) { return check_params(p); }

}  // namespace vmo

using namespace vmo;

extern "C" {

void vmo_default_params(vmo_params* p) {
  if (!p) return;
  p->d = 3;
  p->iters = 100;
  p->sigma = 1.0f;
  p->decay = 0.9f;
  p->occupancy = 8;
  p->multilevel = 1;
  p->match_rounds = 4;
  p->coarse_min = 64;
  p->km_iters = 20;
  p->min_part = 64;
  p->max_depth = 62;
  p->sep_recursion = 0;
  p->cut_order = 0;
  p->sep_order_free = 0;
  p->seed = 1;
}

vmo_status vmo_build_hypergraph(const vmo_csr* a, vmo_model model, const float* vertex_weight, void* stream,
                                vmo_hg* out) {
  if (!out) return invalid("out is null");
  *out = nullptr;
  VMO_TRY(ensure_device());
  if (model < VMO_SYMMETRIC || model > VMO_FINEGRAIN) return invalid("unknown model");
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<vmo_hg_s> h(new vmo_hg_s());
  cudaGetDevice(&h->device);
  VMO_TRY(build_model(a, model, h.get(), s));
  if (vertex_weight) {
    VMO_TRY(h->weight.resize(std::max<int32_t>(h->k, 1)));
    VMO_CUDA(cudaMemcpyAsync(h->weight.ptr, vertex_weight, h->k * sizeof(float), cudaMemcpyDeviceToDevice, s));
    VMO_CUDA(cudaStreamSynchronize(s));
    h->has_weight = true;
  }
  *out = h.release();
  return VMO_OK;
}

int32_t vmo_hg_vertices(vmo_hg hg) { return hg ? hg->k : 0; }
int64_t vmo_hg_nets(vmo_hg hg) { return hg ? hg->l : 0; }

vmo_status vmo_hg_arrays(vmo_hg hg, const int32_t** adj_ptr, const int32_t** adj, int64_t* count_adj,
                         const int32_t** net_ptr, const int32_t** pins, int64_t* count_pins,
                         const int32_t** vtx_ptr, const int32_t** vnets, int64_t* count_vnets) {
  if (!hg) return invalid("handle is null");
  bool graph = hg->model == VMO_SYMMETRIC || hg->model == VMO_BIPARTITE;
  if (adj_ptr) *adj_ptr = graph ? hg->adj_ptr.ptr : nullptr;
  if (adj) *adj = graph ? hg->adj.ptr : nullptr;
  if (count_adj) *count_adj = graph ? hg->nadj : 0;
  if (net_ptr) *net_ptr = hg->net_ptr.ptr;
  if (pins) *pins = hg->pins.ptr;
  if (count_pins) *count_pins = hg->npins;
  if (vtx_ptr) *vtx_ptr = hg->vtx_ptr.ptr;
  if (vnets) *vnets = hg->vnets.ptr;
  if (count_vnets) *count_vnets = hg->nvnets;
  return VMO_OK;
}

vmo_status vmo_components(vmo_hg hg, int32_t* labels, void* stream) {
  VMO_TRY(ensure_device());
  if (!hg || (!labels && hg->k > 0)) return invalid("null argument");
  return components(hg, labels, (cudaStream_t)stream);
}

vmo_status vmo_init_coords(int32_t k, int32_t d, uint64_t seed, float* coords, void* stream) {
  VMO_TRY(ensure_device());
  if (k < 0) return invalid("k < 0");
  if (d < 2 || d > 4) return unsupported("d must be 2, 3 or 4");
  if (k > 0 && (!coords || !aligned16(coords))) return invalid("coords null or not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  LevelBatch lb;
  lb.K = k;
  lb.P = 1;
  lb.vbase = {0, (int64_t)k};
  lb.src = {0};
  VMO_TRY(level_setup(lb, d, 8, s));
  Scratch sc(s);
  uint64_t* sd;
  VMO_TRY(sc.alloc(&sd, 1));
  VMO_CUDA(cudaMemcpyAsync(sd, &seed, 8, cudaMemcpyHostToDevice, s));
  VMO_TRY(init_coords_level(lb, d, sd, (float4*)coords, nullptr, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status vmo_layout(vmo_hg hg, const vmo_params* params, float* coords, int32_t use_given_init, void* stream) {
  VMO_TRY(ensure_device());
  VMO_TRY(check_params(params));
  if (!hg) return invalid("handle is null");
  if (hg->k > 0 && (!coords || !aligned16(coords))) return invalid("coords null or not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  VMO_TRY(run_layout(hg, params, (float4*)coords, use_given_init != 0, s, sc));
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status vmo_layout_step(vmo_hg hg, const vmo_params* params, float* coords, float step, float* y_out,
                           uint32_t* keys_out, int32_t* levels_out, void* stream) {
  VMO_TRY(ensure_device());
  VMO_TRY(check_params(params));
  if (!hg) return invalid("handle is null");
  if (!(step > 0.0f)) return invalid("step must be > 0");
  if (hg->k > 0 && (!coords || !aligned16(coords))) return invalid("coords null or not 16-byte aligned");
  if (y_out && !aligned16(y_out)) return invalid("y_out must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  LevelBatch lb;
  VMO_TRY(single_batch(hg, params->d, params->occupancy, lb, s));
  if (levels_out) *levels_out = lb.L.empty() ? 1 : lb.L[0];
  LayoutOptions o = options_of(params);
  VMO_TRY(layout_level(lb, o, (float4*)coords, 1, step, (float4*)y_out, keys_out, s, sc));
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status vmo_coarsen(vmo_hg hg, const vmo_params* params, int32_t* mate, int32_t* pi, int32_t* kc_out,
                       int32_t* level_sizes, int32_t* nlevels, void* stream) {
  VMO_TRY(ensure_device());
  VMO_TRY(check_params(params));
  if (!hg) return invalid("handle is null");
  if (hg->model != VMO_SYMMETRIC && hg->model != VMO_BIPARTITE) return unsupported("coarsening needs a graph model");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  LevelBatch lb;
  VMO_TRY(single_batch(hg, params->d, params->occupancy, lb, s));
  const int64_t k = hg->k;
  if (mate || pi || kc_out) {
    int32_t *m, *anchor, *rank, *act;
    uint64_t* sd;
    VMO_TRY(sc.alloc(&m, std::max<int64_t>(k, 1)));
    VMO_TRY(sc.alloc(&anchor, std::max<int64_t>(k, 1)));
    VMO_TRY(sc.alloc(&rank, std::max<int64_t>(k, 1)));
    VMO_TRY(sc.alloc(&act, 1));
    VMO_TRY(sc.alloc(&sd, 1));
    int32_t one = 1;
    uint64_t seed = params->seed;
    VMO_CUDA(cudaMemcpyAsync(act, &one, 4, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaMemcpyAsync(sd, &seed, 8, cudaMemcpyHostToDevice, s));
    std::vector<int64_t> kc;
    if (k > 0) {
      VMO_TRY(coarsen_level(lb, sd, 0, params->match_rounds, act, m, anchor, rank, kc, s, sc));
      if (kc_out) *kc_out = (int32_t)kc[0];
      if (mate) VMO_CUDA(cudaMemcpyAsync(mate, m, k * 4, cudaMemcpyDeviceToDevice, s));
      if (pi) {
        launch(k_group_ids, grid_for(k, 256), 256, 0, s, anchor, rank, k, pi);
        VMO_LAUNCHED("group_ids");
      }
    } else if (kc_out) {
      *kc_out = 0;
    }
  }
  if (level_sizes || nlevels) {
    Hierarchy H;
    std::vector<uint64_t> seeds{params->seed};
    VMO_TRY(build_hierarchy(lb, options_of(params), seeds, params->match_rounds, params->coarse_min,
                            params->multilevel != 0, H, s, sc));
    int nl = (int)H.levels.size();
    if (nlevels) *nlevels = nl;
    if (level_sizes)
      for (int j = 0; j < nl && j < 41; ++j) level_sizes[j] = (int32_t)H.levels[j]->K;
  }
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status vmo_hierarchy_level(vmo_hg hg, const vmo_params* params, int32_t level, int32_t* k_out, int64_t* nadj_out,
                               int32_t* adj_ptr, int32_t* adj, float* acost, float* weight, int32_t* pi,
                               void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  LevelBatch lb;
  Hierarchy H;
  VMO_TRY(hierarchy_of(hg, params, level, lb, H, s, sc));
  const LevelBatch& L = *H.levels[level];
  const int64_t k = L.K, na = L.nadj;
  if (k_out) *k_out = (int32_t)k;
  if (nadj_out) *nadj_out = na;
  if (adj_ptr) VMO_CUDA(cudaMemcpyAsync(adj_ptr, L.adj_ptr, (k + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (adj && na > 0) VMO_CUDA(cudaMemcpyAsync(adj, L.adj, na * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (acost && na > 0) {
    if (L.acost) VMO_CUDA(cudaMemcpyAsync(acost, L.acost, na * sizeof(float), cudaMemcpyDeviceToDevice, s));
    else launch(k_fill_f32, grid_for(na, 256), 256, 0, s, acost, na, 1.0f);
  }
  if (weight && k > 0) {
    if (L.w) VMO_CUDA(cudaMemcpyAsync(weight, L.w, k * sizeof(float), cudaMemcpyDeviceToDevice, s));
    else launch(k_fill_f32, grid_for(k, 256), 256, 0, s, weight, k, 1.0f);
  }
  if (pi && level > 0 && H.levels[level - 1]->K > 0)
    VMO_CUDA(cudaMemcpyAsync(pi, H.pis[level - 1], H.levels[level - 1]->K * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                             s));
  VMO_LAUNCHED("hierarchy_level");
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status vmo_hierarchy_prolong(vmo_hg hg, const vmo_params* params, int32_t level, const float* coarse, float* fine,
                                 void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  LevelBatch lb;
  Hierarchy H;
  VMO_TRY(hierarchy_of(hg, params, level, lb, H, s, sc));
  if (level < 1) return invalid("prolongation needs a level >= 1");
  if ((H.levels[level]->K > 0 && (!coarse || !aligned16(coarse))) ||
      (H.levels[level - 1]->K > 0 && (!fine || !aligned16(fine))))
    return invalid("coarse and fine coordinates must be non-null and 16-byte aligned");
  VMO_TRY(prolong_level(H, level - 1, params->d, (const float4*)coarse, (float4*)fine, s, sc));
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status vmo_hierarchy_step(vmo_hg hg, const vmo_params* params, int32_t level, float* coords, float step,
                              float* y_out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  LevelBatch lb;
  Hierarchy H;
  VMO_TRY(hierarchy_of(hg, params, level, lb, H, s, sc));
  if (!(step > 0.0f)) return invalid("step must be > 0");
  LevelBatch& L = *H.levels[level];
  if (L.K > 0 && (!coords || !aligned16(coords))) return invalid("coords null or not 16-byte aligned");
  if (y_out && !aligned16(y_out)) return invalid("y_out must be 16-byte aligned");
  VMO_TRY(layout_level(L, options_of(params), (float4*)coords, 1, step, (float4*)y_out, nullptr, s, sc));
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status vmo_bisect(vmo_hg hg, int32_t d, const float* coords, const int32_t* verts, int32_t nverts, uint64_t seed,
                      uint64_t key, int32_t km_iters, uint8_t* labels, float* z, int32_t* split, void* stream) {
  VMO_TRY(ensure_device());
  if (!hg) return invalid("handle is null");
  if (d < 2 || d > 4) return unsupported("d must be 2, 3 or 4");
  if (nverts < 0 || km_iters < 0) return invalid("negative size");
  if (nverts > 0 && (!coords || !verts || !labels || !aligned16(coords))) return invalid("null or unaligned argument");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  float zh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int32_t sp = 0;
  if (nverts >= 2) {
    OrderState st;
    st.n = nverts;
    VMO_TRY(sc.alloc(&st.ord, nverts));
    VMO_TRY(sc.alloc(&st.xo, nverts));
    VMO_TRY(sc.alloc(&st.seg, nverts));
    VMO_TRY(sc.alloc(&st.lab, nverts));
    VMO_TRY(sc.alloc(&st.seeds, 1));
    VMO_TRY(sc.alloc(&st.nodes, 1));
    VMO_CUDA(cudaMemcpyAsync(st.ord, verts, nverts * 4, cudaMemcpyDeviceToDevice, s));
    VMO_CUDA(cudaMemsetAsync(st.seg, 0, nverts * 4, s));
    VMO_CUDA(cudaMemcpyAsync(st.seeds, &seed, 8, cudaMemcpyHostToDevice, s));
    NodeDev nd;
    memset(&nd, 0, sizeof(nd));
    nd.heap = key;
    nd.off = 0;
    nd.size = nverts;
    VMO_CUDA(cudaMemcpyAsync(st.nodes, &nd, sizeof(nd), cudaMemcpyHostToDevice, s));
    VMO_TRY(gather_coords((const float4*)coords, st.ord, nverts, st.xo, s));
    VMO_TRY(two_means(st, 1, d, km_iters, s, sc));
    VMO_CUDA(cudaMemcpyAsync(&nd, st.nodes, sizeof(nd), cudaMemcpyDeviceToHost, s));
    VMO_CUDA(cudaStreamSynchronize(s));
    if (nd.state == 2) {
      VMO_CUDA(cudaMemsetAsync(labels, 1, nverts, s));
      zh[0] = nd.z1.x; zh[1] = nd.z1.y; zh[2] = nd.z1.z; zh[3] = nd.z1.w;
    } else {
      VMO_CUDA(cudaMemcpyAsync(labels, st.lab, nverts, cudaMemcpyDeviceToDevice, s));
      zh[0] = nd.z1.x; zh[1] = nd.z1.y; zh[2] = nd.z1.z; zh[3] = nd.z1.w;
      zh[4] = nd.z2.x; zh[5] = nd.z2.y; zh[6] = nd.z2.z; zh[7] = nd.z2.w;
      sp = (nd.n1 > 0 && nd.n2 > 0) ? 1 : 0;
    }
  } else if (nverts == 1) {
    VMO_CUDA(cudaMemsetAsync(labels, 1, 1, s));
  }
  if (z) VMO_CUDA(cudaMemcpyAsync(z, zh, sizeof(zh), cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  if (split) *split = sp;
  return VMO_OK;
}

vmo_status vmo_order_bbd(vmo_hg hg, const float* coords, const vmo_params* params, int32_t* row_perm,
                         int32_t* col_perm, vmo_tree* tree, void* stream) {
  return run_order(hg, coords, params, 0, nullptr, row_perm, col_perm, tree, (cudaStream_t)stream);
}

vmo_status vmo_order_sbd(vmo_hg hg, const float* coords, const vmo_params* params, int32_t* row_perm,
                         int32_t* col_perm, vmo_tree* tree, void* stream) {
  return run_order(hg, coords, params, 1, nullptr, row_perm, col_perm, tree, (cudaStream_t)stream);
}

vmo_status vmo_order_vertices(vmo_hg hg, const float* coords, const vmo_params* params, int32_t sbd, int32_t* perm,
                              vmo_tree* tree, void* stream) {
  if (!perm && hg && hg->k > 0) return invalid("perm is null");
  return run_order(hg, coords, params, sbd ? 1 : 0, perm, nullptr, nullptr, tree, (cudaStream_t)stream);
}

vmo_status vmo_order_matched(vmo_hg hg, const float* coords, const vmo_params* params, int32_t sbd,
                             const int32_t* match, int32_t* row_perm, int32_t* col_perm, int32_t* vperm,
                             vmo_tree* tree, void* stream) {
  if (!match) return invalid("match is null");
  if (!row_perm || !col_perm) return invalid("row_perm and col_perm are required");
  return run_order(hg, coords, params, sbd ? 1 : 0, vperm, row_perm, col_perm, tree, (cudaStream_t)stream, match);
}

vmo_status vmo_finegrain_coords(vmo_hg hg, const float* bipartite_coords, float* coords, void* stream) {
  VMO_TRY(ensure_device());
  if (!hg) return invalid("handle is null");
  if (hg->model != VMO_FINEGRAIN) return invalid("finegrain coordinates need a finegrain handle");
  if (hg->k > 0 && (!bipartite_coords || !coords)) return invalid("coordinates are null");
  if (!aligned16(bipartite_coords) || !aligned16(coords)) return invalid("coordinates must be 16-byte aligned");
  return finegrain_coords(hg, bipartite_coords, coords, (cudaStream_t)stream);
}

vmo_status vmo_cut_size(vmo_hg hg, const int32_t* part, int32_t nparts, int64_t* cutnet, int64_t* lambda1,
                        void* stream) {
  VMO_TRY(ensure_device());
  if (!hg) return invalid("handle is null");
  return cut_size(hg, part, nparts, cutnet, lambda1, (cudaStream_t)stream);
}

void vmo_stats_reset(int32_t time_step_kernel, int32_t count_interactions) {
  std::lock_guard<std::mutex> lk(g_stats_mu);
  g_launches.store(0);
  for (auto& t : g_timed) {
    g_event_pool.push_back(t.a);
    g_event_pool.push_back(t.b);
  }
  g_timed.clear();
  g_time = time_step_kernel != 0;
  if (count_interactions) {
    if (!g_icount && cudaMalloc((void**)&g_icount, sizeof(unsigned long long)) != cudaSuccess) {
      g_icount = nullptr;
      (void)cudaGetLastError();
    }
    if (g_icount) cudaMemset(g_icount, 0, sizeof(unsigned long long));
  } else if (g_icount) {
    cudaFree(g_icount);
    g_icount = nullptr;
  }
}

vmo_status vmo_stats_get(vmo_stats* out) {
  if (!out) return invalid("out is null");
  std::lock_guard<std::mutex> lk(g_stats_mu);
  memset(out, 0, sizeof(*out));
  out->launches = g_launches.load();
  out->device_allocations = g_device_allocs.load();
  if (!g_timed.empty() || g_icount) VMO_CUDA(cudaDeviceSynchronize());
  for (auto& t : g_timed) {
    float ms = 0.f;
    VMO_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
    out->step_ms += ms;
    out->step_points += t.points;
    out->step_launches += 1;
  }
  if (g_icount) {
    unsigned long long c = 0;
    VMO_CUDA(cudaMemcpy(&c, g_icount, sizeof(c), cudaMemcpyDeviceToHost));
    out->step_interactions = c;
  }
  return VMO_OK;
}

void vmo_destroy(vmo_hg hg) { delete hg; }

const char* vmo_status_string(vmo_status s) {
  switch (s) {
    case VMO_OK: return "ok";
    case VMO_ERR_INVALID: return "invalid argument";
    case VMO_ERR_OOM: return "out of device memory";
    case VMO_ERR_CUDA: return "CUDA error";
    case VMO_ERR_TIMEOUT: return "device wait timed out";
    case VMO_ERR_BUDGET: return "over admission budget";
    case VMO_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* vmo_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
