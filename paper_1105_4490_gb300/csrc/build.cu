// Hypergraph models of a sparse pattern (Table 1, Sec. 1.1), connected
// components (Algorithm 1) and cut metrics (Sec. 4.1 footnote, Sec. 5).
//
// Every model is built the same way on the device: each nonzero emits 64-bit
// pair keys (row * ncols + col), a radix sort orders them, a flag/scan pass
// drops duplicates and the surviving keys become CSR rows whose pointers come
// from per-row counts and a scan.  Graph models emit both orientations of
// {u, v} so the result is the symmetric adjacency with ascending neighbours.
#include <algorithm>

#include "vmo_internal.cuh"

namespace vmo {

namespace {

__device__ inline int32_t row_of(const int32_t* __restrict__ rowptr, int32_t m, int64_t t) {
  int32_t lo = 0, hi = m;  // rowptr[lo] <= t < rowptr[hi]
  while (hi - lo > 1) {
    int32_t mid = (lo + hi) >> 1;
    if (rowptr[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void validate_csr_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int32_t m,
                                    int32_t n, int64_t nnz, int32_t* __restrict__ bad) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) {
    if (rowptr[t + 1] < rowptr[t]) atomicOr(bad, 1);
  }
  if (t == 0 && (rowptr[0] != 0 || (int64_t)rowptr[m] != nnz)) atomicOr(bad, 2);
  if (t < nnz) {
    int32_t c = colidx[t];
    if (c < 0 || c >= n) atomicOr(bad, 4);
  }
}

// Pair keys of the graph models: both orientations of every off-diagonal
// pattern entry (symmetric: {i, j}; bipartite: {r_i, c_j} = {i, m + j}).
__global__ void graph_keys_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int32_t m,
                                  int64_t nnz, int bipartite, uint64_t K, uint64_t sentinel,
                                  uint64_t* __restrict__ keys) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  uint64_t u = (uint64_t)row_of(rowptr, m, t);
  uint64_t v = bipartite ? (uint64_t)m + (uint64_t)colidx[t] : (uint64_t)colidx[t];
  if (u == v) {
    keys[2 * t] = sentinel;
    keys[2 * t + 1] = sentinel;
  } else {
    keys[2 * t] = u * K + v;
    keys[2 * t + 1] = v * K + u;
  }
}

// Pair keys (row, col) or transposed (col, row) of the pattern itself.
__global__ void pattern_keys_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int32_t m,
                                    int32_t n, int64_t nnz, int transpose, uint64_t* __restrict__ keys) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  uint64_t i = (uint64_t)row_of(rowptr, m, t), j = (uint64_t)colidx[t];
  keys[t] = transpose ? j * (uint64_t)m + i : i * (uint64_t)n + j;
}

__global__ void unique_flags_kernel(const uint64_t* __restrict__ keys, int64_t n, uint64_t sentinel,
                                    int32_t* __restrict__ flag) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  uint64_t k = keys[t];
  flag[t] = (k != sentinel && (t == 0 || keys[t - 1] != k)) ? 1 : 0;
}

__global__ void emit_csr_kernel(const uint64_t* __restrict__ keys, int64_t n, const int32_t* __restrict__ flag,
                                const int32_t* __restrict__ pos, uint64_t ncols, int32_t* __restrict__ idx,
                                int32_t* __restrict__ rowcount) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n || !flag[t]) return;
  uint64_t k = keys[t];
  idx[pos[t]] = (int32_t)(k % ncols);
  atomicAdd(&rowcount[k / ncols], 1);
}

__global__ void set_last_kernel(int32_t* ptr, int64_t n, const int32_t* total) { ptr[n] = *total; }

// Edge list (nets) of a graph model: the adjacency entries u -> v with u < v,
// in adjacency order (lexicographic).  pins[2e], pins[2e+1] = u, v.
__global__ void forward_flags_kernel(const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj, int32_t k,
                                     int64_t nadj, int32_t* __restrict__ flag) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nadj) return;
  int32_t u = row_of(adj_ptr, k, t);
  flag[t] = adj[t] > u ? 1 : 0;
}

__global__ void emit_edges_kernel(const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj, int32_t k,
                                  int64_t nadj, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                  int32_t* __restrict__ net_ptr, int32_t* __restrict__ pins,
                                  int32_t* __restrict__ vnets) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nadj || !flag[t]) return;
  int32_t u = row_of(adj_ptr, k, t), v = adj[t];
  int32_t e = pos[t];
  net_ptr[e] = 2 * e;
  pins[2 * e] = u;
  pins[2 * e + 1] = v;
  vnets[t] = e;
  // position of u in the (ascending) adjacency of v
  int32_t lo = adj_ptr[v], hi = adj_ptr[v + 1];
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    if (adj[mid] < u) lo = mid + 1; else hi = mid;
  }
  vnets[lo] = e;
}

__global__ void net_ptr_last_kernel(int32_t* net_ptr, const int32_t* nedges) { net_ptr[*nedges] = 2 * *nedges; }

// ----------------------------- components ----------------------------------
__device__ inline int32_t cc_find(const int32_t* p, int32_t v) {
  for (;;) {
    int32_t q = __ldcg(p + v);
    if (q == v) return v;
    v = q;
  }
}

__global__ void cc_init_kernel(int32_t* p, int32_t k) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < k) p[v] = v;
}

// Marks the last pin of every net (the pins that start no consecutive pair).
__global__ void cc_last_kernel(const int32_t* __restrict__ net_ptr, int64_t l, uint8_t* __restrict__ last) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= l) return;
  const int32_t b = net_ptr[e + 1];
  if (b > net_ptr[e]) last[b - 1] = 1;
}

// Hooks the roots of consecutive pins of every net to the smaller root.
__global__ void cc_hook_kernel(const int32_t* __restrict__ pins, const uint8_t* __restrict__ last, int64_t npins,
                               int32_t* p, int32_t* changed) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t + 1 >= npins || last[t]) return;  // the last pin of a net pairs with no next pin
  int32_t a = cc_find(p, pins[t]), b = cc_find(p, pins[t + 1]);
  if (a == b) return;
  int32_t hi_ = a > b ? a : b, lo_ = a > b ? b : a;
  atomicMin(p + hi_, lo_);
  *changed = 1;
}

__global__ void cc_compress_kernel(int32_t* p, int32_t k) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < k) p[v] = cc_find(p, v);
}

// ------------------------------- cut size ----------------------------------
// One warp per net.  nparts <= 64: union of part bitmasks; otherwise a pin is
// counted when no earlier pin of the net has its part.
__global__ void cut_kernel(const int32_t* __restrict__ net_ptr, const int32_t* __restrict__ pins, int64_t l,
                           const int32_t* __restrict__ part, int32_t nparts, unsigned long long* __restrict__ out) {
  int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = lane_id();
  if (e >= l) return;
  int32_t a = net_ptr[e], b = net_ptr[e + 1];
  uint32_t lam;
  if (nparts <= 64) {
    uint64_t mask = 0;
    for (int32_t t = a + lane; t < b; t += 32) mask |= 1ull << part[pins[t]];
    uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)mask);
    uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(mask >> 32));
    lam = __popc(lo) + __popc(hi);
  } else {
    uint32_t cnt = 0;
    for (int32_t t = a + lane; t < b; t += 32) {
      int32_t pt = part[pins[t]];
      bool first = true;
      for (int32_t u = a; u < t; ++u)
        if (part[pins[u]] == pt) { first = false; break; }
      cnt += first ? 1u : 0u;
    }
    lam = __reduce_add_sync(0xffffffffu, cnt);
  }
  if (lane == 0 && lam > 1) {
    atomicAdd(out, 1ull);
    atomicAdd(out + 1, (unsigned long long)(lam - 1));
  }
}

}  // namespace

// Checks one CSR on the device; the error bits are or-ed into *bad.
vmo_status validate_csr_async(const vmo_csr* a, int32_t* bad, cudaStream_t s) {
  if (!a || a->m < 0 || a->n < 0 || a->nnz < 0) return invalid("csr: negative size or null");
  if (!a->rowptr || (a->nnz > 0 && !a->colidx)) return invalid("csr: null pointer");
  if (a->nnz > INT32_MAX) return unsupported("csr: more than 2^31-1 nonzeros");
  int64_t n = std::max<int64_t>(a->m, a->nnz);
  launch(validate_csr_kernel, grid_for(n + 1, 256), 256, 0, s, a->rowptr, a->colidx, a->m, a->n, a->nnz, bad);
  VMO_LAUNCHED("validate_csr");
  return VMO_OK;
}

vmo_status validate_csr(const vmo_csr* a, cudaStream_t s, Scratch& sc) {
  if (!a || a->m < 0 || a->n < 0 || a->nnz < 0) return invalid("csr: negative size or null");
  if (!a->rowptr || (a->nnz > 0 && !a->colidx)) return invalid("csr: null pointer");
  if (a->nnz > INT32_MAX) return unsupported("csr: more than 2^31-1 nonzeros");
  int32_t* bad;
  VMO_TRY(sc.alloc(&bad, 1));
  VMO_CUDA(cudaMemsetAsync(bad, 0, 4, s));
  int64_t n = std::max<int64_t>(a->m, a->nnz);
  launch(validate_csr_kernel, grid_for(n + 1, 256), 256, 0, s, a->rowptr, a->colidx, a->m, a->n, a->nnz, bad);
  VMO_LAUNCHED("validate_csr");
  int32_t h = 0;
  VMO_CUDA(cudaMemcpyAsync(&h, bad, 4, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  if (h & 2) return invalid("csr: rowptr[0] != 0 or rowptr[m] != nnz");
  if (h & 1) return invalid("csr: rowptr not monotone");
  if (h & 4) return invalid("csr: column index out of range");
  return VMO_OK;
}

// Sorted-unique CSR of `nrows` rows from pair keys row*ncols+col (keys with
// value >= nrows*ncols are dropped).  Allocates ptr (nrows+1) and idx.
static vmo_status csr_from_keys(uint64_t* keys, int64_t nkeys, int64_t nrows, int64_t ncols, DevArray<int32_t>& ptr,
                                DevArray<int32_t>& idx, int64_t* nout, cudaStream_t s, Scratch& sc) {
  uint64_t sentinel = (uint64_t)nrows * (uint64_t)ncols;
  int bits = bits_for(sentinel);
  uint64_t* sorted;
  int32_t *flag, *pos, *total;
  VMO_TRY(sc.alloc(&sorted, (size_t)std::max<int64_t>(nkeys, 1)));
  VMO_TRY(sc.alloc(&flag, (size_t)std::max<int64_t>(nkeys, 1)));
  VMO_TRY(sc.alloc(&pos, (size_t)std::max<int64_t>(nkeys, 1)));
  VMO_TRY(sc.alloc(&total, 1));
  VMO_TRY(radix_sort_u64(keys, nullptr, sorted, nullptr, nkeys, bits, s, sc));
  if (nkeys > 0) {
    launch(unique_flags_kernel, grid_for(nkeys, 256), 256, 0, s, sorted, nkeys, sentinel, flag);
    VMO_LAUNCHED("unique_flags");
  }
  VMO_TRY(scan_exclusive<int32_t>(flag, pos, nkeys, total, s, sc));
  int32_t h_total = 0;
  VMO_CUDA(cudaMemcpyAsync(&h_total, total, 4, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  VMO_TRY(ptr.resize((size_t)nrows + 1));
  VMO_TRY(idx.resize((size_t)std::max<int32_t>(h_total, 1)));
  VMO_CUDA(cudaMemsetAsync(ptr.ptr, 0, (nrows + 1) * sizeof(int32_t), s));
  if (nkeys > 0) {
    launch(emit_csr_kernel, grid_for(nkeys, 256), 256, 0, s, sorted, nkeys, flag, pos, (uint64_t)ncols, idx.ptr, ptr.ptr);
    VMO_LAUNCHED("emit_csr");
  }
  VMO_TRY(scan_exclusive<int32_t>(ptr.ptr, ptr.ptr, nrows, total, s, sc));
  launch(set_last_kernel, 1, 1, 0, s, ptr.ptr, nrows, total);
  VMO_LAUNCHED("set_last");
  *nout = h_total;
  return VMO_OK;
}

// Finegrain incidence: vertex t (the t-th distinct entry, in row i) lies on
// row net i and column net m + col(t).
__global__ void fg_vnets_kernel(const int32_t* __restrict__ rptr, const int32_t* __restrict__ cidx, int32_t m,
                                int32_t* __restrict__ vtx_ptr, int32_t* __restrict__ vnets) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int32_t t = rptr[i]; t < rptr[i + 1]; ++t) {
    vtx_ptr[t] = 2 * t;
    vnets[2 * t] = i;
    vnets[2 * t + 1] = m + cidx[t];
  }
  if (i == m - 1) vtx_ptr[rptr[m]] = 2 * rptr[m];
}

// Column keys col * u + t of the u distinct entries (row-major vertex ids).
__global__ void fg_col_keys_kernel(const int32_t* __restrict__ cidx, int64_t u, uint64_t* __restrict__ keys) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < u) keys[t] = (uint64_t)cidx[t] * (uint64_t)u + (uint64_t)t;
}

// Nets of the finegrain model: the row nets (vertex ranges of the row CSR)
// followed by the column nets.
__global__ void fg_nets_kernel(const int32_t* __restrict__ rptr, int32_t m, const int32_t* __restrict__ cptr,
                               const int32_t* __restrict__ cpins, int32_t n, int64_t u, int32_t* __restrict__ net_ptr,
                               int32_t* __restrict__ pins) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= m) net_ptr[t] = rptr[t];
  if (t < n) net_ptr[m + 1 + t] = (int32_t)u + cptr[t + 1];
  if (t < u) {
    pins[t] = (int32_t)t;
    pins[u + t] = cpins[t];
  }
}

vmo_status build_model(const vmo_csr* a, vmo_model model, vmo_hg_s* h, cudaStream_t s) {
  Scratch sc(s);
  VMO_TRY(validate_csr(a, s, sc));
  const int32_t m = a->m, n = a->n;
  const int64_t nnz = a->nnz;
  h->model = model;
  h->m = m;
  h->n = n;
  if (model == VMO_SYMMETRIC || model == VMO_BIPARTITE) {
    if (model == VMO_SYMMETRIC && m != n) return invalid("symmetric model needs a square pattern");
    int64_t K = (model == VMO_SYMMETRIC) ? m : (int64_t)m + n;
    if (K > INT32_MAX / 2) return unsupported("too many vertices");
    h->k = (int32_t)K;
    uint64_t* keys;
    VMO_TRY(sc.alloc(&keys, (size_t)std::max<int64_t>(2 * nnz, 1)));
    uint64_t sentinel = (uint64_t)K * (uint64_t)K;
    if (nnz > 0) {
      launch(graph_keys_kernel, grid_for(nnz, 256), 256, 0, s, a->rowptr, a->colidx, m, nnz, model == VMO_BIPARTITE,
                                                           (uint64_t)K, sentinel, keys);
      VMO_LAUNCHED("graph_keys");
    }
    VMO_TRY(csr_from_keys(keys, 2 * nnz, K, K, h->adj_ptr, h->adj, &h->nadj, s, sc));
    // nets = edges u < v
    int64_t nadj = h->nadj;
    int32_t *flag, *pos, *tot;
    VMO_TRY(sc.alloc(&flag, (size_t)std::max<int64_t>(nadj, 1)));
    VMO_TRY(sc.alloc(&pos, (size_t)std::max<int64_t>(nadj, 1)));
    VMO_TRY(sc.alloc(&tot, 1));
    if (nadj > 0) {
      launch(forward_flags_kernel, grid_for(nadj, 256), 256, 0, s, h->adj_ptr.ptr, h->adj.ptr, h->k, nadj, flag);
      VMO_LAUNCHED("forward_flags");
    }
    VMO_TRY(scan_exclusive<int32_t>(flag, pos, nadj, tot, s, sc));
    int64_t ne = nadj / 2;
    h->l = ne;
    h->npins = 2 * ne;
    h->nvnets = nadj;
    VMO_TRY(h->net_ptr.resize((size_t)ne + 1));
    VMO_TRY(h->pins.resize((size_t)std::max<int64_t>(2 * ne, 1)));
    VMO_TRY(h->vnets.resize((size_t)std::max<int64_t>(nadj, 1)));
    VMO_TRY(h->vtx_ptr.resize((size_t)K + 1));
    VMO_CUDA(cudaMemcpyAsync(h->vtx_ptr.ptr, h->adj_ptr.ptr, (K + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (nadj > 0) {
      launch(emit_edges_kernel, grid_for(nadj, 256), 256, 0, s, h->adj_ptr.ptr, h->adj.ptr, h->k, nadj, flag, pos,
                                                            h->net_ptr.ptr, h->pins.ptr, h->vnets.ptr);
      VMO_LAUNCHED("emit_edges");
    }
    launch(net_ptr_last_kernel, 1, 1, 0, s, h->net_ptr.ptr, tot);
    VMO_LAUNCHED("net_ptr_last");
    VMO_CUDA(cudaStreamSynchronize(s));
    return VMO_OK;
  }
  if (model == VMO_ROWNET || model == VMO_COLNET) {
    uint64_t* keys;
    VMO_TRY(sc.alloc(&keys, (size_t)std::max<int64_t>(nnz, 1)));
    DevArray<int32_t>* rows_ptr = (model == VMO_ROWNET) ? &h->net_ptr : &h->vtx_ptr;
    DevArray<int32_t>* rows_idx = (model == VMO_ROWNET) ? &h->pins : &h->vnets;
    DevArray<int32_t>* cols_ptr = (model == VMO_ROWNET) ? &h->vtx_ptr : &h->net_ptr;
    DevArray<int32_t>* cols_idx = (model == VMO_ROWNET) ? &h->vnets : &h->pins;
    int64_t cnt_r = 0, cnt_c = 0;
    if (nnz > 0) {
      launch(pattern_keys_kernel, grid_for(nnz, 256), 256, 0, s, a->rowptr, a->colidx, m, n, nnz, 0, keys);
      VMO_LAUNCHED("pattern_keys");
    }
    VMO_TRY(csr_from_keys(keys, nnz, m, n, *rows_ptr, *rows_idx, &cnt_r, s, sc));
    if (nnz > 0) {
      launch(pattern_keys_kernel, grid_for(nnz, 256), 256, 0, s, a->rowptr, a->colidx, m, n, nnz, 1, keys);
      VMO_LAUNCHED("pattern_keys");
    }
    VMO_TRY(csr_from_keys(keys, nnz, n, m, *cols_ptr, *cols_idx, &cnt_c, s, sc));
    if (model == VMO_ROWNET) {
      h->k = n; h->l = m; h->npins = cnt_r; h->nvnets = cnt_c;
    } else {
      h->k = m; h->l = n; h->npins = cnt_c; h->nvnets = cnt_r;
    }
    VMO_CUDA(cudaStreamSynchronize(s));
    return VMO_OK;
  }
  if (model == VMO_FINEGRAIN) {
    if ((int64_t)m + n > INT32_MAX) return unsupported("too many nets");
    uint64_t* keys;
    VMO_TRY(sc.alloc(&keys, (size_t)std::max<int64_t>(nnz, 1)));
    if (nnz > 0) {
      launch(pattern_keys_kernel, grid_for(nnz, 256), 256, 0, s, a->rowptr, a->colidx, m, n, nnz, 0, keys);
      VMO_LAUNCHED("pattern_keys");
    }
    DevArray<int32_t> rptr, cidx, cptr, cpins;
    int64_t u = 0, uc = 0;
    VMO_TRY(csr_from_keys(keys, nnz, m, n, rptr, cidx, &u, s, sc));
    if (2 * u > INT32_MAX) return unsupported("too many entries");
    h->k = (int32_t)u;
    h->l = (int64_t)m + n;
    h->npins = 2 * u;
    h->nvnets = 2 * u;
    VMO_TRY(h->vtx_ptr.resize((size_t)u + 1));
    VMO_TRY(h->vnets.resize((size_t)std::max<int64_t>(2 * u, 1)));
    VMO_TRY(h->net_ptr.resize((size_t)m + n + 1));
    VMO_TRY(h->pins.resize((size_t)std::max<int64_t>(2 * u, 1)));
    VMO_CUDA(cudaMemsetAsync(h->vtx_ptr.ptr, 0, sizeof(int32_t), s));
    if (m > 0) {
      launch(fg_vnets_kernel, grid_for(m, 256), 256, 0, s, rptr.ptr, cidx.ptr, m, h->vtx_ptr.ptr, h->vnets.ptr);
      VMO_LAUNCHED("fg_vnets");
    }
    uint64_t* ckeys;
    VMO_TRY(sc.alloc(&ckeys, (size_t)std::max<int64_t>(u, 1)));
    if (u > 0) {
      launch(fg_col_keys_kernel, grid_for(u, 256), 256, 0, s, cidx.ptr, u, ckeys);
      VMO_LAUNCHED("fg_col_keys");
    }
    VMO_TRY(csr_from_keys(ckeys, u, n, std::max<int64_t>(u, 1), cptr, cpins, &uc, s, sc));
    const int64_t span = std::max<int64_t>(std::max<int64_t>(u, (int64_t)m + 1), (int64_t)n);
    launch(fg_nets_kernel, grid_for(span, 256), 256, 0, s, rptr.ptr, m, cptr.ptr, cpins.ptr, n, u, h->net_ptr.ptr,
           h->pins.ptr);
    VMO_LAUNCHED("fg_nets");
    VMO_CUDA(cudaStreamSynchronize(s));
    return VMO_OK;
  }
  return invalid("unknown model");
}

// Finegrain layout from the bipartite one (Sec. 4.2): entry t at the mean of
// its row's and its column's points.
__global__ void fg_coords_kernel(const int32_t* __restrict__ vnets, int32_t k, const float4* __restrict__ xb,
                                 float4* __restrict__ xf) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k) return;
  const float4 a = xb[vnets[2 * t]], b = xb[vnets[2 * t + 1]];
  xf[t] = make_float4(0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z), 0.5f * (a.w + b.w));
}

vmo_status finegrain_coords(const vmo_hg_s* h, const float* xb, float* xf, cudaStream_t s) {
  if (h->k > 0) {
    launch(fg_coords_kernel, grid_for(h->k, 256), 256, 0, s, h->vnets.ptr, h->k, (const float4*)xb, (float4*)xf);
    VMO_LAUNCHED("fg_coords");
  }
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status components(const vmo_hg_s* h, int32_t* labels, cudaStream_t s) {
  Scratch sc(s);
  int32_t* changed;
  uint8_t* last = nullptr;
  VMO_TRY(sc.alloc(&changed, 1));
  if (h->k == 0) return VMO_OK;
  launch(cc_init_kernel, grid_for(h->k, 256), 256, 0, s, labels, h->k);
  VMO_LAUNCHED("cc_init");
  if (h->npins > 1) {
    VMO_TRY(sc.alloc(&last, h->npins));
    VMO_CUDA(cudaMemsetAsync(last, 0, h->npins, s));
    if (h->l > 0) launch(cc_last_kernel, grid_for(h->l, 256), 256, 0, s, h->net_ptr.ptr, h->l, last);
    VMO_LAUNCHED("cc_last");
  }
  for (int it = 0; it < 64; ++it) {
    VMO_CUDA(cudaMemsetAsync(changed, 0, 4, s));
    if (h->npins > 1) {
      launch(cc_hook_kernel, grid_for(h->npins, 256), 256, 0, s, h->pins.ptr, last, h->npins, labels, changed);
      VMO_LAUNCHED("cc_hook");
    }
    launch(cc_compress_kernel, grid_for(h->k, 256), 256, 0, s, labels, h->k);
    VMO_LAUNCHED("cc_compress");
    int32_t hc = 0;
    VMO_CUDA(cudaMemcpyAsync(&hc, changed, 4, cudaMemcpyDeviceToHost, s));
    VMO_CUDA(cudaStreamSynchronize(s));
    if (!hc) return VMO_OK;
  }
  return cuda_fail(cudaErrorUnknown, "components did not converge in 64 rounds", __FILE__, __LINE__);
}

vmo_status cut_size(const vmo_hg_s* h, const int32_t* part, int32_t nparts, int64_t* cutnet, int64_t* lambda1,
                    cudaStream_t s) {
  if (nparts < 1) return invalid("cut_size: nparts < 1");
  if (!part && h->k > 0) return invalid("cut_size: part is null");
  Scratch sc(s);
  unsigned long long* acc;
  VMO_TRY(sc.alloc(&acc, 2));
  VMO_CUDA(cudaMemsetAsync(acc, 0, 16, s));
  if (h->l > 0) {
    launch(cut_kernel, grid_for(h->l * 32, 256), 256, 0, s, h->net_ptr.ptr, h->pins.ptr, h->l, part, nparts, acc);
    VMO_LAUNCHED("cut");
  }
  unsigned long long host[2];
  VMO_CUDA(cudaMemcpyAsync(host, acc, 16, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  if (cutnet) *cutnet = (int64_t)host[0];
  if (lambda1) *lambda1 = (int64_t)host[1];
  return VMO_OK;
}

}  // namespace vmo
