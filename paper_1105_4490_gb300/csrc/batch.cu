// Batched ordering: many independent matrices in one launch sequence.
//
// The matrices are joined block-diagonally on the device (one table-driven
// kernel for the row pointers and one for the column indices), the symmetric
// model of the joined pattern is built once, and every connected component of
// every matrix becomes one problem of the layout batch and one root of the
// level-synchronous recursion.  All per-problem arithmetic (grid, group size,
// sort segment, step length, k-means++ draws keyed by heap number) depends on
// the problem alone, so each matrix's permutation is the one it gets when
// ordered by itself.
#include <algorithm>

#include "components.cuh"

namespace vmo {

vmo_status validate_csr_async(const vmo_csr* a, int32_t* bad, cudaStream_t s);
vmo_status build_model(const vmo_csr* a, vmo_model model, vmo_hg_s* h, cudaStream_t s);
vmo_status ensure_device_public();
vmo_status check_params_public(const vmo_params* p);

namespace {

struct MatDesc {
  const int32_t* rowptr;
  const int32_t* colidx;
  int64_t row_base;
  int64_t nnz_base;
};

__device__ inline int find_base(const int64_t* __restrict__ base, int n, int64_t i) {
  int lo = 0, hi = n;  // base[lo] <= i < base[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (base[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_join_rows(const MatDesc* __restrict__ md, const int64_t* __restrict__ row_base, int count,
                            int64_t K, int64_t NNZ, int32_t* __restrict__ rowptr) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > K) return;
  if (r == K) { rowptr[K] = (int32_t)NNZ; return; }
  int i = find_base(row_base, count, r);
  rowptr[r] = (int32_t)(md[i].nnz_base + md[i].rowptr[r - md[i].row_base]);
}

__global__ void k_join_cols(const MatDesc* __restrict__ md, const int64_t* __restrict__ nnz_base, int count,
                            int64_t NNZ, int32_t* __restrict__ colidx) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NNZ) return;
  int i = find_base(nnz_base, count, t);
  colidx[t] = (int32_t)(md[i].row_base + md[i].colidx[t - md[i].nnz_base]);
}

__global__ void k_split_perm(const int32_t* __restrict__ ord, int64_t K, const int64_t* __restrict__ row_base, int count,
                             int32_t* __restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K) return;
  int mi = find_base(row_base, count, i);
  perm[i] = (int32_t)(ord[i] - row_base[mi]);
}

}  // namespace

// Joins the matrices block-diagonally and builds the symmetric model.
struct Joined {
  std::vector<int64_t> row_base;
  int64_t* drb = nullptr;
  int64_t K = 0;
};

static vmo_status join_and_build(const vmo_csr* mats, int32_t count, vmo_hg_s& h, Joined& J, cudaStream_t s,
                                 Scratch& sc) {
  if (count < 0 || (count > 0 && !mats)) return invalid("batch: bad matrix list");
  std::vector<int64_t> row_base(count + 1, 0), nnz_base(count + 1, 0);
  std::vector<MatDesc> md(count);
  for (int i = 0; i < count; ++i) {
    if (mats[i].m != mats[i].n) return invalid("batch: matrix " + std::to_string(i) + " is not square");
    row_base[i + 1] = row_base[i] + mats[i].m;
    nnz_base[i + 1] = nnz_base[i] + mats[i].nnz;
    md[i] = MatDesc{mats[i].rowptr, mats[i].colidx, row_base[i], nnz_base[i]};
  }
  const int64_t K = row_base[count], NNZ = nnz_base[count];
  if (K > INT32_MAX / 2 || NNZ > INT32_MAX) return unsupported("batch: more than 2^30 rows or 2^31 nonzeros");
  J.row_base = row_base;
  J.K = K;
  int32_t* bad;
  VMO_TRY(sc.alloc(&bad, 1));
  VMO_CUDA(cudaMemsetAsync(bad, 0, 4, s));
  for (int i = 0; i < count; ++i) VMO_TRY(validate_csr_async(&mats[i], bad, s));
  int32_t hbad = 0;
  VMO_CUDA(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  if (hbad) return invalid("batch: a matrix has a malformed CSR");
  MatDesc* dmd;
  int64_t *drb, *dnb;
  int32_t *rowptr, *colidx;
  VMO_TRY(sc.alloc(&dmd, std::max(count, 1)));
  VMO_TRY(sc.alloc(&drb, count + 1));
  J.drb = drb;
  VMO_TRY(sc.alloc(&dnb, count + 1));
  VMO_TRY(sc.alloc(&rowptr, K + 1));
  VMO_TRY(sc.alloc(&colidx, std::max<int64_t>(NNZ, 1)));
  VMO_CUDA(cudaMemcpyAsync(dmd, md.data(), count * sizeof(MatDesc), cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(drb, row_base.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(dnb, nnz_base.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  launch(k_join_rows, grid_for(K + 1, 256), 256, 0, s, dmd, drb, count, K, NNZ, rowptr);
  if (NNZ > 0) launch(k_join_cols, grid_for(NNZ, 256), 256, 0, s, dmd, dnb, count, NNZ, colidx);
  VMO_LAUNCHED("join");
  VMO_CUDA(cudaStreamSynchronize(s));  // host tables above must outlive the copies
  vmo_csr joined{(int32_t)K, (int32_t)K, NNZ, rowptr, colidx};
  return build_model(&joined, VMO_SYMMETRIC, &h, s);
}

vmo_status batch_order(const vmo_csr* mats, int32_t count, const float* coords, const vmo_params* p, int32_t sbd,
                       int32_t* perm, cudaStream_t s) {
  Scratch sc(s);
  vmo_hg_s h;
  Joined J;
  VMO_TRY(join_and_build(mats, count, h, J, s, sc));
  const int64_t K = J.K;
  if (K == 0) return VMO_OK;
  if (!perm) return invalid("batch: perm is null");
  ComponentGroups g;
  VMO_TRY(group_components(&h, g, s, sc));
  float4* x = (float4*)coords;
  if (!x) {
    VMO_TRY(sc.alloc(&x, K));
    VMO_TRY(layout_grouped(&h, g, p, x, s, sc));
  }
  OrderState st;
  VMO_TRY(order_grouped(&h, g, x, p, sbd, st, s, sc));
  launch(k_split_perm, grid_for(K, 256), 256, 0, s, st.ord, K, J.drb, count, perm);
  VMO_LAUNCHED("split_perm");
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status batch_layout(const vmo_csr* mats, int32_t count, const vmo_params* p, float* coords, cudaStream_t s) {
  Scratch sc(s);
  vmo_hg_s h;
  Joined J;
  VMO_TRY(join_and_build(mats, count, h, J, s, sc));
  if (J.K == 0) return VMO_OK;
  if (!coords || ((uintptr_t)coords & 15u)) return invalid("batch: coords null or not 16-byte aligned");
  ComponentGroups g;
  VMO_TRY(group_components(&h, g, s, sc));
  VMO_TRY(layout_grouped(&h, g, p, (float4*)coords, s, sc));
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

}  // namespace vmo

using namespace vmo;

extern "C" vmo_status vmo_batch_layout(const vmo_csr* mats, int32_t count, const vmo_params* params, float* coords,
                                       void* stream) {
  VMO_TRY(ensure_device_public());
  VMO_TRY(check_params_public(params));
  return batch_layout(mats, count, params, coords, (cudaStream_t)stream);
}

extern "C" vmo_status vmo_batch_order(const vmo_csr* mats, int32_t count, const float* coords,
                                      const vmo_params* params, int32_t sbd, int32_t* perm, void* stream) {
  VMO_TRY(ensure_device_public());
  VMO_TRY(check_params_public(params));
  if (coords && ((uintptr_t)coords & 15u)) return invalid("coords must be 16-byte aligned");
  return batch_order(mats, count, coords, params, sbd, perm, (cudaStream_t)stream);
}
