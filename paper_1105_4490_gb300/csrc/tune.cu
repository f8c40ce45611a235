// Autotuner of the launch shapes that never change a result: the largest
// step launch that takes the two-rows-in-flight variant of the step kernel,
// the widest radix digit of the binning sort, the positions per thread of
// the Lloyd assignment, and the largest problem whose level is binned by one
// block per problem.  Every candidate orders the caller's matrices
// through vmo_batch_order; the fastest (median of the repetitions, CUDA
// events on the caller's stream) becomes the process-wide setting.  The
// paper has no counterpart: these are choices of this GPU implementation.
#include <algorithm>
#include <vector>

#include "vmo_internal.cuh"

namespace vmo {

Tuning g_tuning;

namespace {

vmo_tuning current() {
  vmo_tuning t;
  t.small_step_threads = g_tuning.small_step_threads.load();
  t.radix_max_bits = g_tuning.radix_max_bits.load();
  t.assign_items = g_tuning.assign_items.load();
  t.small_bin_points = g_tuning.small_bin_points.load();
  return t;
}

void apply(const vmo_tuning& t) {
  g_tuning.small_step_threads.store(t.small_step_threads);
  g_tuning.radix_max_bits.store(t.radix_max_bits);
  g_tuning.assign_items.store(t.assign_items);
  g_tuning.small_bin_points.store(t.small_bin_points);
}

vmo_status valid(const vmo_tuning* t) {
  if (!t) return invalid("tuning is null");
  if (t->small_step_threads < 0 || t->small_step_threads > (int64_t(1) << 40))
    return invalid("small_step_threads must be in [0, 2^40]");
  if (t->radix_max_bits < 8 || t->radix_max_bits > 10) return invalid("radix_max_bits must be 8, 9 or 10");
  if (t->assign_items != 1 && t->assign_items != 2 && t->assign_items != 4 && t->assign_items != 8)
    return invalid("assign_items must be 1, 2, 4 or 8");
  if (t->small_bin_points < 0 || t->small_bin_points > kSortTile)
    return invalid("small_bin_points must be in [0, 2048]");
  return VMO_OK;
}

// Median device time (ms) of `reps` orderings of the matrices, after one
// untimed call.
vmo_status time_order(const vmo_csr* mats, int32_t count, const vmo_params* p, int32_t reps, int32_t* perm,
                      cudaStream_t s, double* ms) {
  cudaEvent_t a, b;
  VMO_CUDA(cudaEventCreate(&a));
  VMO_CUDA(cudaEventCreate(&b));
  vmo_status st = vmo_batch_order(mats, count, nullptr, p, 0, perm, s);
  std::vector<float> t;
  for (int r = 0; r < reps && st == VMO_OK; ++r) {
    cudaEventRecord(a, s);
    st = vmo_batch_order(mats, count, nullptr, p, 0, perm, s);
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "autotune", __FILE__, __LINE__);
    float e = 0.f;
    cudaEventElapsedTime(&e, a, b);
    t.push_back(e);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != VMO_OK) return st;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return VMO_OK;
}

}  // namespace
}  // namespace vmo

using namespace vmo;

extern "C" void vmo_get_tuning(vmo_tuning* out) {
  if (out) *out = current();
}

extern "C" vmo_status vmo_set_tuning(const vmo_tuning* t) {
  VMO_TRY(valid(t));
  apply(*t);
  return VMO_OK;
}

extern "C" vmo_status vmo_autotune(const vmo_csr* mats, int32_t count, const vmo_params* params, int32_t reps,
                                   vmo_tuning* best, double* best_ms, double* default_ms, void* stream) {
  if (!mats || count <= 0) return invalid("autotune needs at least one matrix");
  if (reps < 1 || reps > 100) return invalid("reps must be in [1, 100]");
  int64_t rows = 0;
  for (int32_t i = 0; i < count; ++i) rows += std::max(mats[i].m, 0);
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* perm = nullptr;
  VMO_CUDA(cudaMalloc(&perm, (size_t)std::max<int64_t>(rows, 1) * sizeof(int32_t)));
  g_device_allocs.fetch_add(1, std::memory_order_relaxed);
  const vmo_tuning start = current();
  vmo_tuning bt = start;
  double bms = 0.0, dms = 0.0;
  vmo_status st = time_order(mats, count, params, reps, perm, s, &bms);
  dms = bms;
  // coordinate descent over the four choices, from the current setting
  const std::vector<int64_t> steps = {0, 4864, 9728, 19456, 38912, 77824, 155648};
  const std::vector<int> bits = {8, 9, 10};
  const std::vector<int> items = {1, 2, 4, 8};
  const std::vector<int> bins = {0, 512, kSortTile};
  for (int knob = 0; knob < 4 && st == VMO_OK; ++knob) {
    const size_t nc = knob == 0 ? steps.size() : knob == 1 ? bits.size() : knob == 2 ? items.size() : bins.size();
    for (size_t c = 0; c < nc && st == VMO_OK; ++c) {
      vmo_tuning t = bt;
      if (knob == 0) t.small_step_threads = steps[c];
      if (knob == 1) t.radix_max_bits = bits[c];
      if (knob == 2) t.assign_items = items[c];
      if (knob == 3) t.small_bin_points = bins[c];
      if (t.small_step_threads == bt.small_step_threads && t.radix_max_bits == bt.radix_max_bits &&
          t.assign_items == bt.assign_items && t.small_bin_points == bt.small_bin_points)
        continue;
      apply(t);
      double ms = 0.0;
      st = time_order(mats, count, params, reps, perm, s, &ms);
      if (st == VMO_OK && ms < bms) {
        bms = ms;
        bt = t;
      }
    }
  }
  cudaFree(perm);
  if (st != VMO_OK) {
    apply(start);
    return st;
  }
  apply(bt);
  if (best) *best = bt;
  if (best_ms) *best_ms = bms;
  if (default_ms) *default_ms = dms;
  return VMO_OK;
}
