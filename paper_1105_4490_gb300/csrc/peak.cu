// Throughput microbenchmark of the arithmetic the layout step kernel is made
// of: FP32 fused multiply-add, scalar and packed (two lanes of fp32 per
// instruction), and the approximate reciprocal square root of the
// special-function unit.  The step kernel is bound by these pipes, not by
// memory, so its roofline is this measured rate rather than a figure from
// the data sheet.  No counterpart in the paper: measurement support.
//
// Every thread runs kChains independent dependency chains (enough to cover
// the pipe latency at full occupancy) for `iters` rounds; the grid fills
// every SM several times over.  The accumulators are written out at the end
// so that nothing is optimised away.
#include <algorithm>

#include "vmo_internal.cuh"

namespace vmo {

namespace {

constexpr int kChains = 8;
constexpr int kPeakBlock = 256;

__global__ void __launch_bounds__(kPeakBlock) k_peak_ffma(int iters, float a, float b, float* __restrict__ out) {
  float acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = (float)(threadIdx.x + i);
  for (int t = 0; t < iters; ++t)
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = __fmaf_rn(acc[i], a, b);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakBlock) k_peak_ffma2(int iters, float a, float b, float* __restrict__ out) {
  float2 acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = make_float2((float)threadIdx.x, (float)i);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int t = 0; t < iters; ++t)
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = __ffma2_rn(acc[i], a2, b2);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i].x + acc[i].y;
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakBlock) k_peak_rsqrt(int iters, float* __restrict__ out) {
  float acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = 1.0f + (float)(threadIdx.x + i);
  for (int t = 0; t < iters; ++t)
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      float r;
      asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(acc[i]));
      acc[i] = r;
    }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class F>
vmo_status time_kernel(F&& launch_it, int reps, cudaStream_t s, double* ms_out) {
  cudaEvent_t a, b;
  VMO_CUDA(cudaEventCreate(&a));
  VMO_CUDA(cudaEventCreate(&b));
  launch_it();  // warm-up (clocks up, code loaded)
  VMO_CUDA(cudaEventRecord(a, s));
  for (int r = 0; r < reps; ++r) launch_it();
  VMO_CUDA(cudaEventRecord(b, s));
  VMO_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  VMO_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms_out = ms / reps;
  return VMO_OK;
}

}  // namespace

}  // namespace vmo

using namespace vmo;

extern "C" vmo_status vmo_measure_alu_peaks(double* ffma_tflops, double* ffma2_tflops, double* rsqrt_tops,
                                            int32_t* sms, void* stream) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    (void)cudaGetLastError();
    return cuda_fail(cudaErrorNoDevice, "no usable CUDA device", __FILE__, __LINE__);
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  VMO_CUDA(cudaGetDevice(&dev));
  VMO_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (sms) *sms = nsm;
  const int blocks = nsm * 8;  // 2,048 threads per SM: full occupancy
  const int64_t threads = (int64_t)blocks * kPeakBlock;
  float* out = nullptr;
  VMO_CUDA(cudaMallocAsync((void**)&out, threads * sizeof(float), s));
  g_device_allocs.fetch_add(1, std::memory_order_relaxed);
  const int iters = 4096, reps = 5;
  const float a = 0.999999f, b = 1e-7f;
  double ms = 0.0;
  vmo_status st = VMO_OK;
  if (ffma_tflops) {
    st = time_kernel([&] { k_peak_ffma<<<blocks, kPeakBlock, 0, s>>>(iters, a, b, out); }, reps, s, &ms);
    if (st == VMO_OK) *ffma_tflops = 2.0 * kChains * (double)iters * threads / (ms * 1e-3) / 1e12;
  }
  if (st == VMO_OK && ffma2_tflops) {
    st = time_kernel([&] { k_peak_ffma2<<<blocks, kPeakBlock, 0, s>>>(iters, a, b, out); }, reps, s, &ms);
    if (st == VMO_OK) *ffma2_tflops = 4.0 * kChains * (double)iters * threads / (ms * 1e-3) / 1e12;
  }
  if (st == VMO_OK && rsqrt_tops) {
    st = time_kernel([&] { k_peak_rsqrt<<<blocks, kPeakBlock, 0, s>>>(iters / 4, out); }, reps, s, &ms);
    if (st == VMO_OK) *rsqrt_tops = (double)kChains * (double)(iters / 4) * threads / (ms * 1e-3) / 1e12;
  }
  cudaFreeAsync(out, s);
  if (st == VMO_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "alu peak kernels", __FILE__, __LINE__);
  }
  return st;
}
