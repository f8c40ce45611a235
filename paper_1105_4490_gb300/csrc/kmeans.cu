// m-way k-means++ (Algorithm 5 with m centres): a one-shot m-way partition of
// a point set, in the readings of the recursion's 2-means (integer D^2
// weights on the grid 2^-(34-2e), draws keyed by (seed, key, centre index),
// fp32 distances without FMA, ties to the smaller centre, exact fixed-point
// means on the grid 2^-(30-e)); for m = 2 it is vmo_bisect.
//
// Seeding takes m - 1 rounds of (running minimum distance and weights, scan,
// pick); a Lloyd round is one assignment kernel (centres in shared memory,
// per-block fixed-point sums in shared memory folded into global int64 sums
// with atomics, exact and order-free) and one update kernel.
#include <algorithm>

#include "vmo_internal.cuh"

namespace vmo {

vmo_status ensure_device_public();

namespace {

constexpr int kKmBlock = 256;
constexpr int kKmMaxCentres = 256;

struct KmState {
  int e;             // max |x| < 2^e
  int chosen;        // centres picked by the seeding
  int stopped;       // seeding stopped: every point on a chosen centre
  int converged;     // no label changed in a Lloyd round
  int changed;       // a label changed in the current round
  uint32_t maxabs;   // float bits of max |x|
};

template <int D>
__global__ void k_km_gather(const float4* __restrict__ x, const int32_t* __restrict__ verts, int64_t n,
                            float4* __restrict__ xo, KmState* __restrict__ st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t mx = 0;
  if (i < n) {
    const float4 p = x[verts[i]];
    xo[i] = p;
#pragma unroll
    for (int m = 0; m < D; ++m) mx = max(mx, __float_as_uint(fabsf(comp(p, m))));
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane_id() == 0 && mx) atomicMax(&st->maxabs, mx);
}

// First centre: point floor(n * r0 / 2^64).
__global__ void k_km_seed0(const float4* __restrict__ xo, int64_t n, uint64_t seed, uint64_t key,
                           float4* __restrict__ z, KmState* __restrict__ st) {
  st->e = exponent_of(st->maxabs);
  st->chosen = 1;
  st->stopped = 0;
  st->converged = 0;
  st->changed = 0;
  z[0] = xo[scale_draw((uint64_t)n, rand64(seed ^ kTagKmeans, key, 0))];
}

// Running minimum squared distance to the chosen centres (centre c just
// picked) and its integer D^2 weight floor(dmin * 2^(34 - 2e)).
template <int D>
__global__ void k_km_weights(const float4* __restrict__ xo, int64_t n, const float4* __restrict__ z, int c,
                             float* __restrict__ dmin, unsigned long long* __restrict__ w,
                             const KmState* __restrict__ st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || st->stopped) return;
  const float dd = sqdist32<D>(xo[i], z[c]);
  const float dm = c == 0 ? dd : fminf(dmin[i], dd);
  dmin[i] = dm;
  w[i] = (unsigned long long)floorf(__fmul_rn(dm, exp2i_f(34 - 2 * st->e)));
}

// Centre c: the first point whose inclusive prefix of the weights exceeds
// floor(total * r_c / 2^64); a zero total stops the seeding.
__global__ void k_km_pick(const float4* __restrict__ xo, int64_t n, const unsigned long long* __restrict__ w,
                          const unsigned long long* __restrict__ pre, uint64_t seed, uint64_t key, int c,
                          float4* __restrict__ z, KmState* __restrict__ st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || st->stopped) return;
  const unsigned long long total = pre[n - 1];
  if (total == 0) {
    if (i == 0) st->stopped = 1;
    return;
  }
  const unsigned long long thr = scale_draw(total, rand64(seed ^ kTagKmeans, key, (uint64_t)c));
  if (pre[i] - w[i] <= thr && thr < pre[i]) {
    z[c] = xo[i];
    st->chosen = c + 1;
  }
}

// Centres the seeding did not reach are copies of the first (they never win).
__global__ void k_km_fill(float4* __restrict__ z, int m, const KmState* __restrict__ st) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < m && c >= st->chosen) z[c] = z[0];
}

template <int D>
__device__ __forceinline__ int km_nearest(const float4& p, const float4* zs, int m) {
  int best = 0;
  float bd = sqdist32<D>(p, zs[0]);
  for (int j = 1; j < m; ++j) {
    const float dj = sqdist32<D>(p, zs[j]);
    if (dj < bd) {
      bd = dj;
      best = j;
    }
  }
  return best;
}

// One Lloyd assignment (it >= 0) or the final labelling (it < 0).
template <int D>
__global__ void __launch_bounds__(kKmBlock) k_km_assign(const float4* __restrict__ xo, int64_t n, int m, int it,
                                                        const float4* __restrict__ z, int32_t* __restrict__ lab,
                                                        unsigned long long* __restrict__ S,
                                                        unsigned long long* __restrict__ cnt,
                                                        KmState* __restrict__ st) {
  __shared__ float4 zs[kKmMaxCentres];
  __shared__ unsigned long long ss[kKmMaxCentres * 4];
  __shared__ unsigned long long sc[kKmMaxCentres];
  const bool final_pass = it < 0;
  if (!final_pass && st->converged) return;  // block-uniform
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    zs[j] = z[j];
    sc[j] = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) ss[j * 4 + q] = 0;
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const float fx = exp2i_f(30 - st->e);
  if (i < n) {
    const float4 p = xo[i];
    const int l = km_nearest<D>(p, zs, m);
    if (!final_pass && it > 0 && lab[i] != l) st->changed = 1;
    lab[i] = l;
    atomicAdd(&sc[l], 1ull);
    if (!final_pass) {
#pragma unroll
      for (int q = 0; q < D; ++q)
        atomicAdd(&ss[l * 4 + q], (unsigned long long)__float2ll_rn(__fmul_rn(comp(p, q), fx)));
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    if (sc[j] == 0) continue;
    atomicAdd(&cnt[j], sc[j]);
    if (!final_pass)
      for (int q = 0; q < D; ++q) atomicAdd(&S[j * 4 + q], ss[j * 4 + q]);
  }
}

// Centre update: z = fp32((double(sum) / count) * 2^-(30 - e)) for non-empty
// clusters; a round without a change ends the iteration.
template <int D>
__global__ void k_km_update(float4* __restrict__ z, int m, int it, unsigned long long* __restrict__ S,
                            unsigned long long* __restrict__ cnt, KmState* __restrict__ st) {
  const int j = threadIdx.x;  // one block of at least m threads
  const bool done = st->converged || (it > 0 && !st->changed);
  __syncthreads();
  if (j < m) {
    if (!done && cnt[j] > 0) {
      const double inv = __longlong_as_double((long long)(1023 - (30 - st->e)) << 52);  // 2^-P
      float c[4] = {z[j].x, z[j].y, z[j].z, z[j].w};
#pragma unroll
      for (int q = 0; q < D; ++q)
        c[q] = __double2float_rn(__dmul_rn(__ddiv_rn(__ll2double_rn((long long)S[j * 4 + q]), (double)cnt[j]), inv));
      z[j] = make_float4(c[0], c[1], c[2], c[3]);
    }
    cnt[j] = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) S[j * 4 + q] = 0;
  }
  __syncthreads();
  if (j == 0) {
    if (done) st->converged = 1;
    st->changed = 0;
  }
}

__global__ void k_km_nonempty(const unsigned long long* __restrict__ cnt, int m, int32_t* __restrict__ out) {
  int c = 0;
  for (int j = 0; j < m; ++j) c += cnt[j] > 0;
  *out = c;
}

template <class F>
void km_dispatch(int d, F&& f) {
  if (d == 2) f(std::integral_constant<int, 2>());
  else if (d == 3) f(std::integral_constant<int, 3>());
  else f(std::integral_constant<int, 4>());
}

}  // namespace

vmo_status kmeans_m(int32_t d, const float* coords, const int32_t* verts, int32_t nverts, int32_t m, uint64_t seed,
                    uint64_t key, int32_t km_iters, int32_t* labels, float* centres, int32_t* nonempty,
                    cudaStream_t s) {
  if (d < 2 || d > 4) return unsupported("d must be 2, 3 or 4");
  if (m < 1 || m > kKmMaxCentres) return invalid("m must be in [1, 256]");
  if (nverts < 0 || km_iters < 0) return invalid("negative size");
  if (!centres || ((uintptr_t)centres & 15u)) return invalid("centres null or not 16-byte aligned");
  if (nverts > 0 && (!coords || !verts || !labels || ((uintptr_t)coords & 15u)))
    return invalid("null or unaligned argument");
  VMO_CUDA(cudaMemsetAsync(centres, 0, (size_t)m * sizeof(float4), s));
  if (nverts == 0) {
    if (nonempty) *nonempty = 0;
    return VMO_OK;
  }
  Scratch sc(s);
  const int64_t n = nverts;
  float4 *xo, *z = reinterpret_cast<float4*>(centres);
  float* dmin;
  unsigned long long *w, *pre, *S, *cnt;
  KmState* st;
  int32_t* ne;
  VMO_TRY(sc.alloc(&xo, n));
  VMO_TRY(sc.alloc(&dmin, n));
  VMO_TRY(sc.alloc(&w, n));
  VMO_TRY(sc.alloc(&pre, n));
  VMO_TRY(sc.alloc(&S, (size_t)m * 4));
  VMO_TRY(sc.alloc(&cnt, (size_t)m));
  VMO_TRY(sc.alloc(&st, 1));
  VMO_TRY(sc.alloc(&ne, 1));
  VMO_CUDA(cudaMemsetAsync(st, 0, sizeof(KmState), s));
  VMO_CUDA(cudaMemsetAsync(S, 0, (size_t)m * 4 * sizeof(unsigned long long), s));
  VMO_CUDA(cudaMemsetAsync(cnt, 0, (size_t)m * sizeof(unsigned long long), s));
  const unsigned nb = (unsigned)((n + kKmBlock - 1) / kKmBlock);
  vmo_status stt = VMO_OK;
  km_dispatch(d, [&](auto DC) {
    constexpr int D = decltype(DC)::value;
    launch(k_km_gather<D>, nb, kKmBlock, 0, s, reinterpret_cast<const float4*>(coords), verts, n, xo, st);
    launch(k_km_seed0, 1, 1, 0, s, xo, n, seed, key, z, st);
    for (int c = 1; c < m && stt == VMO_OK; ++c) {
      launch(k_km_weights<D>, nb, kKmBlock, 0, s, xo, n, z, c - 1, dmin, w, st);
      stt = scan_inclusive<uint64_t>((const uint64_t*)w, (uint64_t*)pre, n, s, sc);
      if (stt == VMO_OK) launch(k_km_pick, nb, kKmBlock, 0, s, xo, n, w, pre, seed, key, c, z, st);
    }
    if (stt != VMO_OK) return;
    launch(k_km_fill, 1, kKmMaxCentres, 0, s, z, m, st);
    for (int it = 0; it < km_iters; ++it) {
      launch(k_km_assign<D>, nb, kKmBlock, 0, s, xo, n, m, it, z, labels, S, cnt, st);
      launch(k_km_update<D>, 1, kKmMaxCentres, 0, s, z, m, it, S, cnt, st);
      if (it % 4 == 3 && it + 1 < km_iters) {  // stop early once converged
        KmState h;
        cudaError_t e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
          stt = cuda_fail(e, "kmeans convergence check", __FILE__, __LINE__);
          break;
        }
        if (h.converged) break;
      }
    }
    if (stt != VMO_OK) return;
    launch(k_km_assign<D>, nb, kKmBlock, 0, s, xo, n, m, -1, z, labels, S, cnt, st);
    launch(k_km_nonempty, 1, 1, 0, s, cnt, m, ne);
  });
  VMO_TRY(stt);
  VMO_LAUNCHED("kmeans");
  int32_t h = 0;
  VMO_CUDA(cudaMemcpyAsync(&h, ne, 4, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  if (nonempty) *nonempty = h;
  return VMO_OK;
}

}  // namespace vmo

extern "C" vmo_status vmo_kmeans(int32_t d, const float* coords, const int32_t* verts, int32_t nverts, int32_t m,
                                 uint64_t seed, uint64_t key, int32_t km_iters, int32_t* labels, float* centres,
                                 int32_t* nonempty, void* stream) {
  VMO_TRY(vmo::ensure_device_public());
  return vmo::kmeans_m(d, coords, verts, nverts, m, seed, key, km_iters, labels, centres, nonempty,
                       (cudaStream_t)stream);
}
