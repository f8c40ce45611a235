// Block-level pieces shared by the device-wide radix sort (prims.cu) and the
// one-block binning of small layout levels (layout.cu): warp and block scans,
// and the stable LSD sort of one tile of at most kSortTile (key, value) pairs
// held in shared memory.
#pragma once

#include "vmo_internal.cuh"

namespace vmo {

constexpr int kSortThreads = 256;
constexpr int kSortItems = kSortTile / kSortThreads;  // 8
constexpr int kSortWarps = kSortThreads / 32;

template <class T>
__device__ T warp_inclusive(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if ((int)lane_id() >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024).
template <class T>
__device__ T block_exclusive(T v, T* warp_sums, T* total) {
  const int lane = lane_id(), warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  T inc = warp_inclusive(v);
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T s = (lane < nw) ? warp_sums[lane] : T(0);
    T si = warp_inclusive(s);
    if (lane < nw) warp_sums[lane] = si - s;
    if (lane == nw - 1) warp_sums[32] = si;
  }
  __syncthreads();
  T out = warp_sums[warp] + inc - v;
  if (total) *total = warp_sums[32];
  __syncthreads();
  return out;
}

// Shared memory of one tile sort: two buffers of pairs, per-warp digit
// counters, digit bases and the scan's warp sums.
struct TileSortSmem {
  uint32_t key[2][kSortTile];
  uint32_t val[2][kSortTile];
  uint32_t wcnt[kSortWarps][256];
  uint32_t dbase[256];
  uint32_t ws[33];
};

// Stable sort by bits [0, bits) of the n <= kSortTile pairs the block has
// written to (sm.key[0], sm.val[0]), by all kSortThreads threads of the block
// (every thread calls it).  8-bit digits, LSD; inside a digit the ranks follow
// the input order (a warp's lanes by __match_any_sync, then the warps in
// order).  Returns the buffer that holds the sorted pairs, readable by every
// thread of the block on return.
__device__ inline int tile_sort_smem(TileSortSmem& sm, int n, int bits) {
  constexpr int R = 256;
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    for (int i = threadIdx.x; i < kSortWarps * R; i += blockDim.x) (&sm.wcnt[0][0])[i] = 0;
    __syncthreads();
    uint32_t rank[kSortItems], dig[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const int idx = warp * (32 * kSortItems) + j * 32 + lane;
      const bool valid = idx < n;
      const uint32_t dg = valid ? ((sm.key[cur][idx] >> shift) & (R - 1)) : (uint32_t)R;
      dig[j] = dg;
      const unsigned peers = __match_any_sync(0xffffffffu, dg);
      const uint32_t base = valid ? sm.wcnt[warp][dg] : 0u;
      rank[j] = base + __popc(peers & lt);
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) sm.wcnt[warp][dg] = base + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: prefix over the warps, total; then bases by a block scan
    uint32_t tot = 0;
    {
      const int dg = threadIdx.x;  // blockDim.x == R
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = sm.wcnt[w][dg];
        sm.wcnt[w][dg] = tot;
        tot += c;
      }
    }
    const uint32_t ex = block_exclusive<uint32_t>(tot, sm.ws, nullptr);
    sm.dbase[threadIdx.x] = ex;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      if (dig[j] >= (uint32_t)R) continue;
      const int idx = warp * (32 * kSortItems) + j * 32 + lane;
      const uint32_t dst = sm.dbase[dig[j]] + sm.wcnt[warp][dig[j]] + rank[j];
      sm.key[cur ^ 1][dst] = sm.key[cur][idx];
      sm.val[cur ^ 1][dst] = sm.val[cur][idx];
    }
    __syncthreads();
    cur ^= 1;
  }
  if (bits <= 0) __syncthreads();
  return cur;
}

}  // namespace vmo
