// Device-wide primitives: scans and a stable LSD radix sort.
//
// Scan: reduce tiles -> scan tile sums in one block -> scan each tile with its
// offset (tiles of 2048 elements staged through shared memory so global loads
// and stores are coalesced).
//
// Radix sort: 8-bit digits, one histogram kernel and one scatter kernel per
// pass plus a scan of the (segment, digit, tile)-ordered histogram.  The
// scatter ranks keys stably inside a warp with __match_any_sync, so equal keys
// keep their input order.  Tiles never straddle a segment, so with the
// histogram laid out segment-major the same kernels sort many independent
// segments (one per problem of a batch) in one launch sequence.
#include <algorithm>

#include <type_traits>

#include "blocksort.cuh"

namespace vmo {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__global__ void scan_reduce_kernel(const T* __restrict__ in, int64_t n, T* __restrict__ partial) {
  __shared__ T ws[33];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  T acc = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t g = base + i;
    if (g < n) acc += in[g];
  }
  T tot;
  block_exclusive<T>(acc, ws, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <class T>
__global__ void scan_partials_kernel(T* partial, int64_t ntiles, T* total) {
  __shared__ T ws[33];
  T carry = 0;
  for (int64_t b = 0; b < ntiles; b += blockDim.x) {
    int64_t i = b + threadIdx.x;
    T v = (i < ntiles) ? partial[i] : T(0);
    T tot;
    T ex = block_exclusive<T>(v, ws, &tot);
    if (i < ntiles) partial[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <class T, bool Inclusive>
__global__ void scan_tile_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t n,
                                 const T* __restrict__ partial) {
  __shared__ T tile[kScanTile];
  __shared__ T ws[33];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t g = base + i;
    tile[i] = (g < n) ? in[g] : T(0);
  }
  __syncthreads();
  T loc[kScanItems];
  T acc = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    loc[j] = tile[threadIdx.x * kScanItems + j];
    acc += loc[j];
  }
  T ex = block_exclusive<T>(acc, ws, nullptr) + partial[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    T v = loc[j];
    tile[threadIdx.x * kScanItems + j] = Inclusive ? ex + v : ex;
    ex += v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t g = base + i;
    if (g < n) out[g] = tile[i];
  }
}

template <class T, bool Inclusive>
vmo_status scan_impl(const T* in, T* out, int64_t n, T* total, cudaStream_t s, Scratch& sc) {
  if (n <= 0) {
    if (total) VMO_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
    return VMO_OK;
  }
  int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  T* partial;
  VMO_TRY(sc.alloc(&partial, (size_t)ntiles));
  launch(scan_reduce_kernel<T>, (unsigned)ntiles, kScanThreads, 0, s, in, n, partial);
  launch(scan_partials_kernel<T>, 1, 1024, 0, s, partial, ntiles, total);
  launch(scan_tile_kernel<T, Inclusive>, (unsigned)ntiles, kScanThreads, 0, s, in, out, n, partial);
  VMO_LAUNCHED("scan");
  return VMO_OK;
}

// ------------------------------- radix sort --------------------------------
// LSD passes of B-bit digits, B in {6, 8, 9, 10} chosen per sort: the fewest
// passes of at most 10 bits (or the tuned cap, 8 or 9), then the smallest
// listed width covering the key bits in that many passes (18-bit cell keys:
// 2 passes of 9 bits).
constexpr int kMaxRadixBits = 10;

struct TileInfo {
  int64_t start;
  int32_t count;
  int64_t hist_base;  // index of (digit 0, this tile) in the histogram
  int32_t stride;     // distance between digits (tiles in the segment)
};

__device__ inline TileInfo tile_info(const SortSegments& sg, int64_t n, int64_t t, int radix) {
  TileInfo ti;
  if (sg.tile_seg == nullptr) {
    ti.start = t * kSortTile;
    int64_t c = n - ti.start;
    ti.count = (int32_t)(c < kSortTile ? c : kSortTile);
    ti.hist_base = t;
    ti.stride = (int32_t)sg.ntiles;
  } else {
    int32_t seg = sg.tile_seg[t];
    int32_t t0 = sg.seg_tile0[seg], nt = sg.seg_tile0[seg + 1] - t0;
    ti.start = sg.tile_start[t];
    ti.count = sg.tile_count[t];
    ti.hist_base = (int64_t)t0 * radix + (t - t0);
    ti.stride = nt;
  }
  return ti;
}

template <class K, int BITS>
__global__ void radix_hist_kernel(const K* __restrict__ keys, int64_t n, int shift, SortSegments sg,
                                  uint32_t* __restrict__ hist) {
  pdl_wait();
  constexpr int R = 1 << BITS;
  __shared__ uint32_t h[R];
  for (int i = threadIdx.x; i < R; i += blockDim.x) h[i] = 0;
  __syncthreads();
  TileInfo ti = tile_info(sg, n, blockIdx.x, R);
  for (int i = threadIdx.x; i < ti.count; i += blockDim.x) {
    uint32_t dg = (uint32_t)(keys[ti.start + i] >> shift) & (R - 1);
    atomicAdd(&h[dg], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < R; i += blockDim.x) hist[ti.hist_base + (int64_t)i * ti.stride] = h[i];
}

// Row prefix of the tile histograms: one thread per (segment, digit) row
// (the counts of that digit in the segment's tiles, contiguous): exclusive
// prefix in place, row total to rowtot.
__global__ void radix_rowscan(uint32_t* __restrict__ hist, SortSegments sg, int R, int64_t nrows,
                              uint32_t* __restrict__ rowtot) {
  pdl_wait();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int seg = (int)(r / R), d = (int)(r % R);
  int64_t t0 = 0, nt = sg.ntiles;
  if (sg.tile_seg) {
    t0 = sg.seg_tile0[seg];
    nt = sg.seg_tile0[seg + 1] - t0;
  }
  if (nt > kLongSegTiles || nt <= 1) return;  // long: radix_rowscan_warp; single tile: the scatter's own counts
  uint32_t* row = hist + t0 * R + (int64_t)d * nt;
  uint32_t run = 0;
  int64_t t = 0;
  for (; t + 4 <= nt; t += 4) {
    const uint32_t c0 = row[t], c1 = row[t + 1], c2 = row[t + 2], c3 = row[t + 3];
    row[t] = run;
    run += c0;
    row[t + 1] = run;
    run += c1;
    row[t + 2] = run;
    run += c2;
    row[t + 3] = run;
    run += c3;
  }
  for (; t < nt; ++t) {
    const uint32_t c = row[t];
    row[t] = run;
    run += c;
  }
  rowtot[r] = run;
}

// Same for the rows of long segments (more than kLongSegTiles tiles), one
// warp per row; nrows = R x the long segments (all rows when unsegmented).
__global__ void radix_rowscan_warp(uint32_t* __restrict__ hist, SortSegments sg, int R, int64_t nrows,
                                   uint32_t* __restrict__ rowtot) {
  pdl_wait();
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= nrows) return;
  const int lane = lane_id();
  const int seg = sg.tile_seg ? sg.long_seg[w / R] : 0, d = (int)(w % R);
  const int64_t r = (int64_t)seg * R + d;
  int64_t t0 = 0, nt = sg.ntiles;
  if (sg.tile_seg) {
    t0 = sg.seg_tile0[seg];
    nt = sg.seg_tile0[seg + 1] - t0;
  }
  uint32_t* row = hist + t0 * R + (int64_t)d * nt;
  uint32_t carry = 0;
  for (int64_t b = 0; b < nt; b += 32) {
    const int64_t t = b + lane;
    const uint32_t c = t < nt ? row[t] : 0u;
    const uint32_t inc = warp_inclusive(c);
    if (t < nt) row[t] = carry + inc - c;
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (lane == 0) rowtot[r] = carry;
}

template <class K, bool HasVal, int BITS>
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    const K* __restrict__ keys, const uint32_t* __restrict__ vals, K* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, int64_t n, int shift, SortSegments sg, const uint32_t* __restrict__ offs,
    const uint32_t* __restrict__ rowtot) {
  pdl_wait();
  constexpr int R = 1 << BITS;
  constexpr int PER = (R + kSortThreads - 1) / kSortThreads;
  // the per-warp digit counts, then (once every element knows its place) the
  // tile's keys and values in digit order, so that the writes of a digit's
  // run go out as consecutive addresses
  constexpr int kCountBytes = kSortWarps * R * 4;
  constexpr int kStageBytes = kSortTile * ((int)sizeof(K) + (HasVal ? 4 : 0));
  __shared__ __align__(16) unsigned char raw[kCountBytes > kStageBytes ? kCountBytes : kStageBytes];
  uint32_t(*wcnt)[R] = reinterpret_cast<uint32_t(*)[R]>(raw);
  K* skey = reinterpret_cast<K*>(raw);
  uint32_t* sval = reinterpret_cast<uint32_t*>(raw + kSortTile * sizeof(K));
  __shared__ uint32_t tbase[R];
  __shared__ uint32_t lbase[R];  // the tile's exclusive digit offsets
  __shared__ uint32_t ws[33];
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSortWarps * R; i += blockDim.x) (&wcnt[0][0])[i] = 0;
  TileInfo ti = tile_info(sg, n, blockIdx.x, R);
  const int seg = sg.tile_seg ? sg.tile_seg[blockIdx.x] : 0;
  const int64_t seg_start = sg.seg_base ? sg.seg_base[seg] : 0;
  const int64_t seg_tiles = sg.tile_seg ? sg.seg_tile0[seg + 1] - sg.seg_tile0[seg] : sg.ntiles;
  const bool single = seg_tiles == 1;  // the tile is its whole segment: bases from its own counts
  // destination of digit d in this tile: segment start + keys of the segment
  // with a smaller digit (scan of the row totals) + keys of digit d in the
  // segment's earlier tiles (row prefix)
  if (!single) {
    uint32_t v[PER];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int d = threadIdx.x * PER + j;
      v[j] = d < R ? rowtot[(int64_t)seg * R + d] : 0u;
      sum += v[j];
    }
    uint32_t ex = block_exclusive<uint32_t>(sum, ws, nullptr) + (uint32_t)seg_start;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int d = threadIdx.x * PER + j;
      if (d < R) tbase[d] = ex + offs[ti.hist_base + (int64_t)d * ti.stride];
      ex += v[j];
    }
  }
  __syncthreads();
  K key[kSortItems];
  uint32_t val[kSortItems];
  uint32_t rank[kSortItems];
  uint32_t dig[kSortItems];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    int idx = warp * (32 * kSortItems) + j * 32 + lane;
    bool valid = idx < ti.count;
    key[j] = valid ? keys[ti.start + idx] : K(0);
    if (HasVal) val[j] = valid ? vals[ti.start + idx] : 0u;
    uint32_t dg = valid ? ((uint32_t)(key[j] >> shift) & (R - 1)) : (uint32_t)R;
    dig[j] = dg;
    unsigned peers = __match_any_sync(0xffffffffu, dg);
    uint32_t before = __popc(peers & lt);
    uint32_t base = valid ? wcnt[warp][dg] : 0u;
    rank[j] = base + before;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][dg] = base + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int dg = threadIdx.x; dg < R; dg += blockDim.x) {
    uint32_t run = 0;
    for (int w = 0; w < kSortWarps; ++w) {
      uint32_t c = wcnt[w][dg];
      wcnt[w][dg] = run;
      run += c;
    }
    lbase[dg] = run;  // the tile's count of digit dg
  }
  __syncthreads();
  {  // exclusive scan of the tile's digit counts
    uint32_t v[PER];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int d = threadIdx.x * PER + j;
      v[j] = d < R ? lbase[d] : 0u;
      sum += v[j];
    }
    uint32_t ex = block_exclusive<uint32_t>(sum, ws, nullptr);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int d = threadIdx.x * PER + j;
      if (d < R) {
        lbase[d] = ex;
        if (single) tbase[d] = ex + (uint32_t)seg_start;
      }
      ex += v[j];
    }
  }
  __syncthreads();
  // place of every element in the tile's digit order (stable: within a digit,
  // by warp, then item, then lane, i.e. input order)
  uint32_t lpos[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; ++j)
    lpos[j] = dig[j] < (uint32_t)R ? lbase[dig[j]] + wcnt[warp][dig[j]] + rank[j] : 0u;
  __syncthreads();  // wcnt is overwritten by the staged tile from here on
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    if (dig[j] >= (uint32_t)R) continue;
    skey[lpos[j]] = key[j];
    if (HasVal) sval[lpos[j]] = val[j];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ti.count; e += blockDim.x) {
    const K k = skey[e];
    const uint32_t d = (uint32_t)(k >> shift) & (R - 1);
    const uint32_t dst = tbase[d] + ((uint32_t)e - lbase[d]);
    keys_out[dst] = k;
    if (HasVal) vals_out[dst] = sval[e];
  }
}

// Whole sort of one tile that is its own segment (at most 2,048 keys), all
// passes of 8-bit digits in shared memory, by one block: the sort of the
// small levels of a layout (one launch instead of three per pass).  Ranks
// within a digit follow the input order exactly as in radix_scatter_kernel.
__global__ void __launch_bounds__(kSortThreads) radix_tile_sort_kernel(const uint32_t* __restrict__ keys,
                                                                       const uint32_t* __restrict__ vals,
                                                                       uint32_t* __restrict__ keys_out,
                                                                       uint32_t* __restrict__ vals_out, int64_t n,
                                                                       int bits, SortSegments sg) {
  pdl_wait();
  __shared__ TileSortSmem sm;
  const TileInfo ti = tile_info(sg, n, blockIdx.x, 256);
  for (int i = threadIdx.x; i < ti.count; i += blockDim.x) {
    sm.key[0][i] = keys[ti.start + i];
    sm.val[0][i] = vals[ti.start + i];
  }
  const int cur = tile_sort_smem(sm, ti.count, bits);
  for (int i = threadIdx.x; i < ti.count; i += blockDim.x) {
    keys_out[ti.start + i] = sm.key[cur][i];
    vals_out[ti.start + i] = sm.val[cur][i];
  }
}

inline int digit_bits(int bits, int* passes) {
  const int maxb = std::min(kMaxRadixBits, std::max(8, g_tuning.radix_max_bits.load(std::memory_order_relaxed)));
  const int p = (bits + maxb - 1) / maxb;
  const int need = (bits + p - 1) / p;
  *passes = p;
  return need <= 6 ? 6 : need <= 8 ? 8 : need <= 9 ? 9 : 10;
}

template <class K, int BITS>
void radix_pass(const K* ka, const uint32_t* va, K* kb, uint32_t* vb, int64_t n, int shift, const SortSegments& sg,
                uint32_t* hist, uint32_t* rowtot, cudaStream_t s) {
  constexpr int R = 1 << BITS;
  const int64_t nrows = (int64_t)(sg.tile_seg ? sg.nseg : 1) * R;
  launch(radix_hist_kernel<K, BITS>, (unsigned)sg.ntiles, 256, 0, s, ka, n, shift, sg, hist);
  const int64_t nlong = sg.tile_seg ? sg.nlong : (sg.ntiles > kLongSegTiles ? 1 : 0);
  if (nlong > 0)
    launch(radix_rowscan_warp, (unsigned)((nlong * R * 32 + 255) / 256), 256, 0, s, hist, sg, R, nlong * R, rowtot);
  if (sg.tile_seg ? sg.nmid > 0 : (sg.ntiles > 1 && nlong == 0))
    launch(radix_rowscan, (unsigned)((nrows + 255) / 256), 256, 0, s, hist, sg, R, nrows, rowtot);
  if (va)
    launch(radix_scatter_kernel<K, true, BITS>, (unsigned)sg.ntiles, kSortThreads, 0, s, ka, va, kb, vb, n, shift, sg,
           hist, rowtot);
  else
    launch(radix_scatter_kernel<K, false, BITS>, (unsigned)sg.ntiles, kSortThreads, 0, s, ka, nullptr, kb, nullptr, n,
           shift, sg, hist, rowtot);
}

template <class K>
vmo_status radix_sort_impl(K* keys_in, uint32_t* vals_in, K* keys_out, uint32_t* vals_out, int64_t n, int bits,
                           const SortSegments* segs, cudaStream_t s, Scratch& sc, bool* in_b = nullptr) {
  if (in_b) *in_b = false;
  if (n <= 0) return VMO_OK;
  SortSegments sg;
  if (segs) sg = *segs;
  if (sg.tile_seg == nullptr) sg.ntiles = (n + kSortTile - 1) / kSortTile;
  int passes = 0;
  const int B = bits > 0 ? digit_bits(bits, &passes) : 8;
  if (passes == 0) {
    if (in_b) return VMO_OK;  // already sorted, left in place
    VMO_CUDA(cudaMemcpyAsync(keys_out, keys_in, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
    if (vals_in) VMO_CUDA(cudaMemcpyAsync(vals_out, vals_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    return VMO_OK;
  }
  if constexpr (std::is_same<K, uint32_t>::value) {
    // every segment one tile: the whole sort of each tile in one block
    const bool one_tile = sg.tile_seg ? (sg.nlong == 0 && sg.nmid == 0) : (sg.ntiles == 1);
    if (one_tile && vals_in && bits <= 32) {
      launch(radix_tile_sort_kernel, (unsigned)sg.ntiles, kSortThreads, 0, s, keys_in, vals_in, keys_out, vals_out, n,
             bits, sg);
      VMO_LAUNCHED("radix_tile_sort");
      if (in_b) *in_b = true;
      return VMO_OK;
    }
  }
  uint32_t *hist, *rowtot;
  VMO_TRY(sc.alloc(&hist, (size_t)(sg.ntiles << B)));
  VMO_TRY(sc.alloc(&rowtot, (size_t)(sg.tile_seg ? sg.nseg : 1) << B));
  K* ka = keys_in;
  K* kb = keys_out;
  uint32_t* va = vals_in;
  uint32_t* vb = vals_out;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * B;
    switch (B) {
      case 6: radix_pass<K, 6>(ka, va, kb, vb, n, shift, sg, hist, rowtot, s); break;
      case 8: radix_pass<K, 8>(ka, va, kb, vb, n, shift, sg, hist, rowtot, s); break;
      case 9: radix_pass<K, 9>(ka, va, kb, vb, n, shift, sg, hist, rowtot, s); break;
      default: radix_pass<K, 10>(ka, va, kb, vb, n, shift, sg, hist, rowtot, s); break;
    }
    VMO_LAUNCHED("radix_sort");
    K* tk = ka; ka = kb; kb = tk;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  if (in_b) {
    *in_b = ka == keys_out;
    return VMO_OK;
  }
  if (ka != keys_out) {
    VMO_CUDA(cudaMemcpyAsync(keys_out, ka, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
    if (vals_in) VMO_CUDA(cudaMemcpyAsync(vals_out, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
  return VMO_OK;
}

}  // namespace

template <class T>
vmo_status scan_exclusive(const T* in, T* out, int64_t n, T* total, cudaStream_t s, Scratch& sc) {
  return scan_impl<T, false>(in, out, n, total, s, sc);
}
template <class T>
vmo_status scan_inclusive(const T* in, T* out, int64_t n, cudaStream_t s, Scratch& sc) {
  return scan_impl<T, true>(in, out, n, nullptr, s, sc);
}

template vmo_status scan_exclusive<int32_t>(const int32_t*, int32_t*, int64_t, int32_t*, cudaStream_t, Scratch&);
template vmo_status scan_exclusive<int64_t>(const int64_t*, int64_t*, int64_t, int64_t*, cudaStream_t, Scratch&);
template vmo_status scan_exclusive<uint32_t>(const uint32_t*, uint32_t*, int64_t, uint32_t*, cudaStream_t,
                                             Scratch&);
template vmo_status scan_exclusive<uint64_t>(const uint64_t*, uint64_t*, int64_t, uint64_t*, cudaStream_t,
                                             Scratch&);
template vmo_status scan_inclusive<uint64_t>(const uint64_t*, uint64_t*, int64_t, cudaStream_t, Scratch&);
template vmo_status scan_inclusive<int32_t>(const int32_t*, int32_t*, int64_t, cudaStream_t, Scratch&);
template vmo_status scan_inclusive<int64_t>(const int64_t*, int64_t*, int64_t, cudaStream_t, Scratch&);

vmo_status scan_inclusive_u64_into(const uint64_t* in, uint64_t* out, int64_t n, uint64_t* partial, cudaStream_t s) {
  if (n <= 0) return VMO_OK;
  int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  launch(scan_reduce_kernel<uint64_t>, (unsigned)ntiles, kScanThreads, 0, s, in, n, partial);
  launch(scan_partials_kernel<uint64_t>, 1, 1024, 0, s, partial, ntiles, (uint64_t*)nullptr);
  launch(scan_tile_kernel<uint64_t, true>, (unsigned)ntiles, kScanThreads, 0, s, in, out, n, partial);
  VMO_LAUNCHED("scan");
  return VMO_OK;
}

int64_t scan_partials_needed(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

vmo_status radix_sort_u32(uint32_t* keys_in, uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out, int64_t n,
                          int bits, const SortSegments* segs, cudaStream_t s, Scratch& sc) {
  return radix_sort_impl<uint32_t>(keys_in, vals_in, keys_out, vals_out, n, bits, segs, s, sc);
}

vmo_status radix_sort_u32_pingpong(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b, int64_t n,
                                  int bits, const SortSegments* segs, bool* in_b, cudaStream_t s, Scratch& sc) {
  return radix_sort_impl<uint32_t>(keys_a, vals_a, keys_b, vals_b, n, bits, segs, s, sc, in_b);
}

vmo_status radix_sort_u64(uint64_t* keys_in, uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out, int64_t n,
                          int bits, cudaStream_t s, Scratch& sc) {
  return radix_sort_impl<uint64_t>(keys_in, vals_in, keys_out, vals_out, n, bits, nullptr, s, sc);
}

vmo_status make_sort_segments(const std::vector<int64_t>& base, SortSegments* out, cudaStream_t s, Scratch& sc) {
  int32_t nseg = (int32_t)base.size() - 1;
  std::vector<int32_t> tseg, tcount, t0(nseg + 1);
  std::vector<int64_t> tstart;
  for (int32_t g = 0; g < nseg; ++g) {
    t0[g] = (int32_t)tseg.size();
    int64_t a = base[g], b = base[g + 1];
    for (int64_t x = a; x < b; x += kSortTile) {
      tseg.push_back(g);
      tstart.push_back(x);
      tcount.push_back((int32_t)std::min<int64_t>(kSortTile, b - x));
    }
  }
  t0[nseg] = (int32_t)tseg.size();
  int64_t nt = (int64_t)tseg.size();
  if (nt == 0) {  // all segments empty: one empty tile keeps the kernels well-formed
    tseg.push_back(0); tstart.push_back(0); tcount.push_back(0);
    t0[nseg] = 1;
    for (int32_t g = 1; g < nseg; ++g) t0[g] = 1;
    nt = 1;
  }
  int32_t *d_tseg, *d_tcount, *d_t0;
  int64_t *d_tstart, *d_base;
  VMO_TRY(sc.alloc(&d_tseg, nt));
  VMO_TRY(sc.alloc(&d_tcount, nt));
  VMO_TRY(sc.alloc(&d_tstart, nt));
  VMO_TRY(sc.alloc(&d_t0, nseg + 1));
  VMO_TRY(sc.alloc(&d_base, nseg + 1));
  VMO_CUDA(cudaMemcpyAsync(d_tseg, tseg.data(), nt * 4, cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(d_tcount, tcount.data(), nt * 4, cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(d_tstart, tstart.data(), nt * 8, cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(d_t0, t0.data(), (nseg + 1) * 4, cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(d_base, base.data(), (nseg + 1) * 8, cudaMemcpyHostToDevice, s));
  // host vectors must outlive the asynchronous copies
  VMO_CUDA(cudaStreamSynchronize(s));
  out->nseg = nseg;
  out->seg_base = d_base;
  out->tile_seg = d_tseg;
  out->tile_start = d_tstart;
  out->tile_count = d_tcount;
  out->seg_tile0 = d_t0;
  out->ntiles = nt;
  std::vector<int32_t> lg;
  int32_t nmid = 0;
  for (int32_t g = 0; g < nseg; ++g) {
    const int32_t tiles = t0[g + 1] - t0[g];
    if (tiles > kLongSegTiles) lg.push_back(g);
    else if (tiles > 1) ++nmid;
  }
  out->nlong = (int32_t)lg.size();
  out->nmid = nmid;
  if (!lg.empty()) {
    int32_t* d_lg;
    VMO_TRY(sc.alloc(&d_lg, lg.size()));
    VMO_CUDA(cudaMemcpyAsync(d_lg, lg.data(), lg.size() * 4, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaStreamSynchronize(s));  // lg must outlive the copy
    out->long_seg = d_lg;
  }
  return VMO_OK;
}

}  // namespace vmo
