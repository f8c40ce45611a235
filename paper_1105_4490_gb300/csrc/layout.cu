// Geometry (Sec. 2): steepest descent on the energy of eq. graphenergysimple
// (Algorithm 4) inside the multilevel scheme of Algorithm 3.
//
// One step of a level, for every problem of a batch at once:
//   keys      cell of every point on a uniform grid over the bounding cube
//             (fp32, no FMA), row-major key of the finest cell
//   sort      stable segmented radix sort of (key, vertex)
//   gather    points copied in key order; first point of every finest cell
//             recorded in a dense table
//   aggregate per cell weight and weighted mean: finest cells from their
//             points, coarser cells from their 2^d children (fixed order)
//   attract   y_n = sum_j c_j (x_n - z_j) (2-pin nets: c/2 (x_n - x_u))
//   repulse   near field exactly over the 3^d adjacent finest cells, far field
//             from the cells whose parent is adjacent to the target's parent
//             but which are not adjacent themselves; then the step
//             x_n <- x_n - s_t y_n / ||y_n|| and the next bounding box.
#include <algorithm>
#include <cmath>

#include "blocksort.cuh"
#include "layout.cuh"

namespace vmo {

namespace {

constexpr int kBlock = 256;

__host__ __device__ inline int64_t lvl_off(int d, int l) {
  // sum_{j<l} 2^(d j) = (2^(d l) - 1) / (2^d - 1)
  return ((int64_t(1) << (d * l)) - 1) / ((int64_t(1) << d) - 1);
}

__device__ inline int find_problem(const int64_t* __restrict__ base, int P, int64_t i) {
  int lo = 0, hi = P;  // base[lo] <= i < base[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (base[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// Paired source tables.  The far field and the near field read their sources
// two at a time: sources 2j and 2j+1 share a pair of float4 (three for d = 4)
// holding each coordinate of both side by side, then both weights:
//   d <= 3: (x0, x1, y0, y1), (z0, z1, w0, w1)     (d = 2: z unused)
//   d = 4:  (x0, x1, y0, y1), (z0, z1, u0, u1), (w0, w1, -, -)
// so that one packed fp32x2 instruction (Blackwell f32x2 add / mul / fma)
// computes the same step for both sources.
template <int D>
struct Pair {
  static constexpr int N = D == 4 ? 3 : 2;  // float4 per pair
  static constexpr int WQ = D == 4 ? 2 : 1; // float4 holding the weights
  static constexpr int WO = D == 4 ? 0 : 2; // float offset of the weights in it
};

template <int D>
__device__ __forceinline__ void pair_store(float4* __restrict__ tab, int64_t i, const float* c, float w) {
  float* f = reinterpret_cast<float*>(tab + (i >> 1) * Pair<D>::N);
  const int h = (int)(i & 1);
#pragma unroll
  for (int m = 0; m < D; ++m) f[4 * (m >> 1) + 2 * (m & 1) + h] = c[m];
  f[4 * Pair<D>::WQ + Pair<D>::WO + h] = w;
}

template <int D>
__device__ inline void cell_of(const float4& v, const float* lo, float s, int L, int32_t* c) {
  const int32_t cmax = (1 << L) - 1;
#pragma unroll
  for (int m = 0; m < D; ++m) {
    float t = __fmul_rn(__fsub_rn(comp(v, m), lo[m]), s);
    int32_t q = (int32_t)floorf(t);
    c[m] = q < cmax ? q : cmax;
  }
}

template <int D>
__device__ inline void grid_frame(const uint32_t* __restrict__ bb, int pb, int L, float* lo, float* s) {
  float E = 0.0f;
#pragma unroll
  for (int m = 0; m < D; ++m) {
    lo[m] = ord2f(bb[pb * 8 + m]);
    float hi = ord2f(bb[pb * 8 + 4 + m]);
    float e = __fsub_rn(hi, lo[m]);
    E = e > E ? e : E;
  }
  *s = (E > 0.0f) ? __fdiv_rn((float)(1 << L), E) : 0.0f;
}

template <int D>
__device__ inline int64_t rowmajor(const int32_t* c, int side) {
  int64_t r = 0;
#pragma unroll
  for (int m = D - 1; m >= 0; --m) r = r * side + c[m];
  return r;
}

__host__ __device__ constexpr int field_bits(int D) { return D == 4 ? 8 : 30 / D; }

// Block-level bounding-box accumulation into ordered-uint min/max slots.
// uniform: every valid thread of the block belongs to problem pblock (the
// block result is then published once for pblock); otherwise each valid
// thread publishes its own point for its own problem pb.
template <int D>
__device__ void bbox_accumulate(const float4& v, bool valid, int pb, bool uniform, int pblock,
                                uint32_t* __restrict__ bb) {
  __shared__ uint32_t smn[kBlock / 32][4], smx[kBlock / 32][4];
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  if (!uniform) {
    if (valid)
#pragma unroll
      for (int m = 0; m < D; ++m) {
        uint32_t o = f2ord(comp(v, m));
        atomicMin(&bb[pb * 8 + m], o);
        atomicMax(&bb[pb * 8 + 4 + m], o);
      }
    return;
  }
#pragma unroll
  for (int m = 0; m < D; ++m) {
    uint32_t mn = valid ? f2ord(comp(v, m)) : 0xFFFFFFFFu;
    uint32_t mx = valid ? mn : 0u;
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) { smn[warp][m] = mn; smx[warp][m] = mx; }
  }
  __syncthreads();
  if (threadIdx.x < D) {
    uint32_t mn = 0xFFFFFFFFu, mx = 0u;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      mn = min(mn, smn[w][threadIdx.x]);
      mx = max(mx, smx[w][threadIdx.x]);
    }
    if (mn != 0xFFFFFFFFu) atomicMin(&bb[pblock * 8 + threadIdx.x], mn);
    if (mx != 0u) atomicMax(&bb[pblock * 8 + 4 + threadIdx.x], mx);
  }
}

__global__ void k_bbox_reset(uint32_t* bb, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) bb[i] = ((i & 7) < 4) ? 0xFFFFFFFFu : 0u;
}

template <int D>
__global__ void __launch_bounds__(kBlock) k_bbox(const float4* __restrict__ x, int64_t K,
                                                 const int32_t* __restrict__ vprob, uint32_t* __restrict__ bb) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t first = (int64_t)blockIdx.x * blockDim.x;
  int64_t last = min(first + (int64_t)blockDim.x, K) - 1;
  const int pblock = vprob[first];
  bool uniform = pblock == vprob[last];
  bool valid = i < K;
  float4 v = valid ? x[i] : make_float4(0, 0, 0, 0);
  int pb = valid ? vprob[i] : 0;
  bbox_accumulate<D>(v, valid, pb, uniform, pblock, bb);
}

// Step length of a level: s0 = sigma * Lbox / k^(1/d), Lbox = d-th root of the
// box volume (largest extent if an extent is zero).
template <int D>
__global__ void k_step0(const uint32_t* __restrict__ bb, const ProbDev* __restrict__ prob, int P, float sigma,
                        float* __restrict__ s0) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double vol = 1.0, emax = 0.0;
  bool degenerate = false;
  for (int m = 0; m < D; ++m) {
    double e = (double)ord2f(bb[p * 8 + 4 + m]) - (double)ord2f(bb[p * 8 + m]);
    if (!(e > 0.0)) degenerate = true;
    emax = e > emax ? e : emax;
    vol *= e;
  }
  int k = prob[p].k;
  double Lbox = degenerate ? emax : pow(vol, 1.0 / D);
  s0[p] = (k > 0) ? (float)(sigma * Lbox / pow((double)k, 1.0 / D)) : 0.0f;
}

// Cell keys of the points.  Each thread takes U points, strided by the block
// so that every load is coalesced, and issues all their loads before the
// arithmetic (U = 4 on large levels: more bytes in flight per SM; U = 1 on
// small ones: more blocks); thread 0 advances the level's step counter and
// the grid resets the next bounding boxes.
constexpr int64_t kKeyItemsMin = int64_t(1) << 20;  // points of a level that take 4 per thread

template <int D, int U>
__global__ void __launch_bounds__(kBlock) k_keys(const float4* __restrict__ x, int64_t K, const int32_t* __restrict__ vprob,
                                                 const ProbDev* __restrict__ prob, const uint32_t* __restrict__ bb,
                                                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                 uint32_t* __restrict__ bb_next, int nreset, int32_t* __restrict__ tctr) {
  pdl_wait();
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gt == 0) ++*tctr;  // the level's step (read by the step kernel of this step)
  for (int64_t r = gt; r < nreset; r += (int64_t)gridDim.x * blockDim.x) bb_next[r] = ((r & 7) < 4) ? 0xFFFFFFFFu : 0u;
  const int64_t v0 = (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x;
  float4 xv[U];
  int pb[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t v = v0 + (int64_t)u * blockDim.x;
    xv[u] = v < K ? x[v] : make_float4(0.f, 0.f, 0.f, 0.f);
    pb[u] = v < K ? vprob[v] : 0;
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t v = v0 + (int64_t)u * blockDim.x;
    if (v >= K) break;
    const int L = prob[pb[u]].L;
    float lo[D], s;
    grid_frame<D>(bb, pb[u], L, lo, &s);
    int32_t c[D];
    cell_of<D>(xv[u], lo, s, L, c);
    keys[v] = (uint32_t)rowmajor<D>(c, 1 << L);
    vals[v] = (uint32_t)v;
  }
}

// a[lo..hi) = v, with 16-byte stores over the aligned middle of the range
// (long runs of empty cells between clusters of the layout).
__device__ inline void fill_i32(int32_t* __restrict__ a, int64_t lo, int64_t hi, int32_t v) {
  while (lo < hi && (((uintptr_t)(a + lo)) & 15u)) a[lo++] = v;
  const int4 v4 = make_int4(v, v, v, v);
  for (; lo + 4 <= hi; lo += 4) *reinterpret_cast<int4*>(a + lo) = v4;
  while (lo < hi) a[lo++] = v;
}

// Sorted positions: coordinates and weights in sorted order (plain and in
// the paired table XP), the packed cell of every point, and the cell start
// table.  cst[fbase + pb + c] is the first
// sorted position of problem pb whose key is >= c (so empty cells get the
// start of the next occupied one and a row of cells is one contiguous range),
// with one extra entry per problem holding its end.  Every position writes the
// entries of the cells between its predecessor's key and its own; the last
// position of a problem also writes the cells after its key and the end entry.
template <int D>
__global__ void __launch_bounds__(kBlock) k_gather(const uint32_t* __restrict__ svals,
                                                   const uint32_t* __restrict__ skeys, int64_t K,
                                                   const float4* __restrict__ x, const float* __restrict__ w,
                                                   const int32_t* __restrict__ vprob, const ProbDev* __restrict__ prob,
                                                   const uint32_t* __restrict__ bb, float4* __restrict__ xs,
                                                   float* __restrict__ ws, uint32_t* __restrict__ scell,
                                                   int32_t* __restrict__ cst, float4* __restrict__ XP) {
  pdl_wait();
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= K) return;
  uint32_t v = svals[p];
  int pb = vprob[p];
  ProbDev pr = prob[pb];
  float4 xv = x[v];
  xs[p] = xv;
  const float wv = w ? w[v] : 1.0f;
  if (ws) ws[p] = wv;
  // paired table: the problem's points start at an even slot, so the pairing
  // of its points does not depend on where the problem sits in the batch
  const int64_t e = (pr.vbase + pb + 1) & ~int64_t(1);
  const float xc[4] = {xv.x, xv.y, xv.z, xv.w};
  pair_store<D>(XP, e + (p - pr.vbase), xc, wv);
  if (p == pr.vbase + pr.k - 1 && (pr.k & 1)) {  // unused half of the last pair: finite, weight 0
    const float zero[4] = {0.f, 0.f, 0.f, 0.f};
    pair_store<D>(XP, e + pr.k, zero, 0.0f);
  }
  float lo[D], s;
  grid_frame<D>(bb, pb, pr.L, lo, &s);
  int32_t c[D];
  cell_of<D>(xv, lo, s, pr.L, c);
  uint32_t packed = 0;
#pragma unroll
  for (int m = 0; m < D; ++m) packed |= (uint32_t)c[m] << (m * field_bits(D));
  scell[p] = packed;
  int32_t* cs = cst + pr.fbase + pb;
  const int64_t key = skeys[p];
  const int64_t prev = p == pr.vbase ? -1 : (int64_t)skeys[p - 1];
  fill_i32(cs, prev + 1, key + 1, (int32_t)p);
  if (p == pr.vbase + pr.k - 1) fill_i32(cs, key + 1, (int64_t(1) << (D * pr.L)) + 1, (int32_t)(pr.vbase + pr.k));
}

// Cell sums (St, Wt) at cell index idx, and the cell's charge (weighted mean
// and weight) at index pidx of the paired cell table.
template <int D>
__device__ inline void store_cell(int64_t idx, int64_t pidx, const float* S, float W, float4* __restrict__ St,
                                  float* __restrict__ Wt, float4* __restrict__ CP) {
  St[idx] = make_float4(S[0], D > 1 ? S[1] : 0.f, D > 2 ? S[2] : 0.f, D > 3 ? S[3] : 0.f);
  Wt[idx] = W;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  if (W > 0.0f) {
    float iw = 1.0f / W;
#pragma unroll
    for (int m = 0; m < D; ++m) c[m] = S[m] * iw;
  }
  pair_store<D>(CP, pidx, c, W);
}

// Finest cells: the charge of every cell from its points (the range comes
// from the cell start table written by k_gather; a problem without points
// writes its table here).  A cell of at most kCellSerial points is summed by
// its own thread in point order; a larger cell (dense clusters of the layout)
// by the whole warp: lane-strided partial sums from the cell's first point,
// then a fixed xor tree.  Either way the sums depend only on the cell.
constexpr int kCellSerial = 32;

template <int D>
__device__ __forceinline__ void cell_add(const float4& p, float wq, float* S, float& W) {
  S[0] += wq * p.x;
  if (D > 1) S[1] += wq * p.y;
  if (D > 2) S[2] += wq * p.z;
  if (D > 3) S[3] += wq * p.w;
  W += wq;
}

// Points q0, q0 + stride, ... < q1 added in that order; four loads issued
// before their additions.
template <int D>
__device__ __forceinline__ void cell_sum(const float4* xs, const float* ws, int64_t q0, int64_t q1, int64_t stride,
                                         float* S, float& W) {
  int64_t q = q0;
  for (; q + 3 * stride < q1; q += 4 * stride) {
    float4 p[4];
    float wq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      p[u] = xs[q + u * stride];
      wq[u] = ws ? ws[q + u * stride] : 1.0f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) cell_add<D>(p[u], wq[u], S, W);
  }
  for (; q < q1; q += stride) cell_add<D>(xs[q], ws ? ws[q] : 1.0f, S, W);
}

template <int D>
__global__ void __launch_bounds__(kBlock) k_agg_finest(int64_t ncells, const int64_t* __restrict__ fbase, int P,
                                                       const ProbDev* __restrict__ prob, const float4* __restrict__ xs,
                                                       const float* __restrict__ ws, int32_t* __restrict__ cst,
                                                       float4* __restrict__ St, float* __restrict__ Wt,
                                                       float4* __restrict__ CP) {
  pdl_wait();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < ncells;
  int64_t q0 = 0, q1 = 0, idx = 0, pidx = 0;
  if (valid) {
    const int pb = find_problem(fbase, P, i);
    const ProbDev pr = prob[pb];
    const int64_t c = i - pr.fbase;
    int32_t* cs = cst + pr.fbase + pb;
    if (pr.k == 0) {
      cs[c] = (int32_t)pr.vbase;
      if (c == (int64_t(1) << (D * pr.L)) - 1) cs[c + 1] = (int32_t)pr.vbase;
    } else {
      q0 = cs[c];
      q1 = cs[c + 1];
    }
    idx = pr.cbase + lvl_off(D, pr.L) + c;
    pidx = idx + pb + 1;
  }
  const bool big = valid && q1 - q0 > kCellSerial;
  if (valid && !big) {
    float S[4] = {0.f, 0.f, 0.f, 0.f};
    float W = 0.f;
    cell_sum<D>(xs, ws, q0, q1, 1, S, W);
    store_cell<D>(idx, pidx, S, W, St, Wt, CP);
  }
  const int lane = lane_id();
  unsigned todo = __ballot_sync(0xffffffffu, big);
  while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1;
    const int64_t b0 = __shfl_sync(0xffffffffu, q0, src), b1 = __shfl_sync(0xffffffffu, q1, src);
    float S[4] = {0.f, 0.f, 0.f, 0.f};
    float W = 0.f;
    cell_sum<D>(xs, ws, b0 + lane, b1, 32, S, W);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int m = 0; m < D; ++m) S[m] += __shfl_xor_sync(0xffffffffu, S[m], o);
      W += __shfl_xor_sync(0xffffffffu, W, o);
    }
    if (lane == src) store_cell<D>(idx, pidx, S, W, St, Wt, CP);
  }
}

// Coarse cells: sums of the 2^d children (fixed order), charge at the mean.
template <int D>
__device__ inline void agg_cell(const ProbDev& pr, int pb, int l, int64_t c, float4* __restrict__ St,
                                float* __restrict__ Wt, float4* __restrict__ CP) {
  const int side = 1 << l;
  int32_t cc[D];
  int64_t rem = c;
#pragma unroll
  for (int m = 0; m < D; ++m) {
    cc[m] = (int32_t)(rem % side);
    rem /= side;
  }
  const int64_t child_base = pr.cbase + lvl_off(D, l + 1);
  float S[4] = {0.f, 0.f, 0.f, 0.f};
  float W = 0.f;
#pragma unroll
  for (int ch = 0; ch < (1 << D); ++ch) {
    int32_t q[D];
#pragma unroll
    for (int m = 0; m < D; ++m) q[m] = 2 * cc[m] + ((ch >> m) & 1);
    const int64_t idx = child_base + rowmajor<D>(q, 2 * side);
    const float4 s4 = St[idx];
    S[0] += s4.x;
    if (D > 1) S[1] += s4.y;
    if (D > 2) S[2] += s4.z;
    if (D > 3) S[3] += s4.w;
    W += Wt[idx];
  }
  const int64_t idx = pr.cbase + lvl_off(D, l) + c;
  store_cell<D>(idx, idx + pb + 1, S, W, St, Wt, CP);
}

// Levels of at most 512 cells are aggregated by one block per problem (all of
// them in one launch, a block barrier between levels); the larger coarse
// levels by one launch per level over all problems.
__host__ __device__ constexpr int small_level_max(int d) { return d == 2 ? 4 : (d == 3 ? 3 : 2); }

template <int D>
__global__ void __launch_bounds__(kBlock) k_agg_level(int step, const int64_t* __restrict__ off, int P, int64_t ncells,
                                                      const ProbDev* __restrict__ prob, float4* __restrict__ St,
                                                      float* __restrict__ Wt, float4* __restrict__ CP) {
  pdl_wait();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncells) return;
  int pb = find_problem(off, P, i);
  ProbDev pr = prob[pb];
  agg_cell<D>(pr, pb, pr.L - step, i - off[pb], St, Wt, CP);
}

template <int D>
__global__ void __launch_bounds__(kBlock) k_agg_small(const ProbDev* __restrict__ prob, float4* __restrict__ St,
                                                      float* __restrict__ Wt, float4* __restrict__ CP) {
  pdl_wait();
  const int pb = blockIdx.x;
  const ProbDev pr = prob[pb];
  for (int l = min(pr.L - 1, small_level_max(D)); l >= 2; --l) {
    const int64_t n = int64_t(1) << (D * l);
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) agg_cell<D>(pr, pb, l, c, St, Wt, CP);
    __syncthreads();
  }
}

// One-block binning of a step for levels whose problems all have at most
// kSortTile points and kBinCells finest cells: one block per problem stages
// its points in shared memory, computes the keys (as k_keys), sorts (key,
// local index) stably in shared memory (as the one-tile radix sort), gathers
// (as k_gather, and writes the sorted vertex ids), sums the finest cells from
// the staged points (as k_agg_finest: serially up to kCellSerial points, else
// lane-strided with the xor tree) and every coarser level (agg_cell, a block
// barrier between levels).  The arithmetic and the order of every sum are
// those kernels', so the results are bit-identical, from one launch instead
// of five or more.  The cell charges are read back by other threads of the
// block after a barrier, so those pointers carry no __restrict__.  keys
// (optional): the unsorted keys by vertex, as k_keys writes them.
constexpr int kBinCells = 4096;

struct BinSmem {
  float4 xin[kSortTile];      // the problem's points by local index
  float win[kSortTile];       // their weights (1 without weights)
  int32_t cs[kBinCells + 1];  // cell start table (sorted positions)
  TileSortSmem sort;
};

template <int D>
__global__ void __launch_bounds__(kSortThreads) k_bin_small(
    const float4* __restrict__ x, const float* __restrict__ w, const ProbDev* __restrict__ prob,
    const uint32_t* __restrict__ bb, uint32_t* __restrict__ bb_next, int32_t* __restrict__ tctr,
    uint32_t* __restrict__ keys, uint32_t* __restrict__ svals, float4* __restrict__ xs, float* __restrict__ ws,
    uint32_t* __restrict__ scell, int32_t* __restrict__ cst, float4* __restrict__ XP, float4* St, float* Wt,
    float4* CP) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char bin_raw[];
  BinSmem& sm = *reinterpret_cast<BinSmem*>(bin_raw);
  const int pb = blockIdx.x;
  const ProbDev pr = prob[pb];
  const int k = pr.k;
  const int64_t vb = pr.vbase;
  if (pb == 0 && threadIdx.x == 0) ++*tctr;  // the level's step
  if (threadIdx.x < 8) bb_next[pb * 8 + threadIdx.x] = threadIdx.x < 4 ? 0xFFFFFFFFu : 0u;
  float lo[D], s;
  grid_frame<D>(bb, pb, pr.L, lo, &s);
  {
    // points, weights and keys by local index; a thread's loads issued first
    float4 xv[kSortItems];
    float wv[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const int i = threadIdx.x + j * kSortThreads;
      xv[j] = i < k ? x[vb + i] : make_float4(0.f, 0.f, 0.f, 0.f);
      wv[j] = (i < k && w) ? w[vb + i] : 1.0f;
    }
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const int i = threadIdx.x + j * kSortThreads;
      if (i < k) {
        sm.xin[i] = xv[j];
        sm.win[i] = wv[j];
        int32_t c[D];
        cell_of<D>(xv[j], lo, s, pr.L, c);
        const uint32_t key = (uint32_t)rowmajor<D>(c, 1 << pr.L);
        sm.sort.key[0][i] = key;
        sm.sort.val[0][i] = (uint32_t)i;
        if (keys) keys[vb + i] = key;
      }
    }
  }
  const int cur = tile_sort_smem(sm.sort, k, D * pr.L);
  const uint32_t* skey = sm.sort.key[cur];
  const uint32_t* sloc = sm.sort.val[cur];
  // gather and cell start table (global for the step kernel, shared here)
  const int64_t ncell = int64_t(1) << (D * pr.L);
  const int64_t e = (vb + pb + 1) & ~int64_t(1);
  int32_t* cs = cst + pr.fbase + pb;
  for (int i = threadIdx.x; i < k; i += kSortThreads) {
    const int64_t p = vb + i;
    const uint32_t li = sloc[i];
    svals[p] = (uint32_t)(vb + li);
    const float4 xv = sm.xin[li];
    const float wv = sm.win[li];
    xs[p] = xv;
    if (ws) ws[p] = wv;
    const float xc[4] = {xv.x, xv.y, xv.z, xv.w};
    pair_store<D>(XP, e + i, xc, wv);
    if (i == k - 1 && (k & 1)) {
      const float zero[4] = {0.f, 0.f, 0.f, 0.f};
      pair_store<D>(XP, e + k, zero, 0.0f);
    }
    int32_t c[D];
    cell_of<D>(xv, lo, s, pr.L, c);
    uint32_t packed = 0;
#pragma unroll
    for (int m = 0; m < D; ++m) packed |= (uint32_t)c[m] << (m * field_bits(D));
    scell[p] = packed;
    const int64_t key = skey[i];
    const int64_t prev = i == 0 ? -1 : (int64_t)skey[i - 1];
    for (int64_t q = prev + 1; q <= key; ++q) sm.cs[q] = (int32_t)p;
    fill_i32(cs, prev + 1, key + 1, (int32_t)p);
    if (i == k - 1) {
      for (int64_t q = key + 1; q <= ncell; ++q) sm.cs[q] = (int32_t)(vb + k);
      fill_i32(cs, key + 1, ncell + 1, (int32_t)(vb + k));
    }
  }
  if (k == 0)
    for (int64_t c = threadIdx.x; c <= ncell; c += kSortThreads) {
      cs[c] = (int32_t)vb;
      sm.cs[c] = (int32_t)vb;
    }
  __syncthreads();
  // finest cells from the staged points, a warp per 32 consecutive cells
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  const int64_t cfin = pr.cbase + lvl_off(D, pr.L);
  for (int64_t c0 = (int64_t)warp * 32; c0 < ncell; c0 += kSortThreads) {
    const int64_t c = c0 + lane;
    const bool valid = c < ncell;
    int q0 = 0, q1 = 0;  // problem-local sorted positions
    if (valid && k > 0) {
      q0 = sm.cs[c] - (int)vb;
      q1 = sm.cs[c + 1] - (int)vb;
    }
    const int64_t idx = cfin + c, pidx = idx + pb + 1;
    const bool big = valid && q1 - q0 > kCellSerial;
    if (valid && !big) {
      float S[4] = {0.f, 0.f, 0.f, 0.f};
      float W = 0.f;
      for (int q = q0; q < q1; ++q) cell_add<D>(sm.xin[sloc[q]], sm.win[sloc[q]], S, W);
      store_cell<D>(idx, pidx, S, W, St, Wt, CP);
    }
    unsigned todo = __ballot_sync(0xffffffffu, big);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int b0 = __shfl_sync(0xffffffffu, q0, src), b1 = __shfl_sync(0xffffffffu, q1, src);
      float S[4] = {0.f, 0.f, 0.f, 0.f};
      float W = 0.f;
      for (int q = b0 + lane; q < b1; q += 32) cell_add<D>(sm.xin[sloc[q]], sm.win[sloc[q]], S, W);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int m = 0; m < D; ++m) S[m] += __shfl_xor_sync(0xffffffffu, S[m], o);
        W += __shfl_xor_sync(0xffffffffu, W, o);
      }
      if (lane == src) store_cell<D>(idx, pidx, S, W, St, Wt, CP);
    }
  }
  __syncthreads();
  // coarser levels down to 2, each from its children
  for (int l = pr.L - 1; l >= 2; --l) {
    const int64_t n = int64_t(1) << (D * l);
    for (int64_t c = threadIdx.x; c < n; c += kSortThreads) agg_cell<D>(pr, pb, l, c, St, Wt, CP);
    __syncthreads();
  }
}

// Rubber bands of 2-pin nets: y_v = sum_u c_vu (x_v - x_u) / 2.  Rows are
// split by degree: light rows (<= kLightMax) take one thread, medium rows a
// warp and heavy rows a block; each class sums in a fixed order (sequential,
// lane-strided + xor tree, thread-strided + fixed tree), so the result of a
// vertex depends only on its own row.
constexpr int kLightMax = 32;
constexpr int kWarpMax = 4096;

__device__ inline void add_pull(float* a, const float4& xv, const float4& xu, float c) {
  a[0] += c * (xv.x - xu.x);
  a[1] += c * (xv.y - xu.y);
  a[2] += c * (xv.z - xu.z);
  a[3] += c * (xv.w - xu.w);
}

// a += sum over t = t0, t0 + stride, ... < t1 of c_t (xv - x[adj[t]]), in that
// order; four neighbours per trip with all their loads issued first.
__device__ __forceinline__ void pull_range(float* a, const float4& xv, const int32_t* __restrict__ adj,
                                           const float* __restrict__ acost, const float4* __restrict__ x, int32_t t,
                                           int32_t t1, int32_t stride) {
  constexpr int U = 4;
  for (; t + (U - 1) * stride < t1; t += U * stride) {
    int32_t u[U];
    float c[U];
    float4 q[U];
#pragma unroll
    for (int i = 0; i < U; ++i) {
      u[i] = adj[t + i * stride];
      c[i] = acost ? acost[t + i * stride] : 1.0f;
    }
#pragma unroll
    for (int i = 0; i < U; ++i) q[i] = x[u[i]];
#pragma unroll
    for (int i = 0; i < U; ++i) add_pull(a, xv, q[i], c[i]);
  }
  for (; t < t1; t += stride) add_pull(a, xv, x[adj[t]], acost ? acost[t] : 1.0f);
}

__global__ void __launch_bounds__(kBlock) k_attract(const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                                                    const float* __restrict__ acost, const float4* __restrict__ x,
                                                    int64_t K, float4* __restrict__ y) {
  pdl_wait();
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  int32_t t0 = adj_ptr[v], t1 = adj_ptr[v + 1];
  if (t1 - t0 > kLightMax) return;  // medium and heavy rows: k_attract_warp / k_attract_block
  float4 xv = x[v];
  float a[4] = {0.f, 0.f, 0.f, 0.f};
  pull_range(a, xv, adj, acost, x, t0, t1, 1);
  y[v] = make_float4(0.5f * a[0], 0.5f * a[1], 0.5f * a[2], 0.5f * a[3]);
}

__global__ void __launch_bounds__(kBlock) k_attract_warp(const int32_t* __restrict__ list, int64_t n,
                                                         const int32_t* __restrict__ adj_ptr,
                                                         const int32_t* __restrict__ adj, const float* __restrict__ acost,
                                                         const float4* __restrict__ x, float4* __restrict__ y) {
  pdl_wait();
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;
  const int lane = lane_id();
  int32_t v = list[w];
  float4 xv = x[v];
  float a[4] = {0.f, 0.f, 0.f, 0.f};
  pull_range(a, xv, adj, acost, x, adj_ptr[v] + lane, adj_ptr[v + 1], 32);
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[m] += __shfl_xor_sync(0xffffffffu, a[m], o);
  if (lane == 0) y[v] = make_float4(0.5f * a[0], 0.5f * a[1], 0.5f * a[2], 0.5f * a[3]);
}

__global__ void __launch_bounds__(kBlock) k_attract_block(const int32_t* __restrict__ list,
                                                          const int32_t* __restrict__ adj_ptr,
                                                          const int32_t* __restrict__ adj,
                                                          const float* __restrict__ acost,
                                                          const float4* __restrict__ x, float4* __restrict__ y) {
  pdl_wait();
  __shared__ float part[kBlock / 32][4];
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  int32_t v = list[blockIdx.x];
  float4 xv = x[v];
  float a[4] = {0.f, 0.f, 0.f, 0.f};
  pull_range(a, xv, adj, acost, x, adj_ptr[v] + threadIdx.x, adj_ptr[v + 1], blockDim.x);
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[m] += __shfl_xor_sync(0xffffffffu, a[m], o);
  if (lane == 0)
    for (int m = 0; m < 4; ++m) part[warp][m] = a[m];
  __syncthreads();
  if (threadIdx.x == 0) {
    float b[4] = {0.f, 0.f, 0.f, 0.f};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      for (int m = 0; m < 4; ++m) b[m] += part[w][m];
    y[v] = make_float4(0.5f * b[0], 0.5f * b[1], 0.5f * b[2], 0.5f * b[3]);
  }
}

__global__ void k_degree_class(const int32_t* __restrict__ adj_ptr, int64_t K, int32_t* __restrict__ mid,
                               int32_t* __restrict__ heavy) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  int32_t deg = adj_ptr[v + 1] - adj_ptr[v];
  mid[v] = (deg > kLightMax && deg <= kWarpMax) ? 1 : 0;
  heavy[v] = deg > kWarpMax ? 1 : 0;
}

__global__ void k_compact_flags(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t K,
                                int32_t* __restrict__ out) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < K && flag[v]) out[pos[v]] = (int32_t)v;
}

// Net centres z_j of general nets (Algorithm 4).
__global__ void k_net_center(const int32_t* __restrict__ net_ptr, const int32_t* __restrict__ pins, int64_t l,
                             const float4* __restrict__ x, float4* __restrict__ z) {
  pdl_wait();
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= l) return;
  int32_t a = net_ptr[j], b = net_ptr[j + 1];
  float4 s = make_float4(0, 0, 0, 0);
  for (int32_t t = a; t < b; ++t) {
    float4 q = x[pins[t]];
    s.x += q.x; s.y += q.y; s.z += q.z; s.w += q.w;
  }
  float inv = (b > a) ? 1.0f / (float)(b - a) : 0.f;
  z[j] = make_float4(s.x * inv, s.y * inv, s.z * inv, s.w * inv);
}

__global__ void k_attract_hyper(const int32_t* __restrict__ vtx_ptr, const int32_t* __restrict__ vnets,
                                const float4* __restrict__ x, const float4* __restrict__ z, int64_t K,
                                float4* __restrict__ y) {
  pdl_wait();
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  float4 xv = x[v];
  float4 a = make_float4(0, 0, 0, 0);
  for (int32_t t = vtx_ptr[v]; t < vtx_ptr[v + 1]; ++t) {
    float4 q = z[vnets[t]];
    a.x += xv.x - q.x; a.y += xv.y - q.y; a.z += xv.z - q.z; a.w += xv.w - q.w;
  }
  y[v] = a;
}

// Approximate reciprocal and reciprocal square root (PTX rcp/rsqrt.approx,
// flush-to-zero) for the force terms; the decisions elsewhere use exactly
// rounded intrinsics.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Added to every squared distance fed to the kernels.  A source at the
// target's own position (the target itself, a coincident point) has dx = 0
// and so contributes exactly 0 * g = 0; the offset keeps g finite for it.
// Masked sources (weight 0) contribute 0 the same way.  For real pairs the
// relative change of r^2 is 1e-15 / r^2, negligible at the spacings of a
// layout (mean point spacing ~1).
constexpr float kR2Floor = 1e-15f;

// F += w r^-d (src - xn) for the two sources of a pair; nx holds -xn twice
// per coordinate, w the (masked) weights.  UNIT: both weights are 1 (the
// multiply by w is left out; a half is masked by giving it the target's own
// coordinates instead, so that its dx = 0 contributes 0).
template <int D, bool UNIT = false>
__device__ __forceinline__ void pair_charge(float2* F, const float4* P, const float2* nx, float2 w) {
  float2 dx[D];
  dx[0] = __fadd2_rn(make_float2(P[0].x, P[0].y), nx[0]);
  if (D > 1) dx[1] = __fadd2_rn(make_float2(P[0].z, P[0].w), nx[1]);
  if (D > 2) dx[2] = __fadd2_rn(make_float2(P[1].x, P[1].y), nx[2]);
  if (D > 3) dx[3] = __fadd2_rn(make_float2(P[1].z, P[1].w), nx[3]);
  float2 r2 = make_float2(kR2Floor, kR2Floor);  // offset: a source at the target's position gives 0 * finite
#pragma unroll
  for (int m = 0; m < D; ++m) r2 = __ffma2_rn(dx[m], dx[m], r2);
  float2 g;
  if (D == 2) {
    const float2 i2 = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
    g = UNIT ? i2 : __fmul2_rn(w, i2);
  } else if (D == 3) {
    const float2 ir = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
    g = UNIT ? __fmul2_rn(ir, __fmul2_rn(ir, ir)) : __fmul2_rn(__fmul2_rn(w, ir), __fmul2_rn(ir, ir));
  } else {
    const float2 i2 = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
    g = UNIT ? __fmul2_rn(i2, i2) : __fmul2_rn(__fmul2_rn(w, i2), i2);
  }
#pragma unroll
  for (int m = 0; m < D; ++m) F[m] = __ffma2_rn(g, dx[m], F[m]);
}

// Gives half h of a pair the target's coordinates (-nx), so it contributes 0.
template <int D>
__device__ __forceinline__ void pair_mask_half(float4* P, int h, bool mask, const float2* nx) {
  float* f = reinterpret_cast<float*>(P);
#pragma unroll
  for (int m = 0; m < D; ++m) {
    const int i = 4 * (m >> 1) + 2 * (m & 1);
    if (h == 0) f[i] = mask ? -nx[m].x : f[i];
    else f[i + 1] = mask ? -nx[m].x : f[i + 1];
  }
}

template <int D>
__device__ __forceinline__ float2 pair_weight(const float4* P) {
  const float4& q = P[Pair<D>::WQ];
  return Pair<D>::WO == 0 ? make_float2(q.x, q.y) : make_float2(q.z, q.w);
}

// Far-field charges of one level for a target in cell `me` (level l): the
// cells of the 6^d box spanned by the children of the cells around the
// target's parent cell, minus the 3^d cells adjacent to the target's cell.
// One row of the box along coordinate 0 starts at an even cell and holds 4 or
// 6 cells, i.e. 2 or 3 pairs: all loads are issued first, then the pairs are
// accumulated without branches (a pair beyond the row is loaded as zeros and
// weighs 0).  A cell counts if it holds weight and is not adjacent to the
// target's cell.
template <int D, bool COUNT>
__device__ inline void far_row(const float4* __restrict__ CP, int64_t cell0, int lo0, int hi0, bool incore, int me0,
                               const float2* nx, float2* F, unsigned long long& nint) {
  constexpr int N = Pair<D>::N;
  float4 P[3][N];
  const int npairs = (hi0 - lo0 + 1) >> 1;
  const float4* row = CP + (cell0 >> 1) * N;
  // a row holds 2 or 3 pairs: only the third is conditional
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) P[i][j] = (i < 2 || npairs > 2) ? row[i * N + j] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float2 w = pair_weight<D>(P[i]);
    if (incore) {
      const int xa = lo0 + 2 * i;
      w.x = (xa >= me0 - 1 && xa <= me0 + 1) ? 0.0f : w.x;
      w.y = (xa + 1 >= me0 - 1 && xa + 1 <= me0 + 1) ? 0.0f : w.y;
    }
    pair_charge<D>(F, P[i], nx, w);
    if (COUNT) nint += (w.x > 0.0f) + (w.y > 0.0f);
  }
}

// Far field of one level for one lane of the target's group: the rows of the
// box (row-major order) go round-robin to the G lanes of the group, each lane
// visiting only its own rows.  `cell` is the paired-table index of the
// level's cell 0 (even).
template <int D, bool COUNT>
__device__ inline void far_level_lane(const float4* __restrict__ CP, int64_t cell, const int32_t* me, int l,
                                      const float2* nx, float2* F, int G, int lane_g, unsigned long long& nint) {
  const int sl = 1 << l;
  int lo[D], hi[D];
#pragma unroll
  for (int m = 0; m < D; ++m) {
    int par = me[m] >> 1;
    lo[m] = max(2 * par - 2, 0);
    hi[m] = min(2 * par + 3, sl - 1);
  }
  if (G > 1) {
    // several lanes: the lane's own rows lane_g, lane_g + G, ... (row-major,
    // coordinate 1 fastest), stepped with carries instead of walking the others
    const int e1 = hi[1] - lo[1] + 1, e2 = D > 2 ? hi[2] - lo[2] + 1 : 1;
    int y = lo[1] + lane_g, z = D > 2 ? lo[2] : 0, w = D > 3 ? lo[3] : 0;
    auto carry = [&]() {
      while (y > hi[1]) {
        y -= e1;
        ++z;
        if (D > 3 && z > hi[2]) {
          z -= e2;
          ++w;
        }
      }
    };
    if (D > 2) carry();
    for (;;) {
      if (D == 2 && y > hi[1]) break;
      if (D == 3 && z > hi[2]) break;
      if (D == 4 && w > hi[3]) break;
      bool in = y >= me[1] - 1 && y <= me[1] + 1;
      int64_t idx = y;
      if (D > 2) {
        in = in && z >= me[2] - 1 && z <= me[2] + 1;
        idx = (int64_t)z * sl + y;
      }
      if (D > 3) {
        in = in && w >= me[3] - 1 && w <= me[3] + 1;
        idx = ((int64_t)w * sl + z) * sl + y;
      }
      far_row<D, COUNT>(CP, cell + idx * sl + lo[0], lo[0], hi[0], in, me[0], nx, F, nint);
      y += G;
      if (D > 2) carry();
    }
    return;
  }
  if (D == 2) {
    for (int y = lo[1]; y <= hi[1]; ++y) {
      const bool iny = y >= me[1] - 1 && y <= me[1] + 1;
      far_row<D, COUNT>(CP, cell + (int64_t)y * sl + lo[0], lo[0], hi[0], iny, me[0], nx, F, nint);
    }
  } else if (D == 3) {
    for (int z = lo[2]; z <= hi[2]; ++z) {
      const bool inz = z >= me[2] - 1 && z <= me[2] + 1;
      for (int y = lo[1]; y <= hi[1]; ++y) {
        const bool iny = inz && y >= me[1] - 1 && y <= me[1] + 1;
        far_row<D, COUNT>(CP, cell + ((int64_t)z * sl + y) * sl + lo[0], lo[0], hi[0], iny, me[0], nx, F, nint);
      }
    }
  } else {
    for (int w = lo[3]; w <= hi[3]; ++w) {
      const bool inw = w >= me[3] - 1 && w <= me[3] + 1;
      for (int z = lo[2]; z <= hi[2]; ++z) {
        const bool inz = inw && z >= me[2] - 1 && z <= me[2] + 1;
        for (int y = lo[1]; y <= hi[1]; ++y) {
          const bool iny = inz && y >= me[1] - 1 && y <= me[1] + 1;
          far_row<D, COUNT>(CP, cell + (((int64_t)w * sl + z) * sl + y) * sl + lo[0], lo[0], hi[0], iny, me[0], nx,
                            F, nint);
        }
      }
    }
  }
}

// The same far field with two of the lane's rows in flight: both rows' pairs
// are loaded before either is accumulated, rows taken in the same order (so
// the sums are bit-identical to far_level_lane).  Used for launches too small
// to hide load latency with other warps (the small levels of a hierarchy).
template <int D, bool COUNT>
__device__ inline void far_level_lane2(const float4* __restrict__ CP, int64_t cell, const int32_t* me, int l,
                                       const float2* nx, float2* F, int G, int lane_g, unsigned long long& nint) {
  constexpr int N = Pair<D>::N;
  const int sl = 1 << l;
  int lo[D], hi[D], ext[D];
#pragma unroll
  for (int m = 0; m < D; ++m) {
    int par = me[m] >> 1;
    lo[m] = max(2 * par - 2, 0);
    hi[m] = min(2 * par + 3, sl - 1);
    ext[m] = hi[m] - lo[m] + 1;
  }
  int nrows = 1;
#pragma unroll
  for (int m = 1; m < D; ++m) nrows *= ext[m];
  const int npairs = ext[0] >> 1;
  // row r (row-major over coordinates 1..D-1, coordinate 1 fastest): its
  // first cell and whether it is adjacent to the target's cell in 1..D-1
  auto row_at = [&](int r, int64_t& c0, bool& in) {
    int64_t idx = 0;
    bool adj = true;
    int q[D];
#pragma unroll
    for (int m = 1; m < D; ++m) {
      q[m] = lo[m] + r % ext[m];
      r /= ext[m];
      adj = adj && q[m] >= me[m] - 1 && q[m] <= me[m] + 1;
    }
#pragma unroll
    for (int m = D - 1; m >= 1; --m) idx = idx * sl + q[m];
    c0 = cell + idx * sl + lo[0];
    in = adj;
  };
  auto load = [&](int64_t c0, float4 (*P)[N]) {
    const float4* row = CP + (c0 >> 1) * N;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j) P[i][j] = (i < 2 || npairs > 2) ? row[i * N + j] : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto apply = [&](float4 (*P)[N], bool incore) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float2 w = pair_weight<D>(P[i]);
      if (incore) {
        const int xa = lo[0] + 2 * i;
        w.x = (xa >= me[0] - 1 && xa <= me[0] + 1) ? 0.0f : w.x;
        w.y = (xa + 1 >= me[0] - 1 && xa + 1 <= me[0] + 1) ? 0.0f : w.y;
      }
      pair_charge<D>(F, P[i], nx, w);
      if (COUNT) nint += (w.x > 0.0f) + (w.y > 0.0f);
    }
  };
  int r = lane_g;
  for (; r + G < nrows; r += 2 * G) {
    int64_t ca, cb;
    bool ia, ib;
    row_at(r, ca, ia);
    row_at(r + G, cb, ib);
    float4 A[3][N], B[3][N];
    load(ca, A);
    load(cb, B);
    apply(A, ia);
    apply(B, ib);
  }
  if (r < nrows) {
    int64_t ca;
    bool ia;
    row_at(r, ca, ia);
    float4 A[3][N];
    load(ca, A);
    apply(A, ia);
  }
}

// Next bounding box, folded in by the step kernel: lane 0 of every warp (a
// warp never straddles two problems) applies atomic min / max of the
// order-preserving integer images of its lanes' new coordinates to the
// problem's box, which k_keys reset earlier in the step.  Min and max are
// exact, so the order of the atomics does not matter.
template <int D>
__device__ inline void bbox_warp_fold(const float4& v, bool valid, uint32_t* __restrict__ box) {
  uint32_t mn[4], mx[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    uint32_t o = (valid && m < D) ? f2ord(comp(v, m)) : 0u;
    mn[m] = __reduce_min_sync(0xffffffffu, (valid && m < D) ? o : 0xFFFFFFFFu);
    mx[m] = __reduce_max_sync(0xffffffffu, o);
  }
  if (lane_id() == 0 && mn[0] != 0xFFFFFFFFu) {
#pragma unroll
    for (int m = 0; m < D; ++m) {
      atomicMin(box + m, mn[m]);
      atomicMax(box + 4 + m, mx[m]);
    }
  }
}

// Near field of one row range [qa, qb) of problem-local sorted positions for
// one lane of the target's group: source pairs j = qa/2 + lane_g, + G, ...,
// four pairs per trip (all loads issued before the arithmetic; the order of
// the pairs in the sums is the same as one pair per trip).  Only the first
// pair can start before qa and only the last can end at or after qb; those
// halves are masked (weight 0, or the target's own coordinates when UNIT).
template <int D, bool COUNT, bool UNIT>
__device__ __forceinline__ void near_range(const float4* __restrict__ xp, int qa, int qb, int G, int lane_g,
                                           int64_t tgt, const float2* nx, float2* F, unsigned long long& nint) {
  constexpr int N = Pair<D>::N;
  int j = (qa >> 1) + lane_g;
  for (; 2 * (j + 7 * G) < qb; j += 8 * G) {
    float4 Q[8][N];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int i = 0; i < N; ++i) Q[u][i] = xp[(int64_t)(j + u * G) * N + i];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int h0 = 2 * (j + u * G);
      float2 w = make_float2(1.0f, 1.0f);
      if (UNIT) {
        if (u == 0) pair_mask_half<D>(Q[u], 0, h0 < qa, nx);
        if (u == 7) pair_mask_half<D>(Q[u], 1, h0 + 1 >= qb, nx);
      } else {
        w = pair_weight<D>(Q[u]);
        if (u == 0) w.x = h0 >= qa ? w.x : 0.0f;
        if (u == 7) w.y = h0 + 1 < qb ? w.y : 0.0f;
      }
      pair_charge<D, UNIT>(F, Q[u], nx, w);
      if (COUNT) nint += (h0 >= qa && h0 != tgt) + (h0 + 1 < qb && h0 + 1 != tgt);
    }
  }
  for (; 2 * (j + 3 * G) < qb; j += 4 * G) {
    float4 Q[4][N];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < N; ++i) Q[u][i] = xp[(int64_t)(j + u * G) * N + i];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int h0 = 2 * (j + u * G);
      float2 w = make_float2(1.0f, 1.0f);
      if (UNIT) {
        if (u == 0) pair_mask_half<D>(Q[u], 0, h0 < qa, nx);
        if (u == 3) pair_mask_half<D>(Q[u], 1, h0 + 1 >= qb, nx);
      } else {
        w = pair_weight<D>(Q[u]);
        if (u == 0) w.x = h0 >= qa ? w.x : 0.0f;
        if (u == 3) w.y = h0 + 1 < qb ? w.y : 0.0f;
      }
      pair_charge<D, UNIT>(F, Q[u], nx, w);
      if (COUNT) nint += (h0 >= qa && h0 != tgt) + (h0 + 1 < qb && h0 + 1 != tgt);
    }
  }
  for (; 2 * j < qb; j += G) {
    float4 Q[N];
#pragma unroll
    for (int i = 0; i < N; ++i) Q[i] = xp[(int64_t)j * N + i];
    float2 w = make_float2(1.0f, 1.0f);
    if (UNIT) {
      pair_mask_half<D>(Q, 0, 2 * j < qa, nx);
      pair_mask_half<D>(Q, 1, 2 * j + 1 >= qb, nx);
    } else {
      w = pair_weight<D>(Q);
      w.x = 2 * j >= qa ? w.x : 0.0f;
      w.y = 2 * j + 1 < qb ? w.y : 0.0f;
    }
    pair_charge<D, UNIT>(F, Q, nx, w);
    if (COUNT) nint += (2 * j >= qa && 2 * j != tgt) + (2 * j + 1 < qb && 2 * j + 1 != tgt);
  }
}

// Gradient (eq. graphenergygradientsimple with the grid pyramid) and step of
// every target.  Each problem gives its targets G lanes (G from the problem's
// own size), padded to whole warps; the lanes of a group split the near field
// (strided source pairs) and the far field (rows of every level's box) and
// combine with a fixed xor tree, so a target's result depends only on its own
// problem.  Lane 0 of the group applies the step.  Near field: points are
// sorted by row-major cell index, so the 3 cells of a row along coordinate 0
// form one contiguous range of the sorted points, read in pairs from the
// paired point table XP (a problem's points start at the even slot
// (vbase + pb + 1) & ~1; the halves outside the range weigh 0).  Far field:
// the paired cell table CP, whose index of (problem pb, level l, cell c) is
// cbase + pb + lvl_off(l) + 1 + c (even for even c).
#ifndef VMO_STEP_BLOCK
#define VMO_STEP_BLOCK 128
#endif
#ifndef VMO_STEP_MINBLOCKS
#define VMO_STEP_MINBLOCKS 6
#endif
constexpr int kStepBlock = VMO_STEP_BLOCK;
// step launches of at most g_tuning.small_step_threads threads (default
// about 4 warps per SM) take the far-field variant with two rows in flight

template <int D, bool COUNT, bool MLP>
__global__ void __launch_bounds__(kStepBlock, MLP ? 3 : VMO_STEP_MINBLOCKS) k_repulse_update(
    const float4* __restrict__ xs, const float* __restrict__ ws, const float4* __restrict__ XP,
    const uint32_t* __restrict__ svals, const uint32_t* __restrict__ scell, const int32_t* __restrict__ cst,
    const float4* __restrict__ CP, const float4* __restrict__ yatt, const int64_t* __restrict__ tbase, int P,
    const ProbDev* __restrict__ prob, int64_t T, float kappa, const float* __restrict__ s0,
    const float* __restrict__ scale_tab, const int32_t* __restrict__ tctr,
    float step_override, float4* __restrict__ x, float4* __restrict__ y_out, uint32_t* __restrict__ bb_next,
    unsigned long long* __restrict__ icount) {
  pdl_wait();
  constexpr int N = Pair<D>::N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int pb = find_problem(tbase, P, t < T ? t : T - 1);
  const ProbDev pr = prob[pb];
  const int G = pr.group;
  const int64_t rel = t - pr.tbase;
  const int64_t tgt = rel / G;
  const int lane_g = (int)(rel & (G - 1));
  const bool valid = t < T && tgt < pr.k;
  unsigned long long nint = 0;
  float2 F[D];
#pragma unroll
  for (int m = 0; m < D; ++m) F[m] = make_float2(0.f, 0.f);
  const int64_t p = pr.vbase + tgt;
  float4 xn = make_float4(0, 0, 0, 0);
  if (valid) {
    const int L = pr.L, side = 1 << L;
    xn = xs[p];
    float2 nx[D];
#pragma unroll
    for (int m = 0; m < D; ++m) nx[m] = make_float2(-comp(xn, m), -comp(xn, m));
    const uint32_t packed = scell[p];
    int32_t c[D];
#pragma unroll
    for (int m = 0; m < D; ++m) c[m] = (int32_t)((packed >> (m * field_bits(D))) & ((1u << field_bits(D)) - 1));
    // near field: rows of 3 cells along coordinate 0 around the target's cell
    const int32_t* cs = cst + pr.fbase + pb;
    const float4* xp = XP + ((pr.vbase + pb + 1) >> 1) * N;  // the problem's first pair
    const int xa = max(c[0] - 1, 0), xb = min(c[0] + 1, side - 1);
    constexpr int NR = D == 2 ? 3 : (D == 3 ? 9 : 27);
    // the row ranges [qa, qb) of the problem's sorted points (empty: outside the grid)
    auto row_range = [&](int o, int& qa, int& qb) {
      int32_t cc[D];
      int oo = o;
      bool inside = true;
      cc[0] = xa;
#pragma unroll
      for (int m = 1; m < D; ++m) {
        cc[m] = c[m] + (oo % 3) - 1;
        oo /= 3;
        inside = inside && cc[m] >= 0 && cc[m] < side;
      }
      qa = qb = 0;
      if (!inside) return;
      const int64_t r0 = rowmajor<D>(cc, side);
      qa = cs[r0] - (int)pr.vbase;  // problem-local
      qb = cs[r0 + (xb - xa) + 1] - (int)pr.vbase;
    };
    auto near_row = [&](int qa, int qb) {
      if (qa >= qb) return;
      if (ws)
        near_range<D, COUNT, false>(xp, qa, qb, G, lane_g, tgt, nx, F, nint);
      else
        near_range<D, COUNT, true>(xp, qa, qb, G, lane_g, tgt, nx, F, nint);
    };
    if (MLP && D <= 3) {
      // small launches: all rows' ranges loaded before the first row is used
      int qa[NR], qb[NR];
#pragma unroll
      for (int o = 0; o < NR; ++o) row_range(o, qa[o], qb[o]);
#pragma unroll
      for (int o = 0; o < NR; ++o) near_row(qa[o], qb[o]);
    } else {
      for (int o = 0; o < NR; ++o) {
        int qa, qb;
        row_range(o, qa, qb);
        near_row(qa, qb);
      }
    }
    // far field, levels 2..L
    for (int l = 2; l <= L; ++l) {
      int32_t me[D];
#pragma unroll
      for (int m = 0; m < D; ++m) me[m] = c[m] >> (L - l);
      if (MLP)
        far_level_lane2<D, COUNT>(CP, pr.cbase + pb + lvl_off(D, l) + 1, me, l, nx, F, G, lane_g, nint);
      else
        far_level_lane<D, COUNT>(CP, pr.cbase + pb + lvl_off(D, l) + 1, me, l, nx, F, G, lane_g, nint);
    }
  }
  float Fs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int m = 0; m < D; ++m) Fs[m] = F[m].x + F[m].y;
  // combine the lanes of the group (groups never straddle a warp)
  for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
    for (int m = 0; m < D; ++m) Fs[m] += __shfl_xor_sync(0xffffffffu, Fs[m], o);
  const bool leader = valid && lane_g == 0;
  float4 xnew = make_float4(0, 0, 0, 0);
  if (leader) {
    const float wn = ws ? ws[p] : 1.0f;
    const uint32_t v = svals[p];
    float4 ya = yatt[v];
    float y0 = kappa * wn * Fs[0] + ya.x;
    float y1 = D > 1 ? kappa * wn * Fs[1] + ya.y : 0.f;
    float y2 = D > 2 ? kappa * wn * Fs[2] + ya.z : 0.f;
    float y3 = D > 3 ? kappa * wn * Fs[3] + ya.w : 0.f;
    if (y_out) y_out[v] = make_float4(y0, y1, y2, y3);
    float ny = sqrtf(y0 * y0 + y1 * y1 + y2 * y2 + y3 * y3);
    float step = step_override > 0.0f ? step_override : s0[pb] * scale_tab[*tctr];
    float a = ny > 0.0f ? step / ny : 0.0f;
    xnew = make_float4(xn.x - a * y0, D > 1 ? xn.y - a * y1 : 0.f, D > 2 ? xn.z - a * y2 : 0.f,
                       D > 3 ? xn.w - a * y3 : 0.f);
    x[v] = xnew;
  }
  if (COUNT) {
    unsigned long long tot = nint;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane_id() == 0 && tot) atomicAdd(icount, tot);
  }
  bbox_warp_fold<D>(xnew, leader, bb_next + (int64_t)pb * 8);
}

// Step-length factors decay^t, t < iters: the running double product, each
// rounded to fp32 (one thread, the same operations in the same order on every
// call), so that no host table has to be uploaded per level.
__global__ void k_scale_tab(int iters, double decay, float* __restrict__ tab) {
  double scale = 1.0;
  for (int t = 0; t < iters; ++t) {
    tab[t] = (float)scale;
    scale *= decay;
  }
}

// ------------------------------ initial layout -----------------------------
__global__ void k_init_coords(int64_t K, const int32_t* __restrict__ vprob, const ProbDev* __restrict__ prob,
                              const uint64_t* __restrict__ seeds, const int32_t* __restrict__ start, int D,
                              float4* __restrict__ x) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  int pb = vprob[v];
  if (start && !start[pb]) return;
  ProbDev pr = prob[pb];
  uint64_t lv = (uint64_t)(v - pr.vbase);
  float side = (float)pr.side;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  for (int m = 0; m < D; ++m) {
    uint64_t r = rand64(seeds[pb] ^ kTagCoord, lv, (uint64_t)m);
    float u = __fmul_rn((float)(r >> 40), 0x1p-24f);
    c[m] = __fmul_rn(u, side);
  }
  x[v] = make_float4(c[0], c[1], c[2], c[3]);
}

// Prolongation (Algorithm 3): x(v) = f * x_coarse(pi(v)) + jitter.
__global__ void k_prolong(const float4* __restrict__ xc, const int32_t* __restrict__ pi, int64_t K,
                          const int32_t* __restrict__ vprob, const ProbDev* __restrict__ prob,
                          const float* __restrict__ fac, const uint64_t* __restrict__ seeds, int level, int D,
                          float4* __restrict__ x) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  int pb = vprob[v];
  float f = fac[pb];
  if (!(f > 0.0f)) return;
  uint64_t lv = (uint64_t)(v - prob[pb].vbase);
  float4 q = xc[pi[v]];
  float c[4] = {q.x, q.y, q.z, q.w};
  float o[4] = {0.f, 0.f, 0.f, 0.f};
  for (int m = 0; m < D; ++m) {
    uint64_t r = rand64(seeds[pb] ^ kTagJitter, lv, (uint64_t)(4 * level + m));
    float u = (float)(r >> 40) * 0x1p-24f;
    o[m] = f * c[m] + 0.1f * (u - 0.5f);
  }
  x[v] = make_float4(o[0], o[1], o[2], o[3]);
}

// ------------------------------- coarsening --------------------------------
// Handshake heavy-edge matching round: every unmatched vertex of an active
// problem proposes to its unmatched neighbour with the largest cost, ties by
// the smaller hash of the (local) pair and then the smaller id.  The choice is
// an arg-max under a total order, so light (thread), medium (warp) and heavy
// (block) rows all give the same answer.
struct Proposal {
  float c;
  uint64_t h;
  int32_t u;
};

__device__ inline bool better(const Proposal& a, const Proposal& b) {
  if (a.u < 0) return false;
  if (b.u < 0) return true;
  return a.c > b.c || (a.c == b.c && (a.h < b.h || (a.h == b.h && a.u < b.u)));
}

__device__ inline Proposal scan_row(const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                                    const float* __restrict__ acost, const int32_t* __restrict__ mate, int64_t v,
                                    int64_t vb, uint64_t seed, uint64_t b, int32_t start, int32_t stride) {
  // `better` is a total order on the candidates (a row's neighbours are
  // distinct), so the best does not depend on the order they are seen in:
  // four neighbours per trip, their loads issued together
  Proposal best{0.f, 0ull, -1};
  auto consider = [&](int32_t u, int32_t mu, float c) {
    if (u == v || mu >= 0) return;
    uint64_t lu = (uint64_t)(u - vb), lv = (uint64_t)(v - vb);
    uint64_t lo = lu < lv ? lu : lv, hi = lu < lv ? lv : lu;
    Proposal cand{c, rand64(seed, (lo << 32) | hi, b), u};
    if (better(cand, best)) best = cand;
  };
  const int32_t t1 = adj_ptr[v + 1];
  int32_t t = adj_ptr[v] + start;
  for (; t + 3 * stride < t1; t += 4 * stride) {
    int32_t u[4], mu[4];
    float c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = adj[t + q * stride];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      mu[q] = mate[u[q]];
      c[q] = acost ? acost[t + q * stride] : 1.0f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) consider(u[q], mu[q], c[q]);
  }
  for (; t < t1; t += stride) {
    const int32_t u = adj[t];
    consider(u, mate[u], acost ? acost[t] : 1.0f);
  }
  return best;
}

__device__ inline Proposal warp_best(Proposal p) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Proposal q;
    q.c = __shfl_xor_sync(0xffffffffu, p.c, o);
    q.h = __shfl_xor_sync(0xffffffffu, p.h, o);
    q.u = __shfl_xor_sync(0xffffffffu, p.u, o);
    if (better(q, p)) p = q;
  }
  return p;
}

__global__ void k_propose(const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                          const float* __restrict__ acost, int64_t K, const int32_t* __restrict__ vprob,
                          const ProbDev* __restrict__ prob, const int32_t* __restrict__ active,
                          const uint64_t* __restrict__ seeds, int level, int round, const int32_t* __restrict__ mate,
                          int32_t* __restrict__ prop) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  if (adj_ptr[v + 1] - adj_ptr[v] > kLightMax) return;  // k_propose_wide
  int pb = vprob[v];
  int32_t best = -1;
  if (active[pb] && mate[v] < 0)
    best = scan_row(adj_ptr, adj, acost, mate, v, prob[pb].vbase, seeds[pb] ^ kTagMatch,
                    (uint64_t)level * 256 + (uint64_t)round, 0, 1).u;
  prop[v] = best;
}

// Medium rows (list, warp each) or heavy rows (list, block each).
__global__ void __launch_bounds__(kBlock) k_propose_wide(const int32_t* __restrict__ list, int64_t n, int per_block,
                                                         const int32_t* __restrict__ adj_ptr,
                                                         const int32_t* __restrict__ adj,
                                                         const float* __restrict__ acost,
                                                         const int32_t* __restrict__ vprob,
                                                         const ProbDev* __restrict__ prob,
                                                         const int32_t* __restrict__ active,
                                                         const uint64_t* __restrict__ seeds, int level, int round,
                                                         const int32_t* __restrict__ mate,
                                                         int32_t* __restrict__ prop) {
  __shared__ Proposal part[kBlock / 32];
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  int64_t item = per_block ? (int64_t)blockIdx.x : (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  bool ok = item < n;
  int32_t v = ok ? list[item] : 0;
  int pb = ok ? vprob[v] : 0;
  bool act = ok && active[pb] && mate[v] < 0;
  Proposal best{0.f, 0ull, -1};
  if (act) {
    int32_t start = per_block ? (int32_t)threadIdx.x : lane;
    int32_t stride = per_block ? (int32_t)blockDim.x : 32;
    best = scan_row(adj_ptr, adj, acost, mate, v, prob[pb].vbase, seeds[pb] ^ kTagMatch,
                    (uint64_t)level * 256 + (uint64_t)round, start, stride);
  }
  best = warp_best(best);
  if (!per_block) {
    if (ok && lane == 0) prop[v] = best.u;
    return;
  }
  if (lane == 0) part[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0 && ok) {
    Proposal b = part[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (better(part[w], b)) b = part[w];
    prop[v] = b.u;
  }
}

__global__ void k_resolve(const int32_t* __restrict__ prop, int64_t K, int32_t* __restrict__ mate) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  int32_t u = prop[v];
  if (u >= 0 && prop[u] == v) mate[v] = u;
}

__global__ void k_anchor(const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj, int64_t K,
                         const int32_t* __restrict__ mate, int32_t* __restrict__ anchor, int32_t* __restrict__ isanc) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  int32_t mv = mate[v];
  int32_t a = mv >= 0 ? min((int32_t)v, mv) : (int32_t)v;
  if (mv < 0 && adj_ptr[v + 1] - adj_ptr[v] == 1) {
    int32_t u = adj[adj_ptr[v]];
    if (u != v) {
      int32_t mu = mate[u];
      a = mu >= 0 ? min(u, mu) : u;
    }
  }
  anchor[v] = a;
  isanc[a] = 1;
}

__global__ void k_kc(const int32_t* __restrict__ rank, const int32_t* __restrict__ total, const int64_t* __restrict__ vb,
                     int P, int64_t K, int64_t* __restrict__ kc) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int64_t a = vb[p], b = vb[p + 1];
  int64_t ra = a < K ? rank[a] : *total;
  int64_t rb = b < K ? rank[b] : *total;
  kc[p] = rb - ra;
}

__global__ void k_pi(const int32_t* __restrict__ anchor, const int32_t* __restrict__ rank, int64_t K,
                     const int32_t* __restrict__ vprob, const ProbDev* __restrict__ prob,
                     const int64_t* __restrict__ newbase, int32_t* __restrict__ pi) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  int pb = vprob[v];
  int64_t nb = newbase[pb];
  pi[v] = nb >= 0 ? (int32_t)(nb + rank[anchor[v]] - rank[prob[pb].vbase]) : -1;
}

// Coarse-edge key and cost of the adjacency entries t, t + stride, ... < t1 of
// a row whose vertex has group a: key (a, pi[adj[t]]) in row-major order of
// the coarse pair, the sentinel for an edge inside a group or of a dropped
// vertex.  Every entry's output depends only on the entry, so rows are split
// by degree as for the attraction: a thread per light row (k_contract_keys),
// a warp per medium row, a block per heavy row (the power-law hubs).
__device__ __forceinline__ void contract_row(const int32_t* __restrict__ adj, const float* __restrict__ acost,
                                             const int32_t* __restrict__ pi, int32_t a, int32_t t, int32_t t1,
                                             int32_t stride, uint64_t Kc, uint64_t* __restrict__ keys,
                                             uint32_t* __restrict__ vals) {
  const uint64_t sentinel = Kc * Kc;
  for (; t < t1; t += stride) {
    const int32_t b = a >= 0 ? pi[adj[t]] : -1;
    keys[t] = (a >= 0 && b >= 0 && a != b) ? (uint64_t)a * Kc + (uint64_t)b : sentinel;
    vals[t] = __float_as_uint(acost ? acost[t] : 1.0f);
  }
}

__global__ void k_contract_keys(const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                                const float* __restrict__ acost, int64_t K, const int32_t* __restrict__ pi,
                                uint64_t Kc, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  const int32_t t0 = adj_ptr[v], t1 = adj_ptr[v + 1];
  if (t1 - t0 > kLightMax) return;  // medium and heavy rows: k_contract_keys_warp / _block
  contract_row(adj, acost, pi, pi[v], t0, t1, 1, Kc, keys, vals);
}

__global__ void k_contract_keys_warp(const int32_t* __restrict__ list, int64_t n, const int32_t* __restrict__ adj_ptr,
                                     const int32_t* __restrict__ adj, const float* __restrict__ acost,
                                     const int32_t* __restrict__ pi, uint64_t Kc, uint64_t* __restrict__ keys,
                                     uint32_t* __restrict__ vals) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;
  const int32_t v = list[w];
  contract_row(adj, acost, pi, pi[v], adj_ptr[v] + (int32_t)lane_id(), adj_ptr[v + 1], 32, Kc, keys, vals);
}

__global__ void k_contract_keys_block(const int32_t* __restrict__ list, const int32_t* __restrict__ adj_ptr,
                                      const int32_t* __restrict__ adj, const float* __restrict__ acost,
                                      const int32_t* __restrict__ pi, uint64_t Kc, uint64_t* __restrict__ keys,
                                      uint32_t* __restrict__ vals) {
  const int32_t v = list[blockIdx.x];
  contract_row(adj, acost, pi, pi[v], adj_ptr[v] + (int32_t)threadIdx.x, adj_ptr[v + 1], (int32_t)blockDim.x, Kc,
               keys, vals);
}

__global__ void k_run_flags(const uint64_t* __restrict__ keys, int64_t n, uint64_t sentinel, int32_t* __restrict__ flag) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  uint64_t k = keys[t];
  flag[t] = (k != sentinel && (t == 0 || keys[t - 1] != k)) ? 1 : 0;
}

__global__ void k_emit_coarse(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n,
                              const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, uint64_t Kc,
                              int32_t* __restrict__ adj, float* __restrict__ acost, int32_t* __restrict__ rowcount) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n || !flag[t]) return;
  uint64_t k = keys[t];
  float c = 0.f;
  for (int64_t u = t; u < n && keys[u] == k; ++u) c += __uint_as_float(vals[u]);
  adj[pos[t]] = (int32_t)(k % Kc);
  acost[pos[t]] = c;
  atomicAdd(&rowcount[k / Kc], 1);
}

// Coarse vertex weights (Algorithm 3: a group weighs what its members weigh).
// The fp32 weights are added in FP64, where the sum of a group of fp32 values
// is exact (their exponents lie within the 29 spare bits), so the order of the
// atomics does not change the rounded fp32 result.
__global__ void k_coarse_w(const float* __restrict__ w, const int32_t* __restrict__ pi, int64_t K,
                           double* __restrict__ wc) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  int32_t a = pi[v];
  if (a >= 0) atomicAdd(&wc[a], (double)(w ? w[v] : 1.0f));
}

__global__ void k_round_w(const double* __restrict__ wd, int64_t n, float* __restrict__ w) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = (float)wd[i];
}

__global__ void k_fill_vprob(const int64_t* __restrict__ vb, int P, int64_t K, int32_t* __restrict__ vprob) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= K) return;
  vprob[v] = find_problem(vb, P, v);
}

__global__ void k_set_last(int32_t* ptr, int64_t n, const int32_t* total) { ptr[n] = *total; }

template <class F>
void dispatch_d(int d, F&& f) {
  if (d == 2) f(std::integral_constant<int, 2>());
  else if (d == 3) f(std::integral_constant<int, 3>());
  else f(std::integral_constant<int, 4>());
}

int lmax(int d) { return d == 2 ? 15 : (d == 3 ? 10 : 7); }

}  // namespace

int grid_levels(int64_t k, int d, int occ) {
  int L = 1;
  while (L < lmax(d) && (int64_t)occ * (int64_t(1) << (d * L)) < k) ++L;
  return L;
}

// Lanes per target of the step kernel: enough threads to fill the GPU for a
// small problem; a function of the problem's own size only.
int group_size(int64_t k) {
  // G lanes per target give a small problem (a latency-bound level) G-fold
  // shorter per-target chains, at the cost of the lanes' combining and of the
  // work each lane repeats; in a batch, where many problems already fill the
  // GPU, that cost is all that remains (measured: 4 / 2 lanes for <= 512 /
  // 4,096 vertices order the 4,096-matrix batch 17% faster than 16 / 4, a
  // single small matrix 3% slower).
  if (k <= 512) return 4;
  if (k <= 4096) return 2;
  return 1;
}

static vmo_status classify_degrees(LevelBatch& lb, cudaStream_t s) {
  lb.n_mid = lb.n_heavy = 0;
  if (!lb.adj_ptr || lb.K == 0) return VMO_OK;
  Scratch sc(s);
  int32_t *fm, *fh, *pm, *ph, *tm, *th;
  VMO_TRY(sc.alloc(&fm, lb.K));
  VMO_TRY(sc.alloc(&fh, lb.K));
  VMO_TRY(sc.alloc(&pm, lb.K));
  VMO_TRY(sc.alloc(&ph, lb.K));
  VMO_TRY(sc.alloc(&tm, 1));
  VMO_TRY(sc.alloc(&th, 1));
  launch(k_degree_class, grid_for(lb.K, kBlock), kBlock, 0, s, lb.adj_ptr, lb.K, fm, fh);
  VMO_LAUNCHED("degree_class");
  VMO_TRY(scan_exclusive<int32_t>(fm, pm, lb.K, tm, s, sc));
  VMO_TRY(scan_exclusive<int32_t>(fh, ph, lb.K, th, s, sc));
  int32_t h[2] = {0, 0};
  VMO_CUDA(cudaMemcpyAsync(&h[0], tm, 4, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaMemcpyAsync(&h[1], th, 4, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  lb.n_mid = h[0];
  lb.n_heavy = h[1];
  VMO_TRY(lb.mid_list.resize(std::max<int64_t>(lb.n_mid, 1)));
  VMO_TRY(lb.heavy_list.resize(std::max<int64_t>(lb.n_heavy, 1)));
  if (lb.n_mid) launch(k_compact_flags, grid_for(lb.K, kBlock), kBlock, 0, s, fm, pm, lb.K, lb.mid_list.ptr);
  if (lb.n_heavy) launch(k_compact_flags, grid_for(lb.K, kBlock), kBlock, 0, s, fh, ph, lb.K, lb.heavy_list.ptr);
  VMO_LAUNCHED("compact_flags");
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

int init_side(int64_t k, int d) {
  int64_t s = 1;
  for (;;) {
    int64_t p = 1;
    for (int i = 0; i < d; ++i) p *= s;
    if (p >= k) return (int)s;
    ++s;
  }
}

vmo_status level_setup(LevelBatch& lb, int d, int occ, cudaStream_t s) {
  const int P = lb.P;
  lb.L.assign(P, 1);
  lb.cbase.assign(P + 1, 0);
  lb.fbase.assign(P + 1, 0);
  std::vector<ProbDev> pd(P);
  std::vector<int64_t> tb(P + 1, 0);
  lb.maxL = 1;
  for (int p = 0; p < P; ++p) {
    int64_t k = lb.vbase[p + 1] - lb.vbase[p];
    int L = grid_levels(k, d, occ);
    lb.L[p] = L;
    lb.maxL = std::max(lb.maxL, L);
    lb.cbase[p + 1] = lb.cbase[p] + lvl_off(d, L + 1);
    lb.fbase[p + 1] = lb.fbase[p] + (int64_t(1) << (d * L));
    pd[p].vbase = lb.vbase[p];
    pd[p].cbase = lb.cbase[p];
    pd[p].fbase = lb.fbase[p];
    pd[p].k = (int32_t)k;
    pd[p].L = L;
    pd[p].side = init_side(std::max<int64_t>(k, 1), d);
    pd[p].group = group_size(k);
    pd[p].tbase = tb[p];
    tb[p + 1] = tb[p] + ((k * pd[p].group + 31) / 32) * 32;
  }
  lb.threads = tb[P];
  // prefix tables of the coarse-level aggregation steps: step s covers level L_p - s >= 2
  int nsteps = std::max(lb.maxL - 2, 0);
  std::vector<int64_t> off((size_t)(nsteps + 1) * (P + 1), 0);
  for (int st = 1; st <= nsteps; ++st)
    for (int p = 0; p < P; ++p) {
      int l = lb.L[p] - st;
      int64_t cnt = l > small_level_max(d) ? (int64_t(1) << (d * l)) : 0;
      off[(size_t)st * (P + 1) + p + 1] = off[(size_t)st * (P + 1) + p] + cnt;
    }
  VMO_TRY(lb.prob.resize(std::max(P, 1)));
  VMO_TRY(lb.aggoff.resize(off.size()));
  VMO_TRY(lb.vprob.resize((size_t)std::max<int64_t>(lb.K, 1)));
  VMO_CUDA(cudaMemcpyAsync(lb.prob.ptr, pd.data(), P * sizeof(ProbDev), cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(lb.aggoff.ptr, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  VMO_TRY(lb.tbase.resize(P + 1));
  VMO_CUDA(cudaMemcpyAsync(lb.tbase.ptr, tb.data(), (P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  VMO_TRY(lb.fbase_dev.resize(P + 1));
  VMO_CUDA(cudaMemcpyAsync(lb.fbase_dev.ptr, lb.fbase.data(), (P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  int64_t* vb;
  VMO_CUDA(cudaMallocAsync((void**)&vb, (P + 1) * sizeof(int64_t), s));
  g_device_allocs.fetch_add(1, std::memory_order_relaxed);
  VMO_CUDA(cudaMemcpyAsync(vb, lb.vbase.data(), (P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  if (lb.K > 0) {
    launch(k_fill_vprob, grid_for(lb.K, kBlock), kBlock, 0, s, vb, P, lb.K, lb.vprob.ptr);
    VMO_LAUNCHED("fill_vprob");
  }
  VMO_CUDA(cudaFreeAsync(vb, s));

  // host vectors must outlive the copies
  VMO_CUDA(cudaStreamSynchronize(s));
  return classify_degrees(lb, s);
}

vmo_status init_coords_level(LevelBatch& lb, int d, const uint64_t* seeds_dev, float4* x, const int32_t* start_dev,
                             cudaStream_t s) {
  if (lb.K == 0) return VMO_OK;
  launch(k_init_coords, grid_for(lb.K, kBlock), kBlock, 0, s, lb.K, lb.vprob.ptr, lb.prob.ptr, seeds_dev, start_dev, d, x);
  VMO_LAUNCHED("init_coords");
  return VMO_OK;
}

constexpr int kGraphMinIters = 8;

// Streams of one layout call: `side` for the attraction (fork / join events
// per step) and `main` for the steps when they are replayed from a graph
// (capture needs a stream of its own: the caller's may be the legacy stream);
// destroyed in stream order when the call returns.
struct SideStream {
  cudaStream_t stream = nullptr, main = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, start = nullptr, done = nullptr;
  SideStream() {
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
      (void)cudaGetLastError();
      release();
    }
  }
  void release() {
    for (cudaEvent_t* e : {&fork, &join, &start, &done}) {
      if (*e) cudaEventDestroy(*e);
      *e = nullptr;
    }
    if (stream) cudaStreamDestroy(stream);
    if (main) cudaStreamDestroy(main);
    stream = main = nullptr;
  }
  ~SideStream() { release(); }
};

// Points a Scratch at another stream for a scope (its allocations and frees
// then follow that stream's order).
struct ScratchOnStream {
  Scratch& sc;
  cudaStream_t prev;
  ScratchOnStream(Scratch& s, cudaStream_t st) : sc(s), prev(s.stream) { sc.stream = st; }
  ~ScratchOnStream() { sc.stream = prev; }
};

vmo_status layout_level(LevelBatch& lb, const LayoutOptions& o, float4* x, int iters, float step_override,
                        float4* y_out, uint32_t* keys_out, cudaStream_t s, Scratch& sc) {
  const int64_t K = lb.K;
  const int P = lb.P;
  const int d = o.d;
  if (K == 0 || iters <= 0) return VMO_OK;
  ScratchFrame frame(sc);
  uint32_t *keys, *vals, *skeys, *svals, *scell, *bb;
  float4 *xs, *XP, *yatt, *St, *CP, *z = nullptr;
  float *ws = nullptr, *Wt, *s0;
  int32_t* cst;
  int64_t *fb;
  const int64_t ncell = lb.cbase[P], nfine = lb.fbase[P];
  VMO_TRY(sc.alloc(&keys, K));
  VMO_TRY(sc.alloc(&vals, K));
  VMO_TRY(sc.alloc(&skeys, K));
  VMO_TRY(sc.alloc(&svals, K));
  VMO_TRY(sc.alloc(&scell, K));
  VMO_TRY(sc.alloc(&xs, K));
  VMO_TRY(sc.alloc(&yatt, K));
  if (lb.w) VMO_TRY(sc.alloc(&ws, K));
  VMO_TRY(sc.alloc(&St, ncell));
  VMO_TRY(sc.alloc(&CP, (size_t)((ncell + P) / 2 + 1) * (d == 4 ? 3 : 2)));
  VMO_TRY(sc.alloc(&XP, (size_t)((K + P + 1) / 2 + 1) * (d == 4 ? 3 : 2)));
  VMO_TRY(sc.alloc(&Wt, ncell));
  VMO_TRY(sc.alloc(&cst, nfine + P));
  VMO_TRY(sc.alloc(&bb, (size_t)2 * 8 * P));
  VMO_TRY(sc.alloc(&s0, P));
  if (lb.net_ptr) VMO_TRY(sc.alloc(&z, std::max<int64_t>(lb.nnets, 1)));
  fb = lb.fbase_dev.ptr;
  // levels whose problems all fit one sort tile are binned by one block per
  // problem (k_bin_small) when the tuning allows it
  int64_t kmax = 0;
  for (int p = 0; p < P; ++p) kmax = std::max(kmax, lb.vbase[p + 1] - lb.vbase[p]);
  bool bin1 = kmax <= std::min<int64_t>(kSortTile, g_tuning.small_bin_points.load(std::memory_order_relaxed));
  for (int p = 0; p < P && bin1; ++p) bin1 = (int64_t(1) << (d * lb.L[p])) <= kBinCells;
  if (bin1)
    dispatch_d(d, [&](auto DC) {
      constexpr int D = decltype(DC)::value;
      if (cudaFuncSetAttribute(k_bin_small<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BinSmem)) !=
          cudaSuccess) {
        (void)cudaGetLastError();
        bin1 = false;  // the device-wide sequence then
      }
    });
  SortSegments segs;
  bool segmented = P > 1;
  if (segmented && !bin1) VMO_TRY(make_sort_segments(lb.vbase, &segs, s, sc));
  const int nreset = 8 * P;
  launch(k_bbox_reset, grid_for(16 * P, kBlock), kBlock, 0, s, bb, 16 * P);
  VMO_LAUNCHED("bbox_reset");
  const float kappa = d == 2 ? 1.0f : (float)(d - 2);
  // step lengths s0 * decay^t: decay^t as the running double product, rounded
  // to fp32 (a table read by the step kernel at the level's step counter,
  // which k_keys advances)
  float* scale_tab;
  int32_t* tctr;
  VMO_TRY(sc.alloc(&scale_tab, iters));
  VMO_TRY(sc.alloc(&tctr, 1));
  launch(k_scale_tab, 1, 1, 0, s, iters, (double)o.decay, scale_tab);
  VMO_LAUNCHED("scale_tab");
  VMO_CUDA(cudaMemsetAsync(tctr, 0xFF, sizeof(int32_t), s));  // -1: k_keys advances it at every step
  vmo_status st = VMO_OK;
  SideStream ss;  // attraction stream of this call (none if it cannot be created)
  cudaStream_t side = ss.stream;
  cudaEvent_t ev_fork = ss.fork, ev_join = ss.join;
  dispatch_d(d, [&](auto DC) {
    constexpr int D = decltype(DC)::value;
    launch(k_bbox<D>, grid_for(K, kBlock), kBlock, 0, s, x, K, lb.vprob.ptr, bb);
    launch(k_step0<D>, grid_for(P, kBlock), kBlock, 0, s, bb, lb.prob.ptr, P, o.sigma, s0);
    cudaStream_t ms = s;  // stream of the steps
    // one step t of Algorithm 4 for every problem (only the parity of t and
    // whether it is the first step matter to the launches)
    auto step = [&](int t) -> vmo_status {
      ScratchFrame f2(sc);
      PdlScope pdl;  // every kernel of a step starts with pdl_wait()
      uint32_t* cur = bb + (t & 1) * 8 * P;
      uint32_t* nxt = bb + ((t + 1) & 1) * 8 * P;
      // attraction depends only on x: it runs on the side stream, overlapped
      // with the binning below, and joins before the step kernel
      cudaStream_t as = side ? side : ms;
      if (side) {
        cudaEventRecord(ev_fork, ms);
        cudaStreamWaitEvent(side, ev_fork, 0);
      }
      if (lb.adj_ptr) {
        launch(k_attract, grid_for(K, kBlock), kBlock, 0, as, lb.adj_ptr, lb.adj, lb.acost, x, K, yatt);
        if (lb.n_mid)
          launch(k_attract_warp, grid_for(lb.n_mid * 32, kBlock), kBlock, 0, as, lb.mid_list.ptr, lb.n_mid, lb.adj_ptr,
                 lb.adj, lb.acost, x, yatt);
        if (lb.n_heavy)
          launch(k_attract_block, (unsigned)lb.n_heavy, kBlock, 0, as, lb.heavy_list.ptr, lb.adj_ptr, lb.adj, lb.acost,
                 x, yatt);
      } else if (lb.net_ptr) {
        if (lb.nnets > 0) launch(k_net_center, grid_for(lb.nnets, kBlock), kBlock, 0, as, lb.net_ptr, lb.pins, lb.nnets, x, z);
        launch(k_attract_hyper, grid_for(K, kBlock), kBlock, 0, as, lb.vtx_ptr, lb.vnets, x, z, K, yatt);
      } else {
        cudaMemsetAsync(yatt, 0, K * sizeof(float4), as);
      }
      if (side) cudaEventRecord(ev_join, side);
      if (bin1) {
        launch(k_bin_small<D>, (unsigned)P, kSortThreads, sizeof(BinSmem), ms, x, lb.w, lb.prob.ptr, cur, nxt, tctr,
               keys_out && t == 0 ? keys : nullptr, svals, xs, ws, scell, cst, XP, St, Wt, CP);
        if (keys_out && t == 0) cudaMemcpyAsync(keys_out, keys, K * 4, cudaMemcpyDeviceToDevice, ms);
      } else {
        if (K >= kKeyItemsMin)
          launch(k_keys<D, 4>, grid_for((K + 3) / 4, kBlock), kBlock, 0, ms, x, K, lb.vprob.ptr, lb.prob.ptr, cur, keys,
                 vals, nxt, nreset, tctr);
        else
          launch(k_keys<D, 1>, grid_for(K, kBlock), kBlock, 0, ms, x, K, lb.vprob.ptr, lb.prob.ptr, cur, keys, vals, nxt,
                 nreset, tctr);
        if (keys_out && t == 0) cudaMemcpyAsync(keys_out, keys, K * 4, cudaMemcpyDeviceToDevice, ms);
        bool in_b = false;
        VMO_TRY(radix_sort_u32_pingpong(keys, vals, skeys, svals, K, D * lb.maxL, segmented ? &segs : nullptr, &in_b,
                                        ms, sc));
        if (!in_b) {  // sorted pairs are in (keys, vals): use them as (skeys, svals) from here on
          std::swap(keys, skeys);
          std::swap(vals, svals);
        }
        launch(k_gather<D>, grid_for(K, kBlock), kBlock, 0, ms, svals, skeys, K, x, lb.w, lb.vprob.ptr, lb.prob.ptr,
               cur, xs, ws, scell, cst, XP);
        launch(k_agg_finest<D>, grid_for(nfine, kBlock), kBlock, 0, ms, nfine, fb, P, lb.prob.ptr, xs, ws, cst, St, Wt,
               CP);
        for (int stp = 1; stp <= lb.maxL - 2; ++stp) {
          const int64_t* off = lb.aggoff.ptr + (size_t)stp * (P + 1);
          int64_t n = 0;
          for (int p = 0; p < P; ++p) {
            int l = lb.L[p] - stp;
            n += l > small_level_max(D) ? (int64_t(1) << (D * l)) : 0;
          }
          if (n == 0) continue;
          launch(k_agg_level<D>, grid_for(n, kBlock), kBlock, 0, ms, stp, off, P, n, lb.prob.ptr, St, Wt, CP);
        }
        if (lb.maxL >= 3) launch(k_agg_small<D>, (unsigned)P, kBlock, 0, ms, lb.prob.ptr, St, Wt, CP);
      }
      if (side) cudaStreamWaitEvent(ms, ev_join, 0);
      const bool timed = stats_timing();
      if (timed) stats_time_begin(ms);
      unsigned long long* icount = stats_interaction_counter();
      // few warps per SM: the far-field variant with two rows in flight
      const bool mlp = lb.threads <= g_tuning.small_step_threads.load(std::memory_order_relaxed);
      auto step_kernel = icount ? (mlp ? k_repulse_update<D, true, true> : k_repulse_update<D, true, false>)
                                : (mlp ? k_repulse_update<D, false, true> : k_repulse_update<D, false, false>);
      launch(step_kernel, grid_for(lb.threads, kStepBlock), kStepBlock, 0, ms, xs, ws, XP, svals, scell, cst, CP,
             yatt, lb.tbase.ptr, P, lb.prob.ptr, lb.threads, kappa, s0, scale_tab, tctr, step_override, x, y_out, nxt,
             icount);
      if (timed) stats_time_end(ms, (uint64_t)K);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "layout step", __FILE__, __LINE__);
      return VMO_OK;
    };
    // Steps are replayed from a CUDA graph of two steps (even and odd parity)
    // when the level runs plain steps; the host then issues one graph launch
    // per two steps instead of ~20 kernel launches per step.
    const bool graphs = ss.main && iters >= kGraphMinIters && !y_out && !keys_out && step_override <= 0.0f &&
                        !stats_timing() && !stats_interaction_counter();
    int t = 0;
    if (graphs) {
      // the steps run on the call's own stream, joined back to s at the end
      cudaEventRecord(ss.start, s);
      cudaStreamWaitEvent(ss.main, ss.start, 0);
      ms = ss.main;
    }
    ScratchOnStream on(sc, ms);  // scratch of a step follows the stream of the step
    if (graphs) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      const uint64_t before = g_launches.load();
      bool ok = cudaStreamBeginCapture(ms, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      vmo_status cst0 = VMO_OK;
      if (ok) {
        cst0 = step(0);
        if (cst0 == VMO_OK) cst0 = step(1);
        ok = cudaStreamEndCapture(ms, &g) == cudaSuccess && cst0 == VMO_OK;
      }
      if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
      const uint64_t per_graph = g_launches.load() - before;
      g_launches.fetch_sub(per_graph);  // captured, not launched: counted per replay below
      if (ok) {
        for (; t + 2 <= iters; t += 2) {
          cudaError_t e = cudaGraphLaunch(ge, ms);
          if (e != cudaSuccess) {
            st = cuda_fail(e, "cudaGraphLaunch (layout steps)", __FILE__, __LINE__);
            break;
          }
          g_launches.fetch_add(per_graph);
        }
      } else {
        (void)cudaGetLastError();  // fall back to direct launches
        if (cst0 != VMO_OK) st = cst0;
      }
      if (ge) cudaGraphExecDestroy(ge);
      if (g) cudaGraphDestroy(g);
    }
    for (; t < iters && st == VMO_OK; ++t) st = step(t);
    if (ms != s) {
      cudaEventRecord(ss.done, ms);
      cudaStreamWaitEvent(s, ss.done, 0);
    }
  });
  return st;
}

vmo_status coarsen_level(LevelBatch& lb, const uint64_t* seeds_dev, int j, int rounds, const int32_t* active_dev,
                         int32_t* mate, int32_t* anchor, int32_t* rank, std::vector<int64_t>& kc, cudaStream_t s,
                         Scratch& sc) {
  const int64_t K = lb.K;
  const int P = lb.P;
  ScratchFrame frame(sc);
  int32_t *prop, *isanc, *total;
  int64_t *kcd, *vb;
  VMO_TRY(sc.alloc(&prop, K));
  VMO_TRY(sc.alloc(&isanc, K));
  VMO_TRY(sc.alloc(&total, 1));
  VMO_TRY(sc.alloc(&kcd, P));
  VMO_TRY(sc.alloc(&vb, P + 1));
  VMO_CUDA(cudaMemcpyAsync(vb, lb.vbase.data(), (P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemsetAsync(mate, 0xFF, K * sizeof(int32_t), s));
  VMO_CUDA(cudaMemsetAsync(isanc, 0, K * sizeof(int32_t), s));
  for (int r = 0; r < rounds; ++r) {
    launch(k_propose, grid_for(K, kBlock), kBlock, 0, s, lb.adj_ptr, lb.adj, lb.acost, K, lb.vprob.ptr, lb.prob.ptr,
           active_dev, seeds_dev, j, r, mate, prop);
    if (lb.n_mid)
      launch(k_propose_wide, grid_for(lb.n_mid * 32, kBlock), kBlock, 0, s, lb.mid_list.ptr, lb.n_mid, 0, lb.adj_ptr,
             lb.adj, lb.acost, lb.vprob.ptr, lb.prob.ptr, active_dev, seeds_dev, j, r, mate, prop);
    if (lb.n_heavy)
      launch(k_propose_wide, (unsigned)lb.n_heavy, kBlock, 0, s, lb.heavy_list.ptr, lb.n_heavy, 1, lb.adj_ptr, lb.adj,
             lb.acost, lb.vprob.ptr, lb.prob.ptr, active_dev, seeds_dev, j, r, mate, prop);
    launch(k_resolve, grid_for(K, kBlock), kBlock, 0, s, prop, K, mate);
  }
  launch(k_anchor, grid_for(K, kBlock), kBlock, 0, s, lb.adj_ptr, lb.adj, K, mate, anchor, isanc);
  VMO_LAUNCHED("matching");
  VMO_TRY(scan_exclusive<int32_t>(isanc, rank, K, total, s, sc));
  launch(k_kc, grid_for(P, kBlock), kBlock, 0, s, rank, total, vb, P, K, kcd);
  VMO_LAUNCHED("kc");
  kc.resize(P);
  VMO_CUDA(cudaMemcpyAsync(kc.data(), kcd, P * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

// Builds the next (coarser) level from level `lb` for the problems with
// newbase[p] >= 0 (host), using the grouping (anchor, rank).
static vmo_status contract_level(LevelBatch& lb, const std::vector<int64_t>& newbase, int64_t Kc, const int32_t* anchor,
                                 const int32_t* rank, int32_t* pi, LevelBatch& out, cudaStream_t s, Scratch& sc) {
  const int64_t K = lb.K;
  const int P = lb.P;
  ScratchFrame frame(sc);
  int64_t* nb;
  VMO_TRY(sc.alloc(&nb, P));
  VMO_CUDA(cudaMemcpyAsync(nb, newbase.data(), P * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  launch(k_pi, grid_for(K, kBlock), kBlock, 0, s, anchor, rank, K, lb.vprob.ptr, lb.prob.ptr, nb, pi);
  VMO_LAUNCHED("pi");
  const int64_t n = lb.nadj;
  uint64_t *keys, *skeys;
  uint32_t *vals, *svals;
  int32_t *flag, *pos, *total;
  VMO_TRY(sc.alloc(&keys, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&skeys, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&vals, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&svals, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&flag, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&pos, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&total, 1));
  const uint64_t sentinel = (uint64_t)Kc * (uint64_t)Kc;
  launch(k_contract_keys, grid_for(K, kBlock), kBlock, 0, s, lb.adj_ptr, lb.adj, lb.acost, K, pi, (uint64_t)Kc, keys, vals);
  if (lb.n_mid)
    launch(k_contract_keys_warp, grid_for(lb.n_mid * 32, kBlock), kBlock, 0, s, lb.mid_list.ptr, lb.n_mid, lb.adj_ptr,
           lb.adj, lb.acost, pi, (uint64_t)Kc, keys, vals);
  if (lb.n_heavy)
    launch(k_contract_keys_block, (unsigned)lb.n_heavy, kBlock, 0, s, lb.heavy_list.ptr, lb.adj_ptr, lb.adj, lb.acost,
           pi, (uint64_t)Kc, keys, vals);
  VMO_LAUNCHED("contract_keys");
  VMO_TRY(radix_sort_u64(keys, vals, skeys, svals, n, bits_for(sentinel), s, sc));
  if (n > 0) {
    launch(k_run_flags, grid_for(n, kBlock), kBlock, 0, s, skeys, n, sentinel, flag);
    VMO_LAUNCHED("run_flags");
  }
  VMO_TRY(scan_exclusive<int32_t>(flag, pos, n, total, s, sc));
  int32_t nadj_c = 0;
  VMO_CUDA(cudaMemcpyAsync(&nadj_c, total, 4, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  VMO_TRY(out.own_adj_ptr.resize((size_t)Kc + 1));
  VMO_TRY(out.own_adj.resize(std::max<int32_t>(nadj_c, 1)));
  VMO_TRY(out.own_acost.resize(std::max<int32_t>(nadj_c, 1)));
  VMO_TRY(out.own_w.resize((size_t)std::max<int64_t>(Kc, 1)));
  double* wsum;
  VMO_TRY(sc.alloc(&wsum, std::max<int64_t>(Kc, 1)));
  VMO_CUDA(cudaMemsetAsync(out.own_adj_ptr.ptr, 0, (Kc + 1) * sizeof(int32_t), s));
  VMO_CUDA(cudaMemsetAsync(wsum, 0, std::max<int64_t>(Kc, 1) * sizeof(double), s));
  if (n > 0) {
    launch(k_emit_coarse, grid_for(n, kBlock), kBlock, 0, s, skeys, svals, n, flag, pos, (uint64_t)Kc, out.own_adj.ptr,
                                                         out.own_acost.ptr, out.own_adj_ptr.ptr);
    VMO_LAUNCHED("emit_coarse");
  }
  VMO_TRY(scan_exclusive<int32_t>(out.own_adj_ptr.ptr, out.own_adj_ptr.ptr, Kc, total, s, sc));
  launch(k_set_last, 1, 1, 0, s, out.own_adj_ptr.ptr, Kc, total);
  launch(k_coarse_w, grid_for(K, kBlock), kBlock, 0, s, lb.w, pi, K, wsum);
  if (Kc > 0) launch(k_round_w, grid_for(Kc, kBlock), kBlock, 0, s, wsum, Kc, out.own_w.ptr);
  VMO_LAUNCHED("coarse_w");
  out.K = Kc;
  out.adj_ptr = out.own_adj_ptr.ptr;
  out.adj = out.own_adj.ptr;
  out.acost = out.own_acost.ptr;
  out.w = out.own_w.ptr;
  out.nadj = nadj_c;
  return VMO_OK;
}

vmo_status build_hierarchy(LevelBatch& fine, const LayoutOptions& o, const std::vector<uint64_t>& seeds,
                           int match_rounds, int coarse_min, bool multilevel, Hierarchy& H, cudaStream_t s,
                           Scratch& sc) {
  std::vector<LevelBatch*>& levels = H.levels;
  std::vector<std::unique_ptr<LevelBatch>>& owned = H.owned;
  std::vector<int32_t*>& pis = H.pis;
  std::vector<std::vector<uint64_t>>& lseeds = H.seeds;
  levels.push_back(&fine);
  lseeds.push_back(seeds);
  const bool graph = fine.adj_ptr != nullptr;
  while (multilevel && graph && levels.size() < 41) {
    LevelBatch& cur = *levels.back();
    const int P = cur.P;
    std::vector<int32_t> active(P);
    bool any = false;
    for (int p = 0; p < P; ++p) {
      active[p] = (cur.vbase[p + 1] - cur.vbase[p]) > coarse_min ? 1 : 0;
      any = any || active[p];
    }
    if (!any) break;
    int32_t *act, *mate, *anchor, *rank, *pi;
    uint64_t* sd;
    VMO_TRY(sc.alloc(&act, P));
    VMO_TRY(sc.alloc(&sd, P));
    VMO_TRY(sc.alloc(&mate, cur.K));
    VMO_TRY(sc.alloc(&anchor, cur.K));
    VMO_TRY(sc.alloc(&rank, cur.K));
    VMO_TRY(sc.alloc(&pi, cur.K));
    VMO_CUDA(cudaMemcpyAsync(act, active.data(), P * 4, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaMemcpyAsync(sd, lseeds.back().data(), P * 8, cudaMemcpyHostToDevice, s));
    std::vector<int64_t> kc;
    VMO_TRY(coarsen_level(cur, sd, (int)levels.size() - 1, match_rounds, act, mate, anchor, rank, kc, s, sc));
    std::vector<int64_t> newbase(P, -1);
    auto nxt = std::make_unique<LevelBatch>();
    nxt->vbase.push_back(0);
    std::vector<uint64_t> nseeds;
    for (int p = 0; p < P; ++p) {
      int64_t k = cur.vbase[p + 1] - cur.vbase[p];
      if (!active[p] || (double)kc[p] > 0.95 * (double)k) continue;
      newbase[p] = nxt->vbase.back();
      nxt->vbase.push_back(nxt->vbase.back() + kc[p]);
      nxt->src.push_back(cur.src[p]);
      nseeds.push_back(lseeds.back()[p]);
    }
    nxt->P = (int32_t)nxt->src.size();
    if (nxt->P == 0) break;
    int64_t Kc = nxt->vbase.back();
    VMO_TRY(contract_level(cur, newbase, Kc, anchor, rank, pi, *nxt, s, sc));
    VMO_TRY(level_setup(*nxt, o.d, o.occupancy, s));
    pis.push_back(pi);
    levels.push_back(nxt.get());
    lseeds.push_back(nseeds);
    owned.push_back(std::move(nxt));
  }
  return VMO_OK;
}

// Host tables of level j's start: which problems start here (not present one
// level up) and, for the others, the scale (k_f / k_c)^(1/d) of the
// prolongation.
static void prolong_tables(const Hierarchy& H, int j, int d, std::vector<int32_t>& start, std::vector<float>& fac) {
  const std::vector<LevelBatch*>& levels = H.levels;
  const int nl = (int)levels.size();
  const LevelBatch& cur = *levels[j];
  const int P = cur.P;
  start.assign(P, 1);
  fac.assign(P, -1.0f);
  if (j + 1 < nl) {
    const LevelBatch& up = *levels[j + 1];
    size_t q = 0;
    for (int p = 0; p < P && q < up.src.size(); ++p) {
      if (cur.src[p] == up.src[q]) {
        start[p] = 0;
        double kf = (double)(cur.vbase[p + 1] - cur.vbase[p]);
        double kcq = (double)(up.vbase[q + 1] - up.vbase[q]);
        fac[p] = (float)std::pow(kf / kcq, 1.0 / d);
        ++q;
      }
    }
  }
}

// Level j's start from device tables (start flags, scales, seeds of its
// problems): initial coordinates for the problems that start here, the
// prolongation of xc for the others.
static vmo_status prolong_level_dev(const Hierarchy& H, int j, int d, const float4* xc, float4* xj,
                                    const int32_t* st, const float* fc, const uint64_t* sd, cudaStream_t s) {
  LevelBatch& cur = *H.levels[j];
  VMO_TRY(init_coords_level(cur, d, sd, xj, st, s));
  if (xc && cur.K > 0) {
    launch(k_prolong, grid_for(cur.K, kBlock), kBlock, 0, s, xc, H.pis[j], cur.K, cur.vprob.ptr, cur.prob.ptr, fc, sd,
           j, d, xj);
    VMO_LAUNCHED("prolong");
  }
  return VMO_OK;
}

vmo_status prolong_level(const Hierarchy& H, int j, int d, const float4* xc, float4* xj, cudaStream_t s,
                         Scratch& sc) {
  const int P = H.levels[j]->P;
  std::vector<int32_t> start;
  std::vector<float> fac;
  prolong_tables(H, j, d, start, fac);
  int32_t* st;
  float* fc;
  uint64_t* sd;
  VMO_TRY(sc.alloc(&st, P));
  VMO_TRY(sc.alloc(&fc, P));
  VMO_TRY(sc.alloc(&sd, P));
  VMO_CUDA(cudaMemcpyAsync(st, start.data(), P * 4, cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(fc, fac.data(), P * 4, cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(sd, H.seeds[j].data(), P * 8, cudaMemcpyHostToDevice, s));
  VMO_TRY(prolong_level_dev(H, j, d, xc, xj, st, fc, sd, s));
  VMO_CUDA(cudaStreamSynchronize(s));  // host vectors above must outlive the copies
  return VMO_OK;
}

vmo_status layout_multilevel(LevelBatch& fine, const LayoutOptions& o, const std::vector<uint64_t>& seeds,
                             int match_rounds, int coarse_min, bool multilevel, float4* x, cudaStream_t s,
                             Scratch& sc) {
  Hierarchy H;
  VMO_TRY(build_hierarchy(fine, o, seeds, match_rounds, coarse_min, multilevel, H, s, sc));
  // the start tables of every level uploaded at once, so that the levels are
  // then queued without waiting for the device
  const int nl = (int)H.levels.size();
  std::vector<int64_t> tb(nl + 1, 0);
  for (int j = 0; j < nl; ++j) tb[j + 1] = tb[j] + H.levels[j]->P;
  std::vector<int32_t> start_all((size_t)tb[nl]);
  std::vector<float> fac_all((size_t)tb[nl]);
  std::vector<uint64_t> seed_all((size_t)tb[nl]);
  for (int j = 0; j < nl; ++j) {
    std::vector<int32_t> st;
    std::vector<float> fc;
    prolong_tables(H, j, o.d, st, fc);
    std::copy(st.begin(), st.end(), start_all.begin() + tb[j]);
    std::copy(fc.begin(), fc.end(), fac_all.begin() + tb[j]);
    std::copy(H.seeds[j].begin(), H.seeds[j].end(), seed_all.begin() + tb[j]);
  }
  int32_t* st_d;
  float* fc_d;
  uint64_t* sd_d;
  VMO_TRY(sc.alloc(&st_d, std::max<int64_t>(tb[nl], 1)));
  VMO_TRY(sc.alloc(&fc_d, std::max<int64_t>(tb[nl], 1)));
  VMO_TRY(sc.alloc(&sd_d, std::max<int64_t>(tb[nl], 1)));
  VMO_CUDA(cudaMemcpyAsync(st_d, start_all.data(), tb[nl] * 4, cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(fc_d, fac_all.data(), tb[nl] * 4, cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(sd_d, seed_all.data(), tb[nl] * 8, cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaStreamSynchronize(s));  // the host tables must outlive the copies
  // layout from the coarsest level down
  float4* xc = nullptr;
  for (int j = nl - 1; j >= 0; --j) {
    LevelBatch& cur = *H.levels[j];
    float4* xj = (j == 0) ? x : nullptr;
    if (!xj) VMO_TRY(sc.alloc(&xj, std::max<int64_t>(cur.K, 1)));
    VMO_TRY(prolong_level_dev(H, j, o.d, xc, xj, st_d + tb[j], fc_d + tb[j], sd_d + tb[j], s));
    VMO_TRY(layout_level(cur, o, xj, o.iters, -1.0f, nullptr, nullptr, s, sc));
    xc = xj;
  }
  return VMO_OK;
}

}  // namespace vmo
