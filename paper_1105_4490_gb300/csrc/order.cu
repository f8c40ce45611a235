// Recursive geometric bisection (Sec. 3 and 4.2): 2-means by k-means++
// (Algorithm 5, m = 2), vertex separator (Algorithm 7) and the recursive BBD /
// SBD permutation.
//
// The recursion is processed level by level: every active node of every
// problem of a batch is handled by the same launches.  Nodes are identified by
// their heap number (root 1, children 2h and 2h+1), which keys the k-means++
// draws, so a node's result does not depend on which other nodes share its
// launches or on their order in the node table.
//
// Exactness: every floating point decision (nearest centre, plane distance)
// is made in fp32 with explicitly rounded intrinsics in a fixed order; the
// centre of a cluster is the mean of its points summed exactly in 64-bit
// fixed point; the D^2 sampling of k-means++ uses exact integer prefix sums.
// Given the same coordinates the result is bit-identical to a sequential
// implementation of the same arithmetic.
#include <algorithm>

#include "order.cuh"

namespace vmo {

namespace {

constexpr int kBlock = 256;

template <int D>
__device__ inline float plane_dist(const float4& x, const float4& r, float delta) {
  float acc = 0.0f;
#pragma unroll
  for (int m = 0; m < D; ++m) acc = __fadd_rn(acc, __fmul_rn(comp(x, m), comp(r, m)));
  return fabsf(__fsub_rn(acc, delta));
}

template <int D>
__device__ inline void plane_of(const float4& z1, const float4& z2, float4* r, float* delta) {
  float rr[4] = {0.f, 0.f, 0.f, 0.f};
  float dl = 0.0f;
#pragma unroll
  for (int m = 0; m < D; ++m) {
    rr[m] = __fsub_rn(comp(z2, m), comp(z1, m));
    float mid = __fmul_rn(0.5f, __fadd_rn(comp(z1, m), comp(z2, m)));
    dl = __fadd_rn(dl, __fmul_rn(mid, rr[m]));
  }
  *r = make_float4(rr[0], rr[1], rr[2], rr[3]);
  *delta = dl;
}

// Warp sum of a 64-bit value.
__device__ inline unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_node_reset(NodeDev* __restrict__ nodes, int N) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  NodeDev& nd = nodes[s];
  nd.maxabs = 0u;
  nd.state = 0;
  nd.changed = 0;
  for (int m = 0; m < 4; ++m) { nd.S1[m] = 0; nd.S2[m] = 0; }
  nd.n1 = nd.n2 = 0;
  nd.c1 = nd.c2 = nd.c3 = 0;
  nd.child1 = nd.child2 = nd.child3 = -1;
}

// Positions per thread of the per-position kernels of the 2-means (k_maxabs,
// k_dsq, k_seed2) on large inputs: all of a thread's loads issued together.
constexpr int kPosItems = 4;
constexpr int64_t kPosItemsMin = int64_t(1) << 20;

template <int D, int U>
__global__ void k_maxabs(const float4* __restrict__ xo, const int32_t* __restrict__ seg, int64_t n,
                         NodeDev* __restrict__ nodes) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x;
  // every load in flight together (the coordinates are read whether or not
  // the position is active)
  int sv[U];
  float4 xv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t i = i0 + (int64_t)u * blockDim.x;
    const bool in = i < n;
    sv[u] = in ? seg[i] : -1;
    xv[u] = in ? xo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  uint32_t mx[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    mx[u] = 0;
    if (sv[u] >= 0) {
#pragma unroll
      for (int m = 0; m < D; ++m) mx[u] = max(mx[u], __float_as_uint(fabsf(comp(xv[u], m))));
    }
  }
  // a block of one node (the top of the recursion, where every warp would
  // otherwise send an atomic to the same word) adds its maximum once
  __shared__ int s_first;
  __shared__ uint32_t s_max;
  if (threadIdx.x == 0) { s_first = sv[0]; s_max = 0u; }
  __syncthreads();
  const int s0 = s_first;
  bool same = true;
#pragma unroll
  for (int u = 0; u < U; ++u) same = same && (sv[u] < 0 || sv[u] == s0);
  if (__syncthreads_and(same) && s0 >= 0) {
    uint32_t m = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) m = max(m, mx[u]);
    const uint32_t wm = __reduce_max_sync(0xffffffffu, m);
    if (lane_id() == 0) atomicMax(&s_max, wm);
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&nodes[s0].maxabs, s_max);
    return;
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const unsigned peers = __match_any_sync(0xffffffffu, sv[u]);
    const uint32_t wm = __reduce_max_sync(peers, mx[u]);
    if (sv[u] >= 0 && (int)lane_id() == __ffs(peers) - 1) atomicMax(&nodes[sv[u]].maxabs, wm);
  }
}

// k-means++ first centre: point floor(size * r0 / 2^64) of the node.
__global__ void k_seed1(NodeDev* __restrict__ nodes, int N, const float4* __restrict__ xo,
                        const uint64_t* __restrict__ seeds) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  NodeDev& nd = nodes[s];
  nd.e = exponent_of(nd.maxabs);
  uint64_t r0 = rand64(seeds[nd.prob] ^ kTagKmeans, nd.heap, 0);
  uint64_t i0 = scale_draw((uint64_t)nd.size, r0);
  nd.z1 = xo[nd.off + (int64_t)i0];
}

template <int D, int U>
__global__ void k_dsq(const float4* __restrict__ xo, const int32_t* __restrict__ seg, int64_t n,
                      const NodeDev* __restrict__ nodes, unsigned long long* __restrict__ dval) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x;
  int sv[U];
  float4 xv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {  // every load in flight together
    const int64_t i = i0 + (int64_t)u * blockDim.x;
    const bool in = i < n;
    sv[u] = in ? seg[i] : -1;
    xv[u] = in ? xo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t i = i0 + (int64_t)u * blockDim.x;
    if (i >= n) break;
    unsigned long long v = 0;
    if (sv[u] >= 0) {
      const NodeDev& nd = nodes[sv[u]];
      float dd = sqdist32<D>(xv[u], nd.z1);
      float sc = __fmul_rn(dd, exp2i_f(34 - 2 * nd.e));
      v = (unsigned long long)floorf(sc);
    }
    dval[i] = v;
  }
}

// Second centre: the first point whose inclusive prefix of D exceeds
// floor(total * r1 / 2^64); a node whose total is 0 is not split.
template <int D, int U>
__global__ void k_seed2(const float4* __restrict__ xo, const int32_t* __restrict__ seg, int64_t n,
                        const unsigned long long* __restrict__ dval, const unsigned long long* __restrict__ dpre,
                        NodeDev* __restrict__ nodes, const uint64_t* __restrict__ seeds) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x;
  int sv[U];
  unsigned long long pv[U], vv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {  // every load in flight together
    const int64_t i = i0 + (int64_t)u * blockDim.x;
    const bool in = i < n;
    sv[u] = in ? seg[i] : -1;
    pv[u] = in ? dpre[i] : 0ull;
    vv[u] = in ? dval[i] : 0ull;
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t i = i0 + (int64_t)u * blockDim.x;
    const int s = sv[u];
    if (s < 0) continue;
    NodeDev& nd = nodes[s];
    unsigned long long base = nd.off > 0 ? dpre[nd.off - 1] : 0ull;
    unsigned long long total = dpre[nd.off + nd.size - 1] - base;
    if (total == 0) {
      if (i == nd.off) nd.state = 2;
      continue;
    }
    uint64_t r1 = rand64(seeds[nd.prob] ^ kTagKmeans, nd.heap, 1);
    unsigned long long thr = scale_draw(total, r1);
    unsigned long long pre = pv[u] - base;
    unsigned long long prev = pre - vv[u];
    if (prev <= thr && thr < pre) nd.z2 = xo[i];
  }
}

// One Lloyd assignment: label 1 iff ||x - z1||^2 <= ||x - z2||^2 (fp32),
// change detection against the previous labels, and exact fixed-point sums
// q(x) = rint(x * 2^P), P = 30 - e, of each cluster.
// Lloyd assignment (Algorithm 5) with exact fixed-point centroid sums: every
// block takes items x blockDim consecutive positions (items <= kAssignItems,
// fewer when the positions would not give every SM a few blocks).  A block whose
// positions all lie in one node (the common case above the deepest levels)
// sums in registers and adds its totals with one set of atomics; other blocks
// aggregate per warp and (node, label).  Integer sums make the result
// independent of the order of the additions.
constexpr int kAssignItems = 8;

template <int D>
__device__ inline void assign_one(const float4* __restrict__ xo, int64_t i, const NodeDev& nd, int it,
                                  uint8_t* __restrict__ lab, int final_pass, uint8_t& l, long long* q, bool& chg) {
  float4 x = xo[i];
  l = (sqdist32<D>(x, nd.z1) <= sqdist32<D>(x, nd.z2)) ? 1 : 2;
  if (!final_pass) {
    if (it > 0 && l != lab[i]) chg = true;
    float sc = exp2i_f(30 - nd.e);
#pragma unroll
    for (int m = 0; m < D; ++m) q[m] = __float2ll_rn(__fmul_rn(comp(x, m), sc));
  }
  lab[i] = l;
}

// Replicas of the sums of the first kRepNodes nodes: on large inputs the
// blocks of a node add into kRepR copies (by block index) instead of one, so
// that the atomics of thousands of blocks on the top levels do not queue on
// the same addresses; k_fold_reps adds the copies into the node.  Ten sums per
// node in the order of NodeDev: S1[0..3], S2[0..3], n1, n2.
constexpr int kRepR = 32;
constexpr int kRepNodes = 256;
constexpr int64_t kRepMinPositions = 1 << 19;

__global__ void k_fold_reps(NodeDev* __restrict__ nodes, int N, unsigned long long* __restrict__ rep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * 10) return;
  const int s = i / 10, t = i % 10;
  unsigned long long sum = 0;
  for (int r = 0; r < kRepR; ++r) {
    unsigned long long* p = rep + ((int64_t)s * kRepR + r) * 10 + t;
    sum += *p;
    *p = 0;
  }
  reinterpret_cast<unsigned long long*>(&nodes[s].S1[0])[t] += sum;
}

template <int D, int ITEMS>
__global__ void k_assign(const float4* __restrict__ xo, const int32_t* __restrict__ seg, int64_t n, int it,
                         NodeDev* __restrict__ nodes, uint8_t* __restrict__ lab, int final_pass,
                         unsigned long long* __restrict__ rep) {
  constexpr int items = ITEMS;
  __shared__ int s_first;
  __shared__ unsigned long long red[kBlock / 32][2 * 4 + 2];
  const int64_t base = (int64_t)blockIdx.x * (items * blockDim.x);
  if (threadIdx.x == 0) s_first = base < n ? seg[base] : -1;
  __syncthreads();
  const int s0 = s_first;
  // every load of the thread's positions (node, coordinates, previous label)
  // issued before the barrier, so that they are in flight together
  int sv[ITEMS];
  float4 xv[ITEMS];
  uint8_t lv[ITEMS];
  const bool prev = it > 0 && !final_pass;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int64_t i = base + k * blockDim.x + threadIdx.x;
    const bool in = k < items && i < n;
    sv[k] = in ? seg[i] : -1;
    xv[k] = in ? xo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    lv[k] = in && prev ? lab[i] : 0;
  }
  bool same = true;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int64_t i = base + k * blockDim.x + threadIdx.x;
    same = same && (k >= items || i >= n || sv[k] == s0);
  }
  const bool uniform = __syncthreads_and(same) && s0 >= 0;
  if (uniform) {
    NodeDev& nd = nodes[s0];
    const int st = nd.state;
    if (!(final_pass ? (st != 2) : (st == 0))) return;
    // per thread: the first cluster's sums and the totals of all its items
    // (the second cluster's are their difference); a fixed-point value
    // rint(x 2^(30-e)) has |q| <= 2^30 - 64 (x 2^(30-e) is an fp32 value
    // below 2^30), so it is converted as 32 bits and two of them are added in
    // 32 bits before each 64-bit addition
    long long S1[4] = {0, 0, 0, 0}, T[4] = {0, 0, 0, 0};
    int t32[4] = {0, 0, 0, 0}, s32[4] = {0, 0, 0, 0};
    int c1 = 0, cnt = 0;
    bool chg = false;
    const float sc = exp2i_f(30 - nd.e);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const int64_t i = base + k * blockDim.x + threadIdx.x;
      if (k < items && i < n) {
        const float4 x = xv[k];
        const uint8_t l = (sqdist32<D>(x, nd.z1) <= sqdist32<D>(x, nd.z2)) ? 1 : 2;
        const bool first = l == 1;  // selects, not a computed index: the sums stay in registers
        if (!final_pass) {
          if (prev && l != lv[k]) chg = true;
#pragma unroll
          for (int m = 0; m < D; ++m) {
            const int q = __float2int_rn(__fmul_rn(comp(x, m), sc));
            t32[m] += q;
            s32[m] += first ? q : 0;
          }
        }
        lab[i] = l;
        c1 += first ? 1 : 0;
        ++cnt;
      }
      if ((k & 1) || k == ITEMS - 1) {  // a pair (or the last item) into the 64-bit sums
#pragma unroll
        for (int m = 0; m < D; ++m) {
          T[m] += t32[m];
          S1[m] += s32[m];
          t32[m] = s32[m] = 0;
        }
      }
    }
    // block totals: counts, sums (not in the final pass) and the change flag
    const int warp = threadIdx.x >> 5, lane = lane_id();
    unsigned long long v[2 * 4 + 2];
    v[0] = warp_sum64((unsigned long long)c1);
    v[1] = warp_sum64((unsigned long long)(cnt - c1));
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      v[2 + m] = m < D && !final_pass ? warp_sum64((unsigned long long)S1[m]) : 0ull;
      v[6 + m] = m < D && !final_pass ? warp_sum64((unsigned long long)(T[m] - S1[m])) : 0ull;
    }
    const bool any_chg = __any_sync(0xffffffffu, chg);
    if (lane == 0) {
#pragma unroll
      for (int t = 0; t < 2 * 4 + 2; ++t) red[warp][t] = v[t];
    }
    const bool block_chg = __syncthreads_or(any_chg);
    if (threadIdx.x == 0) {
      unsigned long long tot[2 * 4 + 2];
#pragma unroll
      for (int t = 0; t < 2 * 4 + 2; ++t) {
        tot[t] = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot[t] += red[w][t];
      }
      if (block_chg) nd.changed = 1;
      unsigned long long* acc = rep ? rep + ((int64_t)s0 * kRepR + (blockIdx.x & (kRepR - 1))) * 10
                                    : reinterpret_cast<unsigned long long*>(&nd.S1[0]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (tot[h] == 0) continue;
        if (!final_pass) {
#pragma unroll
          for (int m = 0; m < D; ++m) atomicAdd(acc + 4 * h + m, tot[2 + 4 * h + m]);
        }
        atomicAdd(acc + 8 + h, tot[h]);
      }
    }
    return;
  }
  // positions of several nodes: per warp and (node, label)
#pragma unroll 1
  for (int k = 0; k < items; ++k) {
    const int64_t i = base + k * blockDim.x + threadIdx.x;
    const int s = sv[k];
    bool act = false;
    uint8_t l = 0;
    long long q[4] = {0, 0, 0, 0};
    if (s >= 0) {
      NodeDev& nd = nodes[s];
      const int st = nd.state;
      act = final_pass ? (st != 2) : (st == 0);
      if (act) {
        bool chg = false;
        assign_one<D>(xo, i, nd, it, lab, final_pass, l, q, chg);
        if (chg) nd.changed = 1;
      }
    }
    const int key = act ? s * 2 + (l - 1) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key < 0) continue;
    const int leader = __ffs(peers) - 1;
    const unsigned long long cnt = __popc(peers);
    unsigned long long sum[4] = {0, 0, 0, 0};
    if (!final_pass) {
#pragma unroll
      for (int m = 0; m < D; ++m) {
        unsigned long long acc = 0;
        for (unsigned b = peers; b; b &= b - 1) {
          int src = __ffs(b) - 1;
          acc += (unsigned long long)__shfl_sync(peers, (unsigned long long)q[m], src);
        }
        sum[m] = acc;
      }
    }
    if ((int)lane_id() != leader) continue;
    NodeDev& nd = nodes[s];
    if (!final_pass) {
      unsigned long long* Sx = (unsigned long long*)(l == 1 ? nd.S1 : nd.S2);
#pragma unroll
      for (int m = 0; m < D; ++m) atomicAdd(&Sx[m], sum[m]);
    }
    atomicAdd((unsigned long long*)(l == 1 ? &nd.n1 : &nd.n2), cnt);
  }
}

// Positions per thread: at most the tuned cap (kAssignItems by default), and
// few enough that the blocks fill every SM about four times over.
inline int assign_items(int64_t n) {
  int items = std::min(kAssignItems, std::max(1, g_tuning.assign_items.load(std::memory_order_relaxed)));
  while (items > 1 && n < (int64_t)items * kBlock * 152 * 4) items >>= 1;
  return items;
}

inline unsigned assign_grid(int64_t n) {
  const int64_t per = (int64_t)kBlock * assign_items(n);
  return (unsigned)std::max<int64_t>(1, (n + per - 1) / per);
}

// One Lloyd assignment launch with the instantiation for assign_items(n).
template <int D>
void launch_assign(int64_t n, cudaStream_t s, const float4* xo, const int32_t* seg, int it, NodeDev* nodes,
                   uint8_t* lab, int final_pass, unsigned long long* rep) {
  const unsigned g = assign_grid(n);
  switch (assign_items(n)) {
    case 1: launch(k_assign<D, 1>, g, kBlock, 0, s, xo, seg, n, it, nodes, lab, final_pass, rep); break;
    case 2: launch(k_assign<D, 2>, g, kBlock, 0, s, xo, seg, n, it, nodes, lab, final_pass, rep); break;
    case 4: launch(k_assign<D, 4>, g, kBlock, 0, s, xo, seg, n, it, nodes, lab, final_pass, rep); break;
    default: launch(k_assign<D, 8>, g, kBlock, 0, s, xo, seg, n, it, nodes, lab, final_pass, rep); break;
  }
}

// Centre update: z = fp32((double(sum) / count) * 2^-P); a node whose labels
// did not change is converged.
template <int D>
__global__ void k_update(NodeDev* __restrict__ nodes, int N, int it) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  NodeDev& nd = nodes[s];
  if (nd.state != 0) return;
  if (it > 0 && !nd.changed) {
    nd.state = 1;
  } else {
    double inv = __longlong_as_double((long long)(1023 - (30 - nd.e)) << 52);  // 2^-P
    float z1[4] = {nd.z1.x, nd.z1.y, nd.z1.z, nd.z1.w};
    float z2[4] = {nd.z2.x, nd.z2.y, nd.z2.z, nd.z2.w};
    for (int m = 0; m < D; ++m) {
      if (nd.n1 > 0) z1[m] = __double2float_rn(__dmul_rn(__ddiv_rn(__ll2double_rn(nd.S1[m]), (double)nd.n1), inv));
      if (nd.n2 > 0) z2[m] = __double2float_rn(__dmul_rn(__ddiv_rn(__ll2double_rn(nd.S2[m]), (double)nd.n2), inv));
    }
    nd.z1 = make_float4(z1[0], z1[1], z1[2], z1[3]);
    nd.z2 = make_float4(z2[0], z2[1], z2[2], z2[3]);
  }
  nd.changed = 0;
  for (int m = 0; m < 4; ++m) { nd.S1[m] = 0; nd.S2[m] = 0; }
  nd.n1 = nd.n2 = 0;
}

__global__ void k_count_active(const NodeDev* __restrict__ nodes, int N, int* __restrict__ out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < N && nodes[s].state == 0) atomicAdd(out, 1);
}

__global__ void k_clear_counts(NodeDev* __restrict__ nodes, int N) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  nodes[s].n1 = nodes[s].n2 = 0;
}

// Per-vertex record of the separator phase, one 8-byte word so that a
// neighbour costs one load: high word (node << 2) | label, where label is the
// vertex's final 2-means label (1 or 2) in a split node of this level and 0
// otherwise (also for vertices already placed); low word the bits of the
// plane distance s = |x.r - delta| (s >= 0, so its bits order like its value).
__device__ __forceinline__ uint64_t vrec_make(int node, uint32_t label, float sdist) {
  return ((uint64_t)(((uint32_t)node << 2) | label) << 32) | __float_as_uint(sdist);
}
__device__ __forceinline__ uint32_t vrec_label(uint64_t r) { return (uint32_t)(r >> 32) & 3u; }
__device__ __forceinline__ float vrec_s(uint64_t r) { return __uint_as_float((uint32_t)r); }
// the high word a neighbour in node s with the label other than l (l in {1, 2}) carries
__device__ __forceinline__ uint32_t vrec_other(int s, uint32_t l) { return ((uint32_t)s << 2) | (3u - l); }

template <int D>
__global__ void k_vertex_state(const float4* __restrict__ xo, const int32_t* __restrict__ ord,
                               const int32_t* __restrict__ seg, int64_t n, const NodeDev* __restrict__ nodes,
                               const uint8_t* __restrict__ lab, uint64_t* __restrict__ vrec) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = seg[i];
  const int32_t v = ord[i];   // loads in flight together
  const float4 x = xo[i];
  const uint8_t li = lab[i];
  if (s < 0) return;
  const NodeDev& nd = nodes[s];
  bool split = nd.state != 2 && nd.n1 > 0 && nd.n2 > 0;
  float4 r;
  float delta;
  plane_of<D>(nd.z1, nd.z2, &r, &delta);
  vrec[v] = vrec_make(s, split ? li : 0u, plane_dist<D>(x, r, delta));
}

// Sizes of V1, V2, V3 of the positions of a block added to their nodes' c1,
// c2, c3: once per block when every position of the block lies in one node
// (the top of the recursion, where a level's positions would otherwise all
// hit the same three counters), else once per warp and (node, label).
// Every thread of the block calls it (s < 0 or l == 0: nothing to count).
__device__ void count_labels(int s, uint8_t l, NodeDev* __restrict__ nodes) {
  __shared__ int s_first, s_cnt[3];
  if (threadIdx.x == 0) s_first = s;  // the node of the block's first position
  if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const int s0 = s_first;
  const bool uniform = __syncthreads_and(s < 0 || s == s0) && s0 >= 0;
  const int key = (s >= 0 && l != 0) ? s * 4 + l : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const bool leader = key >= 0 && (int)lane_id() == __ffs(peers) - 1;
  if (uniform) {
    if (leader) atomicAdd(&s_cnt[l - 1], (int)__popc(peers));
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_cnt[0]) atomicAdd(&nodes[s0].c1, s_cnt[0]);
      if (s_cnt[1]) atomicAdd(&nodes[s0].c2, s_cnt[1]);
      if (s_cnt[2]) atomicAdd(&nodes[s0].c3, s_cnt[2]);
    }
  } else if (leader) {
    int* c = l == 1 ? &nodes[s].c1 : (l == 2 ? &nodes[s].c2 : &nodes[s].c3);
    atomicAdd(c, (int)__popc(peers));
  }
}

// A position's contribution to the scan that places the parts: 1 in the low
// word for V1, 1 in the high word for V2, nothing for V3 or a node that is
// not split (label 0).
__device__ __forceinline__ unsigned long long part_count(uint8_t l) {
  return l == 1 ? 1ull : (l == 2 ? (1ull << 32) : 0ull);
}

// Order-free form of the separator loop of Algorithm 7 (mu = identity):
// v joins the separator iff a neighbour w in the same node carries the other
// label and (s(v), v) < (s(w), w).
__global__ void k_separator(const int32_t* __restrict__ ord, const int32_t* __restrict__ seg, int64_t n,
                            const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                            const uint64_t* __restrict__ vrec, NodeDev* __restrict__ nodes,
                            uint8_t* __restrict__ labf, unsigned long long* __restrict__ pk) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int s = i < n ? seg[i] : -1;
  uint8_t l = 0;
  if (s >= 0) {
    const int32_t v = ord[i];
    const uint64_t rv = vrec[v];
    l = (uint8_t)vrec_label(rv);
    if (l != 0) {
      // any neighbour decides, so four are tested at a time with all their
      // loads issued together
      const float sv = vrec_s(rv);
      const uint32_t other = vrec_other(s, l);
      const int32_t t1 = adj_ptr[v + 1];
      bool hit = false;
      for (int32_t t = adj_ptr[v]; t < t1 && !hit; t += 4) {
        int32_t w[4];
        uint64_t rw[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = t + u < t1 ? adj[t + u] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) rw[u] = w[u] >= 0 ? vrec[w[u]] : 0ull;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (w[u] < 0 || (uint32_t)(rw[u] >> 32) != other) continue;  // not in this node, or on the same side
          const float sw = vrec_s(rw[u]);
          if (sv < sw || (sv == sw && v < w[u])) hit = true;
        }
      }
      if (hit) l = 3;
    }
    labf[i] = l;
  }
  if (i < n) pk[i] = part_count(l);
  count_labels(s, l, nodes);
}

// With a strengthened diagonal (Algorithm 7 moves a selected vertex's
// matching partner too), in the order-free reading: every edge cut by the
// 2-means labels selects its end with the smaller (s, id); the selected
// vertices and their partners form V3.  Partners always share a node.
__global__ void k_pick(const int32_t* __restrict__ ord, const int32_t* __restrict__ seg, int64_t n,
                       const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                       const uint64_t* __restrict__ vrec, uint8_t* __restrict__ vpick) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int s = seg[i];
  if (s < 0) return;
  const int32_t v = ord[i];
  const uint64_t rv = vrec[v];
  const uint32_t l = vrec_label(rv);
  uint8_t pick = 0;
  if (l != 0) {
    const float sv = vrec_s(rv);
    const uint32_t other = vrec_other(s, l);
    for (int32_t t = adj_ptr[v]; t < adj_ptr[v + 1]; ++t) {
      const int32_t w = adj[t];
      const uint64_t rw = vrec[w];
      if ((uint32_t)(rw >> 32) != other) continue;
      const float sw = vrec_s(rw);
      if (sv < sw || (sv == sw && v < w)) { pick = 1; break; }
    }
  }
  vpick[v] = pick;
}

__global__ void k_separator_mu(const int32_t* __restrict__ ord, const int32_t* __restrict__ seg, int64_t n,
                               const int32_t* __restrict__ mu, const uint64_t* __restrict__ vrec,
                               const uint8_t* __restrict__ vpick, NodeDev* __restrict__ nodes,
                               uint8_t* __restrict__ labf, unsigned long long* __restrict__ pk) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int s = i < n ? seg[i] : -1;
  uint8_t l = 0;
  if (s >= 0) {
    int32_t v = ord[i];
    l = (uint8_t)vrec_label(vrec[v]);
    if (l != 0 && (vpick[v] | vpick[mu[v]])) l = 3;
    labf[i] = l;
  }
  if (i < n) pk[i] = part_count(l);
  count_labels(s, l, nodes);
}

// ----- Algorithm 7's loop with a strengthened diagonal, in canonical order -----
// The loop visits the edges cut by the 2-means labels in ascending key (s(c),
// c, w), c the end with the smaller (s, id) (the one the loop moves), and an
// edge still cut when reached moves c and mu(c) into V3.  A vertex u is moved
// only by an edge whose moved end is u or mu(u), so the pair class
// P = {u, mu(u)} is moved by at most one edge: the first edge of its candidate
// list M(P) (edges moving a member of P, in key order) whose other end's class
// is not moved before it.  T(P) = key of that edge (infinite if none).  Every
// class walks its list in rounds: its current candidate e = (c, w) is skipped
// when class(w) moved before e, taken when class(w) is known to move after e
// (it is exhausted, took a later edge, or its current candidate is already
// later than e: candidates only advance), else it waits.  The class with the
// globally smallest current candidate always decides, so every round makes
// progress, and the fixed point is the sequential loop's result.
//
// State of a class (one int32 word at its representative min(u, mu(u))):
// (candidate index << 2) | flag, flag 0 undecided, 1 moved, 2 never moved.
// Words only move forward (index up, flag 0 -> 1 or 2), so a stale read gives
// a lower bound on the class's move key and every decision taken from it holds.
constexpr int kMuUndecided = 0, kMuMoved = 1, kMuNever = 2;

__device__ __forceinline__ bool mu_cut_neighbour(int32_t v, float sv, int32_t w, int s, uint32_t l,
                                                 const uint64_t* __restrict__ vrec) {
  const uint64_t rw = vrec[w];
  if ((uint32_t)(rw >> 32) != vrec_other(s, l)) return false;
  const float sw = vrec_s(rw);
  return sv < sw || (sv == sw && v < w);  // v is the end the loop moves
}

// Candidate edges moved through each vertex (edges whose moved end it is).
__global__ void k_mu_count(const int32_t* __restrict__ ord, const int32_t* __restrict__ seg, int64_t n,
                           const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                           const uint64_t* __restrict__ vrec, int32_t* __restrict__ mcnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = seg[i];
  const int32_t v = ord[i];
  int32_t c = 0;
  const uint64_t rv = s >= 0 ? vrec[v] : 0ull;
  const uint32_t l = vrec_label(rv);
  if (l != 0)
    for (int32_t t = adj_ptr[v]; t < adj_ptr[v + 1]; ++t) c += mu_cut_neighbour(v, vrec_s(rv), adj[t], s, l, vrec);
  mcnt[v] = c;
}

__device__ __forceinline__ bool mu_first(int32_t a, int32_t b, const uint64_t* __restrict__ vrec) {
  const float sa = vrec_s(vrec[a]), sb = vrec_s(vrec[b]);
  return sa < sb || (sa == sb && a < b);
}

// Length of every class's candidate list, at its representative.
__global__ void k_mu_total(const int32_t* __restrict__ ord, const int32_t* __restrict__ seg, int64_t n,
                           const int32_t* __restrict__ mu, const int32_t* __restrict__ mcnt,
                           int32_t* __restrict__ mtot) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t v = ord[i];
  const int32_t u = mu[v];
  mtot[v] = (seg[i] >= 0 && v <= u) ? mcnt[v] + (u != v ? mcnt[u] : 0) : 0;
}

// Candidate lists: the edges moving the member with the smaller (s, id)
// first, each member's edges by ascending other end (adjacency order).
__global__ void k_mu_fill(const int32_t* __restrict__ ord, const int32_t* __restrict__ seg, int64_t n,
                          const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                          const uint64_t* __restrict__ vrec, const int32_t* __restrict__ mu,
                          const int32_t* __restrict__ mcnt, const int32_t* __restrict__ mbeg,
                          int32_t* __restrict__ cand_c, int32_t* __restrict__ cand_w, int32_t* __restrict__ mstate) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = seg[i];
  if (s < 0) return;
  const int32_t v = ord[i];
  const int32_t u = mu[v];
  const int32_t rep = v < u ? v : u;
  if (v == rep) {
    const int32_t tot = mcnt[v] + (u != v ? mcnt[u] : 0);
    mstate[rep] = tot > 0 ? kMuUndecided : kMuNever;
  }
  const uint64_t rv = vrec[v];
  const uint32_t l = vrec_label(rv);
  if (l == 0 || mcnt[v] == 0) return;
  const bool first = u == v || mu_first(v, u, vrec);
  int32_t o = mbeg[rep] + (first ? 0 : mcnt[u]);
  for (int32_t t = adj_ptr[v]; t < adj_ptr[v + 1]; ++t) {
    const int32_t w = adj[t];
    if (!mu_cut_neighbour(v, vrec_s(rv), w, s, l, vrec)) continue;
    cand_c[o] = v;
    cand_w[o] = w;
    ++o;
  }
}

// (s, id) key of a candidate's moved end, as one ordered 64-bit number (s >= 0).
__device__ __forceinline__ uint64_t mu_key(int32_t c, const uint64_t* __restrict__ vrec) {
  return ((uint64_t)(uint32_t)vrec[c] << 32) | (uint32_t)c;
}

// One round over every undecided class; *busy counts classes still undecided.
__global__ void k_mu_round(const int32_t* __restrict__ ord, const int32_t* __restrict__ seg, int64_t n,
                           const int32_t* __restrict__ mu, const int32_t* __restrict__ mbeg,
                           const int32_t* __restrict__ mtot, const int32_t* __restrict__ cand_c,
                           const int32_t* __restrict__ cand_w, const uint64_t* __restrict__ vrec,
                           int32_t* __restrict__ mstate, int* __restrict__ busy) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || seg[i] < 0) return;
  const int32_t p = ord[i];
  if (mu[p] < p) return;  // not the representative
  volatile int32_t* vst = mstate;
  int32_t w0 = vst[p];
  if ((w0 & 3) != kMuUndecided) return;
  int32_t ptr = w0 >> 2;
  const int32_t tot = mtot[p], base = mbeg[p];
  int32_t out = -1;
  while (out < 0) {
    if (ptr >= tot) { out = (ptr << 2) | kMuNever; break; }
    const int32_t c = cand_c[base + ptr], w = cand_w[base + ptr];
    const int32_t q = min(w, mu[w]);
    if (q == p) { out = (ptr << 2) | kMuMoved; break; }  // edge between the partners
    const uint64_t ke = mu_key(c, vrec);
    const int32_t sq = vst[q];
    const int fq = sq & 3;
    if (fq == kMuNever) { out = (ptr << 2) | kMuMoved; break; }
    const uint64_t kq = mu_key(cand_c[mbeg[q] + (sq >> 2)], vrec);
    if (fq == kMuMoved) {
      if (kq < ke) { ++ptr; continue; }  // class(w) moved first: the edge is no longer cut
      out = (ptr << 2) | kMuMoved;
      break;
    }
    if (kq > ke) { out = (ptr << 2) | kMuMoved; break; }  // class(w) cannot move before this edge
    break;  // wait for class(w)
  }
  if (out >= 0) {
    vst[p] = out;
  } else {
    if (ptr != (w0 >> 2)) vst[p] = ptr << 2;
    if (busy) atomicAdd(busy, 1);
  }
}

// Final labels: both members of a moved class are in V3.
__global__ void k_separator_mu_loop(const int32_t* __restrict__ ord, const int32_t* __restrict__ seg, int64_t n,
                                    const int32_t* __restrict__ mu, const uint64_t* __restrict__ vrec,
                                    const int32_t* __restrict__ mstate, NodeDev* __restrict__ nodes,
                                    uint8_t* __restrict__ labf, unsigned long long* __restrict__ pk) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int s = i < n ? seg[i] : -1;
  uint8_t l = 0;
  if (s >= 0) {
    int32_t v = ord[i];
    l = (uint8_t)vrec_label(vrec[v]);
    if (l != 0 && (mstate[min(v, mu[v])] & 3) == kMuMoved) l = 3;
    labf[i] = l;
  }
  if (i < n) pk[i] = part_count(l);
  count_labels(s, l, nodes);
}

// Stable partition of every split node into [V1, V2, V3] (BBD) or
// [V1, V3, V2] (SBD); other positions are copied.  Every position also gets
// its node of the next level (seg2): the child of its node that holds its part
// (k_children has numbered them), or -1 when its vertex is placed now (a
// leaf, or a separator that is not recursed into); such a vertex's separator
// record is cleared, so that no later level takes it for a neighbour in one
// of its nodes (the records of the others are rewritten by the next level's
// k_vertex_state).
__global__ void k_scatter(const int32_t* __restrict__ ord, const float4* __restrict__ xo,
                          const int32_t* __restrict__ seg, const uint8_t* __restrict__ labf, int64_t n,
                          const NodeDev* __restrict__ nodes, const unsigned long long* __restrict__ pre, int sbd,
                          int32_t* __restrict__ ord2, float4* __restrict__ xo2, int32_t* __restrict__ seg2,
                          uint64_t* __restrict__ vrec) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = seg[i];
  const int32_t v = ord[i];   // loads in flight together
  const float4 xi = xo[i];
  const uint8_t li = labf[i];
  int64_t dst = i;
  int32_t next = -1;
  if (s >= 0) {
    const NodeDev& nd = nodes[s];
    int c1 = nd.c1, c2 = nd.c2, c3 = nd.c3;
    if (c1 + c2 + c3 > 0) {
      const uint8_t l = li;
      unsigned long long base = nd.off > 0 ? pre[nd.off - 1] : 0ull;
      unsigned long long own = (l == 1) ? 1ull : (l == 2 ? (1ull << 32) : 0ull);
      unsigned long long ex = pre[i] - base - own;
      int64_t r1 = (int64_t)(ex & 0xffffffffull), r2 = (int64_t)(ex >> 32);
      int64_t r3 = (i - nd.off) - r1 - r2;
      int64_t o;
      if (l == 1) o = r1;
      else if (l == 2) o = sbd ? (int64_t)c1 + c3 + r2 : (int64_t)c1 + r2;
      else o = sbd ? (int64_t)c1 + r3 : (int64_t)c1 + c2 + r3;
      dst = nd.off + o;
      next = l == 1 ? nd.child1 : (l == 2 ? nd.child2 : nd.child3);
    }
  }
  ord2[dst] = v;
  xo2[dst] = xi;
  seg2[dst] = next;
  if (s >= 0 && next < 0) vrec[v] = 0ull;
}

// Tree records and the next level's node table.  Children: V1 and V2, and
// with separator recursion V3 too (keys 2h + side, or 3h - 1 + side).
__global__ void k_children(NodeDev* __restrict__ nodes, int N, const int64_t* __restrict__ pbase, int min_part,
                           int max_depth, int sbd, int sep_rec, NodeDev* __restrict__ next,
                           int* __restrict__ next_count, int next_cap, TreeDev tree, int* __restrict__ err) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  NodeDev& nd = nodes[s];
  bool split = nd.c1 + nd.c2 + nd.c3 > 0;
  int slot = atomicAdd(tree.count, 1);
  if (slot >= tree.cap) { atomicOr(err, 1); return; }
  tree.heap[slot] = nd.heap;
  tree.prob[slot] = nd.prob;
  tree.offset[slot] = (int32_t)nd.off;
  tree.depth[slot] = nd.depth;
  if (!split) {
    tree.n1[slot] = nd.size; tree.n2[slot] = 0; tree.nsep[slot] = 0;
    return;
  }
  tree.n1[slot] = nd.c1; tree.n2[slot] = nd.c2; tree.nsep[slot] = nd.c3;
  for (int side = 0; side < (sep_rec ? 3 : 2); ++side) {
    int size = side == 0 ? nd.c1 : (side == 1 ? nd.c2 : nd.c3);
    if (size == 0) continue;
    int64_t off = nd.off + (side == 0 ? 0 : side == 1 ? (sbd ? nd.c1 + nd.c3 : nd.c1) : (sbd ? nd.c1 : nd.c1 + nd.c2));
    uint64_t heap = sep_rec ? 3 * nd.heap - 1 + side : 2 * nd.heap + side;
    int depth = nd.depth + 1;
    if (size > min_part && depth < max_depth) {
      int c = atomicAdd(next_count, 1);
      if (c >= next_cap) { atomicOr(err, 2); continue; }
      NodeDev& ch = next[c];
      ch.heap = heap; ch.off = off; ch.size = size; ch.depth = depth; ch.prob = nd.prob;
      if (side == 0) nd.child1 = c; else if (side == 1) nd.child2 = c; else nd.child3 = c;
    } else {
      int t = atomicAdd(tree.count, 1);
      if (t >= tree.cap) { atomicOr(err, 1); continue; }
      tree.heap[t] = heap; tree.prob[t] = nd.prob; tree.offset[t] = (int32_t)off;
      tree.depth[t] = depth; tree.n1[t] = size; tree.n2[t] = 0; tree.nsep[t] = 0;
    }
  }
}

__global__ void k_root_nodes(NodeDev* __restrict__ nodes, const int64_t* __restrict__ pbase, const int32_t* __restrict__ ids,
                             int N, const uint64_t* __restrict__ heaps) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  int p = ids[s];
  NodeDev& nd = nodes[s];
  nd.heap = heaps ? heaps[s] : 1ull;
  nd.off = pbase[p];
  nd.size = (int32_t)(pbase[p + 1] - pbase[p]);
  nd.depth = 0;
  nd.prob = p;
}

__global__ void k_seg_init(int32_t* __restrict__ seg, const int32_t* __restrict__ ord,
                           int64_t n, const int64_t* __restrict__ pbase, int P, const int32_t* __restrict__ node_of_prob) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pbase[mid] <= i) lo = mid; else hi = mid;
  }
  seg[i] = node_of_prob[lo];
}

__global__ void k_gather_coords(const float4* __restrict__ x, const int32_t* __restrict__ ord, int64_t n,
                                float4* __restrict__ xo) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) xo[i] = x[ord[i]];
}

__global__ void k_iota(int32_t* a, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (int32_t)i;
}

__global__ void k_tree_keys(const TreeDev tree, int n, int by_prob, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  keys[t] = by_prob ? (uint64_t)tree.prob[t] : tree.heap[t];
  vals[t] = (uint32_t)t;
}

__global__ void k_tree_regather(const uint32_t* __restrict__ idx, int n, int by_prob, const TreeDev tree,
                                uint64_t* __restrict__ keys) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  keys[t] = by_prob ? (uint64_t)tree.prob[idx[t]] : tree.heap[idx[t]];
}

__global__ void k_tree_out(const uint32_t* __restrict__ idx, int n, const TreeDev tree, uint64_t* heap,
                           int32_t* offset, int32_t* n1, int32_t* n2, int32_t* nsep, int32_t* depth, int32_t* prob) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  uint32_t j = idx[t];
  if (heap) heap[t] = tree.heap[j];
  if (offset) offset[t] = tree.offset[j];
  if (n1) n1[t] = tree.n1[j];
  if (n2) n2[t] = tree.n2[j];
  if (nsep) nsep[t] = tree.nsep[j];
  if (depth) depth[t] = tree.depth[j];
  if (prob) prob[t] = tree.prob[j];
}

template <class F>
void dispatch_d(int d, F&& f) {
  if (d == 2) f(std::integral_constant<int, 2>());
  else if (d == 3) f(std::integral_constant<int, 3>());
  else f(std::integral_constant<int, 4>());
}

// ---- cut-row/column ordering of the separators (Sec. 4.2) ----------------
// Every position belongs to one tree record: a leaf's vertices or a split
// node's separator.  Records are indexed in (problem, heap) order.
struct CutRec {
  uint64_t heap;
  int32_t depth;
  int32_t a;   // separator start (split nodes)
  int32_t ns;  // separator size (0 for leaves)
};

// One warp per record: lane 0 fills the record, the warp marks its positions.
__global__ void k_cut_recs(const TreeDev tree, const uint32_t* __restrict__ idx, int n, int sbd,
                           CutRec* __restrict__ cr, int32_t* __restrict__ own, int64_t* __restrict__ sz) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = lane_id();
  if (w >= n) return;
  const int i = (int)w;
  const uint32_t r = idx[i];
  const int32_t o = tree.offset[r], n1 = tree.n1[r], n2 = tree.n2[r], ns = tree.nsep[r];
  const bool leaf = n2 == 0 && ns == 0;
  const int32_t a = leaf ? o : (sbd ? o + n1 : o + n1 + n2);
  if (lane == 0) {
    CutRec c;
    c.heap = tree.heap[r];
    c.depth = tree.depth[r];
    c.a = a;
    c.ns = leaf ? 0 : ns;
    cr[i] = c;
    sz[i] = c.ns;
  }
  const int32_t len = leaf ? n1 : ns;
  for (int32_t p = lane; p < len; p += 32) own[a + p] = i;
}

__global__ void k_inverse_perm(const int32_t* __restrict__ ord, int64_t n, int32_t* __restrict__ pos) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) pos[ord[p]] = (int32_t)p;
}

// Pairs 1..b of the vertex at every separator position (pair l in bits
// 2(b - l), 2(b - l) + 1).  A neighbour owned by a record D levels deep below
// the separator's node (depth d, heap h) lies in the first (second) part of
// the split of its ancestor at depth d + l when D >= d + l + 1 and its heap
// number takes the branch 2h' (2h' + 1) at depth d + l + 1.  Owners outside
// the node's subtree (ancestors, the node itself) add nothing.
__global__ void k_cut_codes(const int32_t* __restrict__ ord, const int32_t* __restrict__ pos,
                            const int32_t* __restrict__ own, int64_t n, const CutRec* __restrict__ cr,
                            const int32_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj, int b,
                            uint32_t* __restrict__ vcode) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || own[p] < 0) return;
  const CutRec c = cr[own[p]];
  if (c.ns == 0) return;
  const int32_t w = ord[p];
  uint32_t code = 0;
  for (int32_t t = adj_ptr[w]; t < adj_ptr[w + 1]; ++t) {
    const int32_t ou = own[pos[adj[t]]];
    if (ou < 0) continue;
    const CutRec u = cr[ou];
    if (u.depth <= c.depth || (u.heap >> (u.depth - c.depth)) != c.heap) continue;
    for (int l = 1; l <= b && u.depth >= c.depth + l + 1; ++l) {
      const uint32_t second = (uint32_t)(u.heap >> (u.depth - c.depth - l - 1)) & 1u;
      code |= (second ? 2u : 1u) << (2 * (b - l));
    }
  }
  vcode[w] = code;
}

// Sort key (record, ranks of pairs 1..b) of every separator position; other
// positions sort last.  With a matching a vertex is ranked by its pair's
// number (its own bits or its partner's): row and matched column share one
// position.
__global__ void k_cut_keys(const int32_t* __restrict__ ord, const int32_t* __restrict__ own, int64_t n,
                           const CutRec* __restrict__ cr, const uint32_t* __restrict__ vcode,
                           const int32_t* __restrict__ mu, int sbd, int b, uint64_t sentinel,
                           uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int i = own[p];
  uint64_t key = sentinel;
  if (i >= 0 && cr[i].ns > 0) {
    const int32_t w = ord[p];
    const uint32_t code = vcode[w] | (mu ? vcode[mu[w]] : 0u);
    uint64_t rk = 0;
    for (int l = 1; l <= b; ++l) {
      const uint32_t f = (code >> (2 * (b - l))) & 3u;
      const uint32_t r = sbd ? (f ^ 1u) : f;  // SBD: 01, 00, 11, 10
      rk = 4 * rk + r;
    }
    key = ((uint64_t)i << (2 * b)) | rk;
  }
  keys[p] = key;
  vals[p] = (uint32_t)p;
}

// Separator positions in (record, ranks, position) order back into their
// record's separator range.
__global__ void k_cut_scatter(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t m,
                              int b, const CutRec* __restrict__ cr, const int64_t* __restrict__ gstart,
                              const int32_t* __restrict__ ord, int32_t* __restrict__ ord2) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int i = (int)(keys[j] >> (2 * b));
  ord2[cr[i].a + (j - gstart[i])] = ord[vals[j]];
}

}  // namespace

// 2-means of every node of the table (Algorithm 5), leaving the final labels
// in lab (position order) and the node fields z1, z2, n1, n2, state.  The
// working arrays come from the caller: dval, dpre (n values), cnt (one int),
// partial (scan_partials_needed(n) values) and, optionally, rep (per-node
// replicas of the Lloyd sums, N * kRepR * 10 values, zeroed).
static vmo_status two_means_body(OrderState& st, int N, int d, int km_iters, unsigned long long* dval,
                                 unsigned long long* dpre, int* cnt, uint64_t* partial, unsigned long long* rep,
                                 cudaStream_t s) {
  const int64_t n = st.n;
  vmo_status stt = VMO_OK;
  dispatch_d(d, [&](auto DC) {
    constexpr int D = decltype(DC)::value;
    launch(k_node_reset, grid_for(N, kBlock), kBlock, 0, s, st.nodes, N);
    const bool wide = n >= kPosItemsMin;  // kPosItems positions per thread
    if (wide)
      launch(k_maxabs<D, kPosItems>, grid_for((n + kPosItems - 1) / kPosItems, kBlock), kBlock, 0, s, st.xo, st.seg,
             n, st.nodes);
    else
      launch(k_maxabs<D, 1>, grid_for(n, kBlock), kBlock, 0, s, st.xo, st.seg, n, st.nodes);
    launch(k_seed1, grid_for(N, kBlock), kBlock, 0, s, st.nodes, N, st.xo, st.seeds);
    if (wide)
      launch(k_dsq<D, kPosItems>, grid_for((n + kPosItems - 1) / kPosItems, kBlock), kBlock, 0, s, st.xo, st.seg, n,
             st.nodes, dval);
    else
      launch(k_dsq<D, 1>, grid_for(n, kBlock), kBlock, 0, s, st.xo, st.seg, n, st.nodes, dval);
    stt = scan_inclusive_u64_into((const uint64_t*)dval, (uint64_t*)dpre, n, partial, s);
    if (stt != VMO_OK) return;
    if (wide)
      launch(k_seed2<D, kPosItems>, grid_for((n + kPosItems - 1) / kPosItems, kBlock), kBlock, 0, s, st.xo, st.seg,
             n, dval, dpre, st.nodes, st.seeds);
    else
      launch(k_seed2<D, 1>, grid_for(n, kBlock), kBlock, 0, s, st.xo, st.seg, n, dval, dpre, st.nodes, st.seeds);
    for (int it = 0; it < km_iters; ++it) {
      launch_assign<D>(n, s, st.xo, st.seg, it, st.nodes, st.lab, 0, rep);
      if (rep) launch(k_fold_reps, grid_for(N * 10, kBlock), kBlock, 0, s, st.nodes, N, rep);
      launch(k_update<D>, grid_for(N, kBlock), kBlock, 0, s, st.nodes, N, it);
      if (it % 4 == 3 && it + 1 < km_iters) {  // stop early once every node has converged
        int h = 0;
        cudaError_t e = cudaMemsetAsync(cnt, 0, 4, s);
        if (e != cudaSuccess) { stt = cuda_fail(e, "two_means: clear counter", __FILE__, __LINE__); return; }
        launch(k_count_active, grid_for(N, kBlock), kBlock, 0, s, st.nodes, N, cnt);
        e = cudaMemcpyAsync(&h, cnt, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { stt = cuda_fail(e, "two_means: convergence check", __FILE__, __LINE__); return; }
        if (h == 0) break;
      }
    }
    launch(k_clear_counts, grid_for(N, kBlock), kBlock, 0, s, st.nodes, N);
    launch_assign<D>(n, s, st.xo, st.seg, 0, st.nodes, st.lab, 1, rep);
    if (rep) launch(k_fold_reps, grid_for(N * 10, kBlock), kBlock, 0, s, st.nodes, N, rep);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) stt = cuda_fail(e, "two_means", __FILE__, __LINE__);
  });
  return stt;
}

vmo_status two_means(OrderState& st, int N, int d, int km_iters, cudaStream_t s, Scratch& sc) {
  const int64_t n = st.n;
  ScratchFrame frame(sc);
  unsigned long long *dval, *dpre, *rep = nullptr;
  uint64_t* partial;
  int* cnt;
  VMO_TRY(sc.alloc(&dval, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&dpre, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&partial, std::max<int64_t>(scan_partials_needed(n), 1)));
  VMO_TRY(sc.alloc(&cnt, 1));
  if (N <= kRepNodes && n >= kRepMinPositions) {
    VMO_TRY(sc.alloc(&rep, (size_t)N * kRepR * 10));
    VMO_CUDA(cudaMemsetAsync(rep, 0, (size_t)N * kRepR * 10 * sizeof(unsigned long long), s));
  }
  return two_means_body(st, N, d, km_iters, dval, dpre, cnt, partial, rep, s);
}

vmo_status two_means_into(OrderState& st, int N, int d, int km_iters, unsigned long long* dval,
                          unsigned long long* dpre, int* cnt, uint64_t* partial, cudaStream_t s) {
  return two_means_body(st, N, d, km_iters, dval, dpre, cnt, partial, nullptr, s);
}

// Separator of every split node of the level by Algorithm 7's loop with the
// strengthened diagonal, in canonical edge order (the class rounds above).
static vmo_status mu_loop_separator(OrderState& st, int64_t n, uint8_t* labf, unsigned long long* pk, cudaStream_t s,
                                    Scratch& sc) {
  if (n == 0) return VMO_OK;
  ScratchFrame frame(sc);
  int32_t *mcnt, *mtot, *mbeg, *mstate, *total;
  int* busy;
  VMO_TRY(sc.alloc(&mcnt, n));
  VMO_TRY(sc.alloc(&mtot, n));
  VMO_TRY(sc.alloc(&mbeg, n));
  VMO_TRY(sc.alloc(&mstate, n));
  VMO_TRY(sc.alloc(&total, 1));
  VMO_TRY(sc.alloc(&busy, 1));
  launch(k_mu_count, grid_for(n, kBlock), kBlock, 0, s, st.ord, st.seg, n, st.adj_ptr, st.adj, st.vrec, mcnt);
  launch(k_mu_total, grid_for(n, kBlock), kBlock, 0, s, st.ord, st.seg, n, st.mu, mcnt, mtot);
  VMO_TRY(scan_exclusive<int32_t>(mtot, mbeg, n, total, s, sc));
  int32_t ncand = 0;
  VMO_CUDA(cudaMemcpyAsync(&ncand, total, 4, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  int32_t *cand_c, *cand_w;
  VMO_TRY(sc.alloc(&cand_c, std::max<int32_t>(ncand, 1)));
  VMO_TRY(sc.alloc(&cand_w, std::max<int32_t>(ncand, 1)));
  launch(k_mu_fill, grid_for(n, kBlock), kBlock, 0, s, st.ord, st.seg, n, st.adj_ptr, st.adj, st.vrec, st.mu, mcnt,
         mbeg, cand_c, cand_w, mstate);
  // every round decides at least one class (the one with the smallest
  // current candidate), so ncand + 1 rounds always suffice
  constexpr int kRoundsPerCheck = 4;
  int64_t rounds = 0;
  for (;;) {
    for (int r = 0; r < kRoundsPerCheck; ++r) {
      if (r == kRoundsPerCheck - 1) VMO_CUDA(cudaMemsetAsync(busy, 0, sizeof(int), s));
      launch(k_mu_round, grid_for(n, kBlock), kBlock, 0, s, st.ord, st.seg, n, st.mu, mbeg, mtot, cand_c, cand_w,
             st.vrec, mstate, r == kRoundsPerCheck - 1 ? busy : (int*)nullptr);
    }
    rounds += kRoundsPerCheck;
    int h = 0;
    VMO_CUDA(cudaMemcpyAsync(&h, busy, sizeof(int), cudaMemcpyDeviceToHost, s));
    VMO_CUDA(cudaStreamSynchronize(s));
    if (h == 0) break;
    if (rounds > (int64_t)ncand + 2 * kRoundsPerCheck)
      return cuda_fail(cudaErrorUnknown, "separator: the matched-pair rounds did not settle", __FILE__, __LINE__);
  }
  launch(k_separator_mu_loop, grid_for(n, kBlock), kBlock, 0, s, st.ord, st.seg, n, st.mu, st.vrec, mstate, st.nodes,
         labf, pk);
  VMO_LAUNCHED("separator_mu_loop");
  return VMO_OK;
}

vmo_status order_levels(OrderState& st, const OrderParams& op, cudaStream_t s, Scratch& sc) {
  const int64_t n = st.n;
  int N = st.nroots;
  int32_t *ord2, *seg2, *next_count, *err;
  float4* xo2;
  uint8_t* labf;
  unsigned long long *pk, *pre;
  NodeDev* next;
  VMO_TRY(sc.alloc(&ord2, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&seg2, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&xo2, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&labf, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&pk, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&pre, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&next, st.node_cap));
  VMO_TRY(sc.alloc(&next_count, 1));
  VMO_TRY(sc.alloc(&err, 1));
  VMO_CUDA(cudaMemsetAsync(err, 0, 4, s));
  while (N > 0) {
    VMO_TRY(two_means(st, N, op.d, op.km_iters, s, sc));
    dispatch_d(op.d, [&](auto DC) {
      constexpr int D = decltype(DC)::value;
      launch(k_vertex_state<D>, grid_for(n, kBlock), kBlock, 0, s, st.xo, st.ord, st.seg, n, st.nodes, st.lab,
                                                               st.vrec);
    });
    if (st.mu && op.mu_order_free) {
      launch(k_pick, grid_for(n, kBlock), kBlock, 0, s, st.ord, st.seg, n, st.adj_ptr, st.adj, st.vrec, st.vpick);
      launch(k_separator_mu, grid_for(n, kBlock), kBlock, 0, s, st.ord, st.seg, n, st.mu, st.vrec, st.vpick, st.nodes,
             labf, pk);
    } else if (st.mu) {
      VMO_TRY(mu_loop_separator(st, n, labf, pk, s, sc));
    } else {
      launch(k_separator, grid_for(n, kBlock), kBlock, 0, s, st.ord, st.seg, n, st.adj_ptr, st.adj, st.vrec, st.nodes,
             labf, pk);
    }
    VMO_LAUNCHED("separator");
    VMO_TRY(scan_inclusive<uint64_t>((const uint64_t*)pk, (uint64_t*)pre, n, s, sc));
    // children first (they number the next level's nodes), then the scatter
    // writes every position's next node
    VMO_CUDA(cudaMemsetAsync(next_count, 0, 4, s));
    const int max_depth = op.sep_rec ? std::min(op.max_depth, kSepRecMaxDepth) : op.max_depth;
    launch(k_children, grid_for(N, kBlock), kBlock, 0, s, st.nodes, N, st.pbase, op.min_part, max_depth, op.sbd,
           op.sep_rec, next, next_count, st.node_cap, st.tree, err);
    launch(k_scatter, grid_for(n, kBlock), kBlock, 0, s, st.ord, st.xo, st.seg, labf, n, st.nodes, pre, op.sbd, ord2, xo2,
                                                     seg2, st.vrec);
    VMO_LAUNCHED("partition");
    // the scattered arrays become the current ones
    std::swap(st.ord, ord2);
    std::swap(st.xo, xo2);
    std::swap(st.seg, seg2);
    int hN = 0, herr = 0;
    VMO_CUDA(cudaMemcpyAsync(&hN, next_count, 4, cudaMemcpyDeviceToHost, s));
    VMO_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
    VMO_CUDA(cudaStreamSynchronize(s));
    if (herr) return cuda_fail(cudaErrorUnknown, "ordering: node table or tree capacity exceeded", __FILE__, __LINE__);
    std::swap(st.nodes, next);
    N = hN;
  }
  return VMO_OK;
}

vmo_status order_setup(OrderState& st, const float4* x, const std::vector<int64_t>& pbase_host,
                       const std::vector<uint64_t>& seeds, const OrderParams& op, const uint32_t* init_ord,
                       cudaStream_t s, Scratch& sc) {
  const int64_t n = pbase_host.back();
  const int P = (int)pbase_host.size() - 1;
  if (n >= (int64_t(1) << 30) - 64) return invalid("ordering: more than 2^30 - 64 vertices");
  st.n = n;
  VMO_TRY(sc.alloc(&st.ord, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&st.xo, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&st.seg, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&st.lab, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&st.vrec, std::max<int64_t>(n, 1)));
  VMO_CUDA(cudaMemsetAsync(st.vrec, 0, std::max<int64_t>(n, 1) * sizeof(uint64_t), s));  // no vertex in a split node
  if (st.mu) VMO_TRY(sc.alloc(&st.vpick, std::max<int64_t>(n, 1)));
  VMO_TRY(sc.alloc(&st.pbase, P + 1));
  VMO_TRY(sc.alloc(&st.seeds, std::max(P, 1)));
  // node table capacity: active nodes of one level have > min_part vertices each
  st.node_cap = (int)std::min<int64_t>(n / (std::max(op.min_part, 1) + 1) + P + 16, n + 16);
  VMO_TRY(sc.alloc(&st.nodes, st.node_cap));
  // tree capacity: at most 2 records per vertex
  st.tree.cap = (int)std::min<int64_t>(2 * n + 16, INT32_MAX);
  VMO_TRY(sc.alloc(&st.tree.heap, st.tree.cap));
  VMO_TRY(sc.alloc(&st.tree.prob, st.tree.cap));
  VMO_TRY(sc.alloc(&st.tree.offset, st.tree.cap));
  VMO_TRY(sc.alloc(&st.tree.n1, st.tree.cap));
  VMO_TRY(sc.alloc(&st.tree.n2, st.tree.cap));
  VMO_TRY(sc.alloc(&st.tree.nsep, st.tree.cap));
  VMO_TRY(sc.alloc(&st.tree.depth, st.tree.cap));
  VMO_TRY(sc.alloc(&st.tree.count, 1));
  VMO_CUDA(cudaMemsetAsync(st.tree.count, 0, 4, s));
  VMO_CUDA(cudaMemcpyAsync(st.pbase, pbase_host.data(), (P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(st.seeds, seeds.data(), P * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  if (n > 0) {
    if (init_ord)
      VMO_CUDA(cudaMemcpyAsync(st.ord, init_ord, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    else
      launch(k_iota, grid_for(n, kBlock), kBlock, 0, s, st.ord, n);
    launch(k_gather_coords, grid_for(n, kBlock), kBlock, 0, s, x, st.ord, n, st.xo);
    VMO_LAUNCHED("order_setup");
  }
  // roots: problems with more than min_part vertices and max_depth > 0 are
  // active; the others are leaves at once
  std::vector<int32_t> ids, node_of_prob(P, -1);
  for (int p = 0; p < P; ++p) {
    int64_t k = pbase_host[p + 1] - pbase_host[p];
    if (k > op.min_part && op.max_depth > 0) {
      node_of_prob[p] = (int32_t)ids.size();
      ids.push_back(p);
    }
  }
  st.nroots = (int)ids.size();
  std::vector<int32_t> leaf_probs;
  for (int p = 0; p < P; ++p)
    if (node_of_prob[p] < 0 && pbase_host[p + 1] > pbase_host[p]) leaf_probs.push_back(p);
  int32_t *d_ids, *d_nop;
  VMO_TRY(sc.alloc(&d_ids, std::max<size_t>(ids.size(), 1)));
  VMO_TRY(sc.alloc(&d_nop, std::max(P, 1)));
  if (!ids.empty())
    VMO_CUDA(cudaMemcpyAsync(d_ids, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaMemcpyAsync(d_nop, node_of_prob.data(), P * 4, cudaMemcpyHostToDevice, s));
  if (st.nroots > 0) {
    launch(k_root_nodes, grid_for(st.nroots, kBlock), kBlock, 0, s, st.nodes, st.pbase, d_ids, st.nroots, nullptr);
    VMO_LAUNCHED("roots");
  }
  if (n > 0) {
    launch(k_seg_init, grid_for(n, kBlock), kBlock, 0, s, st.seg, st.ord, n, st.pbase, P, d_nop);
    VMO_LAUNCHED("seg_init");
  }
  // leaf roots become tree records directly
  if (!leaf_probs.empty()) {
    std::vector<int32_t> hc(1);
    int nl = (int)leaf_probs.size();
    std::vector<uint64_t> h(nl, 1ull);
    std::vector<int32_t> zero(nl, 0), sz(nl), offs(nl);
    for (int i = 0; i < nl; ++i) {
      sz[i] = (int32_t)(pbase_host[leaf_probs[i] + 1] - pbase_host[leaf_probs[i]]);
      offs[i] = (int32_t)pbase_host[leaf_probs[i]];
    }
    VMO_CUDA(cudaMemcpyAsync(st.tree.heap, h.data(), nl * 8, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaMemcpyAsync(st.tree.prob, leaf_probs.data(), nl * 4, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaMemcpyAsync(st.tree.offset, offs.data(), nl * 4, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaMemcpyAsync(st.tree.n1, sz.data(), nl * 4, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaMemcpyAsync(st.tree.n2, zero.data(), nl * 4, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaMemcpyAsync(st.tree.nsep, zero.data(), nl * 4, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaMemcpyAsync(st.tree.depth, zero.data(), nl * 4, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaMemcpyAsync(st.tree.count, &nl, 4, cudaMemcpyHostToDevice, s));
    VMO_CUDA(cudaStreamSynchronize(s));
  }
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status tree_sorted(OrderState& st, bool by_prob, int32_t* count_out, uint32_t** idx_out, cudaStream_t s,
                       Scratch& sc) {
  int n = 0;
  VMO_CUDA(cudaMemcpyAsync(&n, st.tree.count, 4, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  *count_out = n;
  uint64_t *k1, *k2;
  uint32_t *v1, *v2;
  VMO_TRY(sc.alloc(&k1, std::max(n, 1)));
  VMO_TRY(sc.alloc(&k2, std::max(n, 1)));
  VMO_TRY(sc.alloc(&v1, std::max(n, 1)));
  VMO_TRY(sc.alloc(&v2, std::max(n, 1)));
  if (n == 0) { *idx_out = v2; return VMO_OK; }
  launch(k_tree_keys, grid_for(n, kBlock), kBlock, 0, s, st.tree, n, 0, k1, v1);
  VMO_LAUNCHED("tree_keys");
  VMO_TRY(radix_sort_u64(k1, v1, k2, v2, n, 64, s, sc));
  if (by_prob) {
    launch(k_tree_regather, grid_for(n, kBlock), kBlock, 0, s, v2, n, 1, st.tree, k1);
    VMO_LAUNCHED("tree_regather");
    VMO_TRY(radix_sort_u64(k1, v2, k2, v1, n, 32, s, sc));
    *idx_out = v1;
  } else {
    *idx_out = v2;
  }
  return VMO_OK;
}

// Cut-row/column ordering (Sec. 4.2): every separator stably sorted by b
// two-bit numbers of its vertices' links into the first / second parts of the
// splits of the node's descendants 1..b levels down (per pair BBD: 00, 01,
// 10, 11; SBD: 01, 00, 11, 10).  Applied after the recursion, when the
// separators are not recursed into.
vmo_status cut_order_pass(OrderState& st, const OrderParams& op, cudaStream_t s, Scratch& sc) {
  const int64_t n = st.n;
  const int b = op.cut_order;
  if (n == 0 || b <= 0) return VMO_OK;
  ScratchFrame frame(sc);
  int nrec = 0;
  uint32_t* idx;
  VMO_TRY(tree_sorted(st, true, &nrec, &idx, s, sc));
  if (nrec == 0) return VMO_OK;
  CutRec* cr;
  int32_t *own, *pos, *ord2;
  uint32_t* vcode;
  int64_t *sz, *gstart, *total;
  uint64_t *k1, *k2;
  uint32_t *v1, *v2;
  VMO_TRY(sc.alloc(&cr, nrec));
  VMO_TRY(sc.alloc(&own, n));
  VMO_TRY(sc.alloc(&pos, n));
  VMO_TRY(sc.alloc(&ord2, n));
  VMO_TRY(sc.alloc(&vcode, n));
  VMO_TRY(sc.alloc(&sz, nrec));
  VMO_TRY(sc.alloc(&gstart, nrec));
  VMO_TRY(sc.alloc(&total, 1));
  VMO_TRY(sc.alloc(&k1, n));
  VMO_TRY(sc.alloc(&k2, n));
  VMO_TRY(sc.alloc(&v1, n));
  VMO_TRY(sc.alloc(&v2, n));
  VMO_CUDA(cudaMemsetAsync(own, 0xFF, n * sizeof(int32_t), s));  // every position is owned; -1 would be skipped
  launch(k_cut_recs, grid_for((int64_t)nrec * 32, kBlock), kBlock, 0, s, st.tree, idx, nrec, op.sbd, cr, own, sz);
  launch(k_inverse_perm, grid_for(n, kBlock), kBlock, 0, s, st.ord, n, pos);
  launch(k_cut_codes, grid_for(n, kBlock), kBlock, 0, s, st.ord, pos, own, n, cr, st.adj_ptr, st.adj, b, vcode);
  const uint64_t sentinel = (uint64_t)nrec << (2 * b);
  int bits = 1;
  while (bits < 64 && (1ull << bits) <= sentinel) ++bits;
  launch(k_cut_keys, grid_for(n, kBlock), kBlock, 0, s, st.ord, own, n, cr, vcode, st.mu, op.sbd, b, sentinel, k1,
         v1);
  VMO_LAUNCHED("cut_codes");
  VMO_TRY(scan_exclusive<int64_t>(sz, gstart, nrec, total, s, sc));
  int64_t m = 0;
  VMO_CUDA(cudaMemcpyAsync(&m, total, 8, cudaMemcpyDeviceToHost, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  if (m == 0) return VMO_OK;
  VMO_TRY(radix_sort_u64(k1, v1, k2, v2, n, bits, s, sc));
  VMO_CUDA(cudaMemcpyAsync(ord2, st.ord, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  launch(k_cut_scatter, grid_for(m, kBlock), kBlock, 0, s, k2, v2, m, b, cr, gstart, st.ord, ord2);
  VMO_LAUNCHED("cut_scatter");
  VMO_CUDA(cudaMemcpyAsync(st.ord, ord2, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  return VMO_OK;
}

vmo_status gather_coords(const float4* x, const int32_t* ord, int64_t n, float4* xo, cudaStream_t s) {
  if (n <= 0) return VMO_OK;
  launch(k_gather_coords, grid_for(n, kBlock), kBlock, 0, s, x, ord, n, xo);
  VMO_LAUNCHED("gather_coords");
  return VMO_OK;
}

vmo_status tree_write(OrderState& st, const uint32_t* idx, int n, uint64_t* heap, int32_t* offset, int32_t* n1,
                      int32_t* n2, int32_t* nsep, int32_t* depth, int32_t* prob, cudaStream_t s) {
  if (n == 0) return VMO_OK;
  launch(k_tree_out, grid_for(n, kBlock), kBlock, 0, s, idx, n, st.tree, heap, offset, n1, n2, nsep, depth, prob);
  VMO_LAUNCHED("tree_out");
  return VMO_OK;
}

}  // namespace vmo
