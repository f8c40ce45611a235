// Internal declarations of the VMO CUDA library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "../../include/vmo.h"

namespace vmo {

// ---------------------------------------------------------------------------
// Errors: a failing call records a message for vmo_last_error() and returns a
// status; nothing throws across the C-ABI.
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);

struct Status {
  vmo_status code = VMO_OK;
  bool ok() const { return code == VMO_OK; }
};

#define VMO_TRY(expr)                          \
  do {                                         \
    vmo_status _s = (expr);                    \
    if (_s != VMO_OK) return _s;               \
  } while (0)

vmo_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define VMO_CUDA(call)                                                   \
  do {                                                                   \
    cudaError_t _e = (call);                                             \
    if (_e != cudaSuccess) return ::vmo::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define VMO_LAUNCHED(name)                                                     \
  do {                                                                         \
    cudaError_t _e = cudaGetLastError();                                       \
    if (_e != cudaSuccess) return ::vmo::cuda_fail(_e, name, __FILE__, __LINE__); \
  } while (0)

vmo_status invalid(const std::string& msg);
vmo_status unsupported(const std::string& msg);

// ---------------------------------------------------------------------------
// Device memory.  Scratch of one call is taken from the stream-ordered pool
// (cudaMallocAsync) and released on the same stream when the call ends.
// ---------------------------------------------------------------------------
struct Scratch {
  cudaStream_t stream = nullptr;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : stream(s) {}
  ~Scratch();
  template <class T>
  vmo_status alloc(T** p, size_t count) {
    return alloc_bytes(reinterpret_cast<void**>(p), count * sizeof(T));
  }
  vmo_status alloc_bytes(void** p, size_t bytes);
  size_t mark() const { return ptrs.size(); }
  void release_to(size_t m);  // frees (stream-ordered) everything allocated after mark m
};

// Returns the scratch taken inside a scope to the pool when the scope ends.
struct ScratchFrame {
  Scratch& sc;
  size_t m;
  explicit ScratchFrame(Scratch& s) : sc(s), m(s.mark()) {}
  ~ScratchFrame() { sc.release_to(m); }
};

// Stream for the allocations of DevArray in the calling thread.  By default a
// DevArray uses cudaMalloc / cudaFree; inside a DevArrayStreamScope it takes
// its memory from the stream-ordered pool on the scope's stream and returns it
// on that stream, so threads working on different streams (the request
// server's slots) never wait for each other in an allocation or a free.
extern std::atomic<uint64_t> g_device_allocs;
extern thread_local cudaStream_t g_devarray_stream;
extern thread_local bool g_devarray_async;

struct DevArrayStreamScope {
  cudaStream_t prev_s;
  bool prev_a;
  explicit DevArrayStreamScope(cudaStream_t s) : prev_s(g_devarray_stream), prev_a(g_devarray_async) {
    g_devarray_stream = s;
    g_devarray_async = true;
  }
  ~DevArrayStreamScope() {
    g_devarray_stream = prev_s;
    g_devarray_async = prev_a;
  }
};

// Persistent device buffer owned by a handle.
template <class T>
struct DevArray {
  T* ptr = nullptr;
  size_t count = 0;
  bool async = false;            // allocated from the stream-ordered pool
  cudaStream_t astream = nullptr;
  vmo_status resize(size_t n);  // contents not preserved
  void release();
  ~DevArray() { release(); }
  DevArray() = default;
  DevArray(const DevArray&) = delete;
  DevArray& operator=(const DevArray&) = delete;
};

template <class T>
vmo_status DevArray<T>::resize(size_t n) {
  if (n <= count && ptr) return VMO_OK;
  release();
  if (n == 0) n = 1;
  const bool as = g_devarray_async;
  cudaError_t e = as ? cudaMallocAsync(reinterpret_cast<void**>(&ptr), n * sizeof(T), g_devarray_stream)
                     : cudaMalloc(reinterpret_cast<void**>(&ptr), n * sizeof(T));
  if (e != cudaSuccess) {
    ptr = nullptr;
    (void)cudaGetLastError();
    set_error("device allocation of " + std::to_string(n * sizeof(T)) + " bytes failed");
    return VMO_ERR_OOM;
  }
  count = n;
  async = as;
  astream = g_devarray_stream;
  g_device_allocs.fetch_add(1, std::memory_order_relaxed);
  return VMO_OK;
}

template <class T>
void DevArray<T>::release() {
  if (ptr) {
    if (async) cudaFreeAsync(ptr, astream);
    else cudaFree(ptr);
  }
  ptr = nullptr;
  count = 0;
}

// ---------------------------------------------------------------------------
// Hypergraph handle.
// ---------------------------------------------------------------------------
struct Graph {
  // Adjacency CSR over global vertex ids, with optional per-entry edge costs
  // and per-vertex weights (null = 1).
  int64_t k = 0;
  int64_t nadj = 0;
  const int32_t* adj_ptr = nullptr;  // k+1 (int32 offsets)
  const int32_t* adj = nullptr;
  const float* acost = nullptr;      // nadj or null
  const float* w = nullptr;          // k or null
};

}  // namespace vmo

struct vmo_hg_s {
  vmo_model model;
  int32_t m = 0, n = 0;
  int32_t k = 0;        // vertices
  int64_t l = 0;        // nets
  vmo::DevArray<int32_t> adj_ptr, adj;      // graph models
  vmo::DevArray<int32_t> net_ptr, pins;     // all models
  vmo::DevArray<int32_t> vtx_ptr, vnets;    // all models
  vmo::DevArray<float> weight;              // optional vertex weights
  int64_t nadj = 0, npins = 0, nvnets = 0;
  bool has_weight = false;
  int device = 0;
};

namespace vmo {

// ---------------------------------------------------------------------------
// Primitives (prims.cu).
// ---------------------------------------------------------------------------
// Exclusive scan of n values; if total != nullptr the sum is written there
// (device).  In-place (in == out) is allowed.
template <class T>
vmo_status scan_exclusive(const T* in, T* out, int64_t n, T* total, cudaStream_t s, Scratch& sc);
template <class T>
vmo_status scan_inclusive(const T* in, T* out, int64_t n, cudaStream_t s, Scratch& sc);

// Inclusive scan that allocates nothing: `partial` must hold
// scan_partials_needed(n) values.
vmo_status scan_inclusive_u64_into(const uint64_t* in, uint64_t* out, int64_t n, uint64_t* partial, cudaStream_t s);
int64_t scan_partials_needed(int64_t n);

// Segment map for the radix sort: tiles never straddle segments.
struct SortSegments {
  int32_t nseg = 1;               // number of segments
  const int64_t* seg_base = nullptr;  // device, nseg+1 element offsets (null: one segment [0, n))
  const int32_t* tile_seg = nullptr;  // device, per tile: segment
  const int64_t* tile_start = nullptr;// device, per tile: first element
  const int32_t* tile_count = nullptr;// device, per tile: elements
  const int32_t* seg_tile0 = nullptr; // device, per segment: first tile (nseg+1)
  int64_t ntiles = 0;
  const int32_t* long_seg = nullptr;  // device, segments of more than kLongSegTiles tiles
  int32_t nlong = 0;
  int32_t nmid = 0;                   // segments of 2..kLongSegTiles tiles
};
constexpr int kLongSegTiles = 16;
constexpr int kSortTile = 2048;  // 256 threads x 8 keys

// Stable LSD radix sort of (key, value) pairs on bits [0, bits).  Keys are
// sorted within each segment.  Buffers are ping-ponged; the sorted result ends
// in (keys_out, vals_out).  vals may be null (keys only).
vmo_status radix_sort_u32(uint32_t* keys_in, uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                          int64_t n, int bits, const SortSegments* segs, cudaStream_t s, Scratch& sc);
// Same sort without the final copy: the sorted keys and values are left in
// (keys_b, vals_b) if *in_b, else in (keys_a, vals_a); the other pair is
// overwritten.
vmo_status radix_sort_u32_pingpong(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b, uint32_t* vals_b, int64_t n,
                                  int bits, const SortSegments* segs, bool* in_b, cudaStream_t s, Scratch& sc);
vmo_status radix_sort_u64(uint64_t* keys_in, uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                          int64_t n, int bits, cudaStream_t s, Scratch& sc);

// Build SortSegments for segments given by host base offsets.
vmo_status make_sort_segments(const std::vector<int64_t>& seg_base_host, SortSegments* out, cudaStream_t s,
                              Scratch& sc);

// ---------------------------------------------------------------------------
// Instrumentation: every kernel launch of the library goes through launch(),
// which counts it; the layout step kernel can also be timed with CUDA events
// and can count the interactions it evaluates (vmo_stats_* in the C-ABI).
// ---------------------------------------------------------------------------
extern std::atomic<uint64_t> g_launches;
bool stats_timing();
unsigned long long* stats_interaction_counter();  // null unless counting is on
void stats_time_begin(cudaStream_t s);
void stats_time_end(cudaStream_t s, uint64_t points);

// Programmatic dependent launch: inside a PdlScope the calling thread's
// launches carry the programmatic-serialization attribute, so a kernel's launch
// is processed while its predecessor in the stream still runs.  Every kernel
// launched that way starts with pdl_wait(), which returns once the preceding
// kernel has completed and its writes are visible (and at once when the kernel
// was launched without the attribute).
extern thread_local bool g_pdl;

// Launch-shape choices that never change a result (tune.cu): the largest
// step launch that takes the variant with two far-field rows in flight, the
// widest radix digit, and the positions per thread of the Lloyd assignment.
// Process-wide; set by vmo_set_tuning / vmo_autotune.
struct Tuning {
  std::atomic<int64_t> small_step_threads{152 * 4 * 32};
  std::atomic<int> radix_max_bits{10};
  std::atomic<int> assign_items{4};  // 4 measured best for a million-point Lloyd round (8 and 2 slower)
  std::atomic<int> small_bin_points{kSortTile};
};
extern Tuning g_tuning;
struct PdlScope {
  bool prev;
  PdlScope() : prev(g_pdl) { g_pdl = true; }
  ~PdlScope() { g_pdl = prev; }
};

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... KArgs, class... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  } else {
    kernel<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
  }
}

inline int bits_for(uint64_t maxval) {
  int b = 0;
  while (b < 64 && (maxval >> b) != 0) ++b;
  return b;
}

inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// ---------------------------------------------------------------------------
// Device helpers.  Floating point that decides an integer uses explicitly
// rounded intrinsics so the compiler cannot contract or reorder it.
// ---------------------------------------------------------------------------
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kTagCoord = 0x636f6f7264000000ull;   // initial layout
constexpr uint64_t kTagKmeans = 0x6b6d65616e730000ull;  // k-means++ draws
constexpr uint64_t kTagMatch = 0x6d61746368000000ull;   // matching tie-breaks
constexpr uint64_t kTagJitter = 0x6a69747465720000ull;  // prolongation jitter

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t rand64(uint64_t seed, uint64_t a, uint64_t b) {
  return mix64(mix64(seed + kGolden * (a + 1)) + kGolden * (b + 1));
}

// floor(n * r / 2^64)
__device__ inline uint64_t scale_draw(uint64_t n, uint64_t r) { return __umul64hi(n, r); }

// Exponent e with max |x| < 2^e (0 for max = 0) from the float bits of the max
// (the fixed-point grid of the k-means sums is 2^-(30 - e)).
__device__ inline int exponent_of(uint32_t maxbits) {
  float mx = __uint_as_float(maxbits);
  if (mx == 0.0f) return 0;
  int e;
  frexpf(mx, &e);
  return e;
}

// Order-preserving map float -> uint32 (for atomicMin/Max on floats).
__device__ inline uint32_t f2ord(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ inline float ord2f(uint32_t u) {
  uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}

// Exact 2^e as float for -126 <= e <= 127.
__device__ inline float exp2i_f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// Squared distance of two points in fp32, coordinates 0..d-1 in order, no FMA.
template <int D>
__device__ inline float sqdist32(const float4& a, const float4& b) {
  float q = __fsub_rn(a.x, b.x);
  float s = __fmul_rn(q, q);
  if (D > 1) { q = __fsub_rn(a.y, b.y); s = __fadd_rn(s, __fmul_rn(q, q)); }
  if (D > 2) { q = __fsub_rn(a.z, b.z); s = __fadd_rn(s, __fmul_rn(q, q)); }
  if (D > 3) { q = __fsub_rn(a.w, b.w); s = __fadd_rn(s, __fmul_rn(q, q)); }
  return s;
}

__device__ inline float comp(const float4& v, int m) {
  return m == 0 ? v.x : (m == 1 ? v.y : (m == 2 ? v.z : v.w));
}

__device__ inline unsigned lane_id() { return threadIdx.x & 31u; }

}  // namespace vmo
