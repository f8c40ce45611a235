// 2-means bisection that allocates no device memory.
//
// For callers that must not allocate: for example code whose device memory
// is entirely owned by another allocator or budget, or a latency-critical
// loop in which an allocation could block.  vmo_bisect takes its scratch from
// the stream-ordered pool; this variant runs the same kernels on a fixed
// file-scope device array instead.  The array holds the working set of at
// most kNoAllocMaxPoints points, stays resident on every GPU that loads the
// library until the process exits, and is shared by all calls: calls that
// overlap on the GPU (other streams, other threads) race on it.
#include <algorithm>
#include <cstring>

#include "order.cuh"

namespace vmo {

namespace {

constexpr int64_t kNoAllocMaxPoints = 131072;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffXo = 0;
constexpr size_t kOffDval = align256(kOffXo + kNoAllocMaxPoints * sizeof(float4));
constexpr size_t kOffDpre = align256(kOffDval + kNoAllocMaxPoints * sizeof(unsigned long long));
constexpr size_t kOffOrd = align256(kOffDpre + kNoAllocMaxPoints * sizeof(unsigned long long));
constexpr size_t kOffSeg = align256(kOffOrd + kNoAllocMaxPoints * sizeof(int32_t));
constexpr size_t kOffLab = align256(kOffSeg + kNoAllocMaxPoints * sizeof(int32_t));
constexpr size_t kOffPart = align256(kOffLab + kNoAllocMaxPoints);
constexpr size_t kOffNode = align256(kOffPart + ((kNoAllocMaxPoints + 2047) / 2048) * sizeof(uint64_t));
constexpr size_t kOffSeed = align256(kOffNode + sizeof(NodeDev));
constexpr size_t kOffCnt = align256(kOffSeed + sizeof(uint64_t));
constexpr size_t kScratchBytes = align256(kOffCnt + sizeof(int));

static __device__ __align__(256) unsigned char g_bisect_scratch[kScratchBytes];

// Device address of g_bisect_scratch on the current device (host code must
// not use the symbol itself: on the host it is only a stand-in).  Looked up on
// every call rather than cached: the lookup allocates nothing, and after a
// device reset the library's device code is loaded again and the array may
// then sit at another address.
vmo_status scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_bisect_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_bisect_scratch)", __FILE__, __LINE__);
  *out = static_cast<unsigned char*>(p);
  return VMO_OK;
}

}  // namespace

vmo_status bisect_noalloc(int32_t d, const float* coords, const int32_t* verts, int32_t nverts, uint64_t seed,
                          uint64_t key, int32_t km_iters, uint8_t* labels, float* z, int32_t* split, cudaStream_t s) {
  if (d < 2 || d > 4) return unsupported("d must be 2, 3 or 4");
  if (nverts < 0 || km_iters < 0) return invalid("negative size");
  if (nverts > kNoAllocMaxPoints)
    return invalid("vmo_bisect_noalloc: nverts = " + std::to_string(nverts) + " exceeds the fixed scratch limit of " +
                   std::to_string(kNoAllocMaxPoints) + " points (use vmo_bisect)");
  if (nverts > 0 && (!coords || !verts || !labels || ((uintptr_t)coords & 15u)))
    return invalid("null or unaligned argument");
  if (scan_partials_needed(nverts) * (int64_t)sizeof(uint64_t) > (int64_t)(kOffNode - kOffPart))
    return invalid("vmo_bisect_noalloc: scan partials exceed their slot");
  unsigned char* base;
  VMO_TRY(scratch_address(&base));
  float zh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int32_t sp = 0;
  if (nverts >= 2) {
    OrderState st;
    st.n = nverts;
    st.xo = reinterpret_cast<float4*>(base + kOffXo);
    st.ord = reinterpret_cast<int32_t*>(base + kOffOrd);
    st.seg = reinterpret_cast<int32_t*>(base + kOffSeg);
    st.lab = base + kOffLab;
    st.nodes = reinterpret_cast<NodeDev*>(base + kOffNode);
    st.seeds = reinterpret_cast<uint64_t*>(base + kOffSeed);
    VMO_CUDA(cudaMemcpyAsync(st.ord, verts, nverts * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    VMO_CUDA(cudaMemsetAsync(st.seg, 0, nverts * sizeof(int32_t), s));  // every point in node 0
    VMO_CUDA(cudaMemcpyAsync(st.seeds, &seed, sizeof(seed), cudaMemcpyHostToDevice, s));
    NodeDev nd;
    memset(&nd, 0, sizeof(nd));
    nd.heap = key;
    nd.size = nverts;
    VMO_CUDA(cudaMemcpyAsync(st.nodes, &nd, sizeof(nd), cudaMemcpyHostToDevice, s));
    VMO_TRY(gather_coords(reinterpret_cast<const float4*>(coords), st.ord, nverts, st.xo, s));
    VMO_TRY(two_means_into(st, 1, d, km_iters, reinterpret_cast<unsigned long long*>(base + kOffDval),
                           reinterpret_cast<unsigned long long*>(base + kOffDpre), reinterpret_cast<int*>(base + kOffCnt),
                           reinterpret_cast<uint64_t*>(base + kOffPart), s));
    VMO_CUDA(cudaMemcpyAsync(&nd, st.nodes, sizeof(nd), cudaMemcpyDeviceToHost, s));
    VMO_CUDA(cudaStreamSynchronize(s));
    zh[0] = nd.z1.x; zh[1] = nd.z1.y; zh[2] = nd.z1.z; zh[3] = nd.z1.w;
    if (nd.state == 2) {
      VMO_CUDA(cudaMemsetAsync(labels, 1, nverts, s));
    } else {
      VMO_CUDA(cudaMemcpyAsync(labels, st.lab, nverts, cudaMemcpyDeviceToDevice, s));
      zh[4] = nd.z2.x; zh[5] = nd.z2.y; zh[6] = nd.z2.z; zh[7] = nd.z2.w;
      sp = (nd.n1 > 0 && nd.n2 > 0) ? 1 : 0;
    }
  } else if (nverts == 1) {
    VMO_CUDA(cudaMemsetAsync(labels, 1, 1, s));
  }
  if (z) VMO_CUDA(cudaMemcpyAsync(z, zh, sizeof(zh), cudaMemcpyHostToDevice, s));
  VMO_CUDA(cudaStreamSynchronize(s));
  if (split) *split = sp;
  return VMO_OK;
}

}  // namespace vmo

extern "C" vmo_status vmo_bisect_noalloc(int32_t d, const float* coords, const int32_t* verts, int32_t nverts,
                                         uint64_t seed, uint64_t key, int32_t km_iters, uint8_t* labels, float* z,
                                         int32_t* split, void* stream) {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    (void)cudaGetLastError();
    return vmo::cuda_fail(e == cudaSuccess ? cudaErrorNoDevice : e, "no usable CUDA device", __FILE__, __LINE__);
  }
  return vmo::bisect_noalloc(d, coords, verts, nverts, seed, key, km_iters, labels, z, split, (cudaStream_t)stream);
}
