// noalloc.cu -- fixed device scratch for tn_energy_noalloc.
//
// Some callers cannot allocate device memory when they want a ground-state
// energy: code that records work inside a CUDA stream capture (cudaMalloc is
// not allowed while capturing), frameworks whose caching allocator owns the
// whole device, and latency-bound loops that cannot afford the implicit
// device synchronisation of cudaMalloc/cudaFree.  For them the contraction
// can run in this file-scope array instead of a context-owned arena.  The
// array is part of the module image: every GPU that loads libtn.so holds its
// TN_NOALLOC_SCRATCH_BYTES until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "kernels.h"

#define TN_NOALLOC_SCRATCH_BYTES (32ull << 20)

static __device__ __align__(256) char g_noalloc_scratch[TN_NOALLOC_SCRATCH_BYTES];

namespace tn {

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
char *g_addr[kMaxDevices] = {};
}  // namespace

size_t noalloc_scratch_bytes() { return TN_NOALLOC_SCRATCH_BYTES; }

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
cudaError_t noalloc_scratch(char **ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<char *>(p);
  }
  *ptr = g_addr[dev];
  return cudaSuccess;
}

// Leaf descriptors travel as kernel parameters (copied into the launch by
// the driver, and by value into a graph node when the launch is captured),
// so no host-to-device copy and no device buffer is needed for them.
struct LeafArg {
  int64_t off_x;       // byte offset of the leaf's values in the scratch
  int32_t edge, u, v;
  int32_t bits;        // bit 0: isolated spin (kind 1); bit 1: fu; bit 2: fv
};
constexpr int kLeafChunk = 1024;   // 24 KiB of parameters per launch
struct LeafChunk {
  int32_t n;
  LeafArg L[kLeafChunk];
};
static_assert(sizeof(LeafChunk) <= 32000, "kernel parameter space");

template <typename T> __device__ __forceinline__ T leaf_val(float x);
template <> __device__ __forceinline__ float leaf_val<float>(float x) { return x; }
template <> __device__ __forceinline__ int32_t leaf_val<int32_t>(float x) {
  return (int32_t)lrintf(x);
}

// Bond tensor [[J, -J], [-J, J]] with the absorbed fields diag(h, -h) (Sec.
// II), or the Potts bond J delta(a, b); one thread per leaf element.
template <typename T>
__global__ void k_leaves_param(const LeafChunk c, int q, const float *__restrict__ J,
                               const float *__restrict__ h, char *scratch) {
  const int per = q * q;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= c.n * per) return;
  const LeafArg &L = c.L[tid / per];
  const int e = tid % per;
  T *out = reinterpret_cast<T *>(scratch + L.off_x);
  if (L.bits & 1) {              // isolated spin: a one-leg leaf [h, -h] (Potts: zeros)
    if (e >= q) return;
    T v = T(0);
    if (q == 2 && (L.bits & 2)) {
      T hu = leaf_val<T>(h[L.u]);
      v = e == 0 ? hu : -hu;
    }
    out[e] = v;
    return;
  }
  const int a = e / q, b = e % q;
  const T j = leaf_val<T>(J[L.edge]);
  T v;
  if (q == 2) {
    v = (a == b) ? j : -j;
    if (L.bits & 2) { T hu = leaf_val<T>(h[L.u]); v = v + (a == 0 ? hu : -hu); }
    if (L.bits & 4) { T hv = leaf_val<T>(h[L.v]); v = v + (b == 0 ? hv : -hv); }
  } else {
    v = (a == b) ? j : T(0);
  }
  out[a * q + b] = v;
}

cudaError_t launch_leaves_param(Dtype dt, int q, const LeafDesc *leaves, int nleaves,
                                const float *J, const float *h, char *scratch, cudaStream_t st) {
  static LeafChunk c;            // host staging of one launch's parameters
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  for (int b = 0; b < nleaves; b += kLeafChunk) {
    c.n = nleaves - b < kLeafChunk ? nleaves - b : kLeafChunk;
    for (int i = 0; i < c.n; ++i) {
      const LeafDesc &d = leaves[b + i];
      c.L[i] = LeafArg{d.off_x, d.edge, d.u, d.v, (d.kind == 1 ? 1 : 0) | (d.fu ? 2 : 0) |
                                                      (d.fv ? 4 : 0)};
    }
    const int threads = 256;
    const int blocks = (c.n * q * q + threads - 1) / threads;
    if (dt == DT_F32)
      k_leaves_param<float><<<blocks, threads, 0, st>>>(c, q, J, h, scratch);
    else
      k_leaves_param<int32_t><<<blocks, threads, 0, st>>>(c, q, J, h, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
__global__ void k_energy_out(const T *root, float *E) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *E = -(float)(*root);
}

cudaError_t launch_energy_out(Dtype dt, const void *root, float *E, cudaStream_t st) {
  if (dt == DT_F32)
    k_energy_out<float><<<1, 32, 0, st>>>(static_cast<const float *>(root), E);
  else
    k_energy_out<int32_t><<<1, 32, 0, st>>>(static_cast<const int32_t *>(root), E);
  return cudaGetLastError();
}

}  // namespace tn
