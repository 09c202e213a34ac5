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
