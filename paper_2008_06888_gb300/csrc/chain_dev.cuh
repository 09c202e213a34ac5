// chain_dev.cuh -- device helpers shared by the compiled kernels and by the
// register-chain kernels generated and compiled at run time (NVRTC), so that
// both build bit-identical gate tables.  Needs tn_internal.h.
#pragma once
#include "tn_internal.h"

namespace tn {

template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 t; };
template <> struct Vec2<int32_t> { typedef int2 t; };
template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 t; };
template <> struct Vec4<int32_t> { typedef int4 t; };

// Pointer of instance blockIdx.y in a batch whose arena slices are ib bytes apart.
template <typename P>
__device__ __forceinline__ P *inst_ptr(P *p, int64_t ib) {
  return reinterpret_cast<P *>(reinterpret_cast<char *>(const_cast<void *>(
                                   static_cast<const void *>(p))) + blockIdx.y * ib);
}

// Asynchronous 4-, 8- and 16-byte global -> shared copies (cp.async) and their groups.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 16 bytes, cached in L2 only (a streamed tile is not re-read)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 16 bytes through L1 (the lanes that share a 32-byte sector are served by one
// sector read even where their shared-memory destinations are apart)
__device__ __forceinline__ void cp_async16ca(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ void build_tables(const ChainParams &p, const T *X, T *sT) {
  // one table value per thread at a time; its components load together
  for (int i = threadIdx.x; i < p.ttotal; i += blockDim.x) {
    int k = 0;
    while (k + 1 < p.ntg && p.tg[k + 1].toff <= i) ++k;
    const TGate &t = p.tg[k];
    const int li = i - t.toff;
    T val[TN_TG_MAXC];
#pragma unroll
    for (int c = 0; c < TN_TG_MAXC; ++c) {
      if (c >= t.ncomp) break;
      const ChainGate &g = p.g[t.cg[c]];
      const int64_t st[4] = {g.sBk, g.sBn, g.sBb[0], g.sBb[1]};
      int64_t o = 0;
#pragma unroll
      for (int l = 0; l < 4; ++l)
        if (t.cbit[c][l] >= 0) o += (int64_t)((li >> t.cbit[c][l]) & 1) * st[l];
      val[c] = X[g.offB + o];
    }
    T acc = val[0];
#pragma unroll
    for (int c = 1; c < TN_TG_MAXC; ++c)
      if (c < t.ncomp) acc = acc + val[c];
    sT[i] = acc;
  }
}

}  // namespace tn
