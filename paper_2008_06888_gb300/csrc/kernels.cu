// kernels.cu -- CUDA kernels of the tropical contraction (sm_103a).
//
// Element algebra (Eq. 2): (+) = max, (.) = +.  Counting tuples (Sec. II):
// (x1, n1) (.) (x2, n2) = (x1 + x2, n1 n2); (+) keeps the larger x and adds
// the counts on a tie.  Counts are residues modulo 61-bit primes 2^61 - c.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>
#include <cstdlib>
#include <stdint.h>

#include "kernels.h"
#include "perm_bits.h"
#include "chain_dev.cuh"
#include "modarith.cuh"

namespace tn {

// ---------------------------------------------------------------- helpers

template <typename T> struct Lim;
template <> struct Lim<float> {
  __device__ __forceinline__ static float neg() { return -INFINITY; }
};
template <> struct Lim<int32_t> {
  // Integer stand-in for -inf: NEG + NEG = INT32_MIN does not overflow, and
  // |real values| stay far below 2^29.
  __device__ __forceinline__ static int32_t neg() { return -(1 << 30); }
};

// modular arithmetic of the residue planes: modarith.cuh

// Streaming multiprocessors of the current device (GB300: 152), queried once
// per device; grid sizes are multiples of it.
int num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
    return 152;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// Resident blocks of `kernel` on the device (occupancy of its registers and
// shared memory), queried once per kernel.
template <typename K>
static int64_t resident_slots(K kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, int> per_sm;   // (kernel, device)
  int dev = 0;
  cudaGetDevice(&dev);
  const std::pair<const void *, int> key(reinterpret_cast<const void *>(kernel), dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = per_sm.find(key);
  if (it == per_sm.end()) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, smem) != cudaSuccess ||
        v <= 0)
      v = 1;
    it = per_sm.emplace(key, v).first;
  }
  return (int64_t)it->second * num_sms();
}

// Blocks per instance of a grid-stride kernel with `need` blocks of work per
// instance, B instances and `slots` resident blocks: whole waves when a
// multiple of the slots is within 16 waves, else about 8 waves so the last,
// partial one is a small part of the launch.
static int64_t wave_blocks(int64_t need, int B, int64_t slots) {
  if (need * B <= slots) return need;
  const int64_t whole = slots / std::gcd(slots, (int64_t)B);
  if (whole <= need && whole * B <= 16 * slots) return whole;
  return std::min(need, std::max<int64_t>(1, 8 * slots / B));
}

static inline int grid_for(int64_t n, int threads, int max_blocks = 0) {
  if (max_blocks <= 0) max_blocks = num_sms() * 32;
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// ---------------------------------------------------------------- leaves

template <typename T> __device__ __forceinline__ T to_val(float x);
template <> __device__ __forceinline__ float to_val<float>(float x) { return x; }
template <> __device__ __forceinline__ int32_t to_val<int32_t>(float x) { return (int32_t)lrintf(x); }

// Bond tensor [[J, -J], [-J, J]] (Sec. II) plus the absorbed vertex tensors
// diag(h, -h); Potts bond J delta(a, b).  One thread per leaf element.
template <typename T, typename R>
__global__ void k_leaves(const LeafDesc *__restrict__ d, int nleaves, int q,
                         const float *__restrict__ J, const float *__restrict__ h, char *arena,
                         int P, int64_t jstride, int64_t hstride, int64_t ib) {
  // instance blockIdx.y: its couplings and its slice of the arena
  J += blockIdx.y * jstride;
  h += blockIdx.y * hstride;
  arena += blockIdx.y * ib;
  const int per = q * q;
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)nleaves * per) return;
  const LeafDesc L = d[tid / per];
  int e = (int)(tid % per);
  int a, b;
  T v;
  if (L.kind == 0) {
    a = e / q;
    b = e % q;
    T j = to_val<T>(J[L.edge]);
    if (q == 2) {
      int sa = a == 0 ? 1 : -1, sb = b == 0 ? 1 : -1;
      v = (sa * sb > 0) ? j : -j;
      if (L.fu) { T hu = to_val<T>(h[L.u]); v = v + (sa > 0 ? hu : -hu); }
      if (L.fv) { T hv = to_val<T>(h[L.v]); v = v + (sb > 0 ? hv : -hv); }
    } else {
      v = (a == b) ? j : T(0);
    }
  } else {
    if (e >= q) return;
    a = e;
    b = 0;
    v = T(0);
    if (q == 2 && L.fu) { T hu = to_val<T>(h[L.u]); v = (a == 0) ? hu : -hu; }
  }
  int idx = (L.kind == 0) ? a * q + b : a;
  reinterpret_cast<T *>(arena + L.off_x)[idx] = v;
  if (P > 0) {
    R *n = reinterpret_cast<R *>(arena + L.off_n);
    for (int i = 0; i < P; ++i) n[i * L.plane + idx] = R(1);
  }
}

cudaError_t launch_leaves(Dtype dt, int q, const LeafDesc *d_leaves, int nleaves, const float *J,
                          const float *h, char *arena, int P, int rbytes, const Batch &bt,
                          cudaStream_t st) {
  if (nleaves == 0) return cudaSuccess;
  int64_t total = (int64_t)nleaves * q * q;
  int threads = 256;
  dim3 grid((unsigned)((total + threads - 1) / threads), bt.B);
#define TN_LEAVES(T_, R_)                                                                       \
  k_leaves<T_, R_><<<grid, threads, 0, st>>>(d_leaves, nleaves, q, J, h, arena, P, bt.jstride, \
                                            bt.hstride, bt.ib)
  if (dt == DT_F32) {
    if (rbytes == 4) TN_LEAVES(float, uint32_t); else TN_LEAVES(float, uint64_t);
  } else {
    if (rbytes == 4) TN_LEAVES(int32_t, uint32_t); else TN_LEAVES(int32_t, uint64_t);
  }
#undef TN_LEAVES
  return cudaGetLastError();
}

// ---------------------------------------------------------------- gate contraction

// C[o, n] = max_k A[o, k] + B[o, k, n], one outer index per thread.
template <typename T, bool COUNT, typename R = uint64_t>
__global__ void __launch_bounds__(256) k_gate(const GateParams p, const T *__restrict__ A,
                                              const T *__restrict__ B, T *__restrict__ C,
                                              const R *__restrict__ nA,
                                              const R *__restrict__ nB,
                                              R *__restrict__ nC, const PrimeSet ps,
                                              int64_t ib) {
  A = inst_ptr(A, ib);
  C = inst_ptr(C, ib);
  if (p.hasB) B = inst_ptr(B, ib);
  if (COUNT) {
    nA = inst_ptr(nA, ib);
    nC = inst_ptr(nC, ib);
    if (p.hasB) nB = inst_ptr(nB, ib);
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < p.outer; o += stride) {
    int64_t r = o, oa = 0, ob = 0, oc = 0;
    for (int s = p.nseg - 1; s >= 0; --s) {
      int64_t i;
      if (p.seg_sh[s] >= 0) {
        i = r & (p.seg_size[s] - 1);
        r >>= p.seg_sh[s];
      } else {
        i = r % p.seg_size[s];
        r /= p.seg_size[s];
      }
      oa += i * p.seg_sA[s];
      ob += i * p.seg_sB[s];
      oc += i * p.seg_sC[s];
    }
    for (int n = 0; n < p.Ns; ++n) {
      T best = Lim<T>::neg();
      R cnt[TN_MAX_PRIMES];
#pragma unroll
      for (int i = 0; i < TN_MAX_PRIMES; ++i) cnt[i] = 0;
      for (int k = 0; k < p.Ks; ++k) {
        T v = A[oa + p.kA[k]];
        if (p.hasB) v = v + B[ob + p.kB[k] + p.nB[n]];
        bool gt = (k == 0) || (v > best);
        if (COUNT) {
          bool eq = !gt && (v == best);
          if (gt || eq) {
#pragma unroll
            for (int i = 0; i < TN_MAX_PRIMES; ++i) {
              if (i < p.P) {
                R na = nA[i * p.planeA + oa + p.kA[k]];
                R t = (p.hasB && !p.unitB)
                          ? mulmodR(na, nB[i * p.planeB + ob + p.kB[k] + p.nB[n]], ps.c[i])
                          : na;
                cnt[i] = gt ? t : addmodR(cnt[i], t, ps.c[i]);
              }
            }
          }
        }
        if (gt) best = v;
      }
      C[oc + p.nC[n]] = best;
      if (COUNT) {
#pragma unroll
        for (int i = 0; i < TN_MAX_PRIMES; ++i)
          if (i < p.P) nC[i * p.planeC + oc + p.nC[n]] = cnt[i];
      }
    }
  }
}

// Values-only gate contraction with the numbers of contracted and new states
// known at compile time (the common 1 / 2 cases): offsets held in registers,
// two outer indices per thread for independent loads.
template <typename T, int KS, int NS>
__global__ void __launch_bounds__(256) k_gate_t(const GateParams p, const T *__restrict__ A,
                                                const T *__restrict__ B, T *__restrict__ C,
                                                int64_t ib) {
  A = inst_ptr(A, ib);
  C = inst_ptr(C, ib);
  if (p.hasB) B = inst_ptr(B, ib);
  int64_t kA[KS], kB[KS], nB[NS], nC[NS];
#pragma unroll
  for (int k = 0; k < KS; ++k) { kA[k] = p.kA[k]; kB[k] = p.kB[k]; }
#pragma unroll
  for (int n = 0; n < NS; ++n) { nB[n] = p.nB[n]; nC[n] = p.nC[n]; }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o0 < p.outer; o0 += 2 * stride) {
    int64_t oa[2], ob[2], oc[2];
    bool live[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t o = o0 + u * stride;
      live[u] = o < p.outer;
      int64_t r = live[u] ? o : 0;
      oa[u] = ob[u] = oc[u] = 0;
      for (int s = p.nseg - 1; s >= 0; --s) {
        int64_t i;
        if (p.seg_sh[s] >= 0) {
          i = r & (p.seg_size[s] - 1);
          r >>= p.seg_sh[s];
        } else {
          i = r % p.seg_size[s];
          r /= p.seg_size[s];
        }
        oa[u] += i * p.seg_sA[s];
        ob[u] += i * p.seg_sB[s];
        oc[u] += i * p.seg_sC[s];
      }
    }
    T a[2][KS];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int k = 0; k < KS; ++k) a[u][k] = live[u] ? A[oa[u] + kA[k]] : T(0);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!live[u]) continue;
#pragma unroll
      for (int n = 0; n < NS; ++n) {
        T best = a[u][0] + (p.hasB ? B[ob[u] + kB[0] + nB[n]] : T(0));
#pragma unroll
        for (int k = 1; k < KS; ++k)
          best = max(best, a[u][k] + (p.hasB ? B[ob[u] + kB[k] + nB[n]] : T(0)));
        C[oc[u] + nC[n]] = best;
      }
    }
  }
}

template <typename T>
static bool launch_gate_t(const GateParams &p, const T *A, const T *B, T *C, dim3 blocks,
                          int threads, int64_t ib, cudaStream_t st) {
#define TN_GATE_CASE(KS_, NS_)                                                                 \
  if (p.Ks == KS_ && p.Ns == NS_) {                                                            \
    k_gate_t<T, KS_, NS_><<<blocks, threads, 0, st>>>(p, A, B, C, ib);                         \
    return true;                                                                               \
  }
  TN_GATE_CASE(1, 1)
  TN_GATE_CASE(1, 2)
  TN_GATE_CASE(2, 1)
  TN_GATE_CASE(2, 2)
  TN_GATE_CASE(4, 1)
  TN_GATE_CASE(1, 4)
#undef TN_GATE_CASE
  return false;
}

// ---- streaming q = 2 gate contractions (values).
//
// When every size is a power of two, C keeps A's leg order with the K leg
// removed and the N leg (if any) innermost, an output index is
// (j, n) with j the outer index: A's offset is j with a 0/1 digit inserted at
// bit pk of the contracted leg, and B reduces to a table over (k, n) and at
// most two batch digits of j.  Each thread maps 4 consecutive j to one or
// two 16-byte loads of A per digit and one or two 16-byte stores of C.
struct Gate2 {
  int pk;          // bit of the contracted leg in A's offset (KS == 2)
  int nbd;         // batch legs (digits of j read by B)
  int pb[2];       // their bits in j
  int64_t sb[2];   // their strides in B
};

template <typename T, int KS, int NS>
__global__ void __launch_bounds__(256) k_gate2(const GateParams p, const Gate2 g,
                                               const T *__restrict__ A, const T *__restrict__ B,
                                               T *__restrict__ C, int64_t ib) {
  typedef typename Vec4<T>::t V;
  A = inst_ptr(A, ib);
  C = inst_ptr(C, ib);
  if (p.hasB) B = inst_ptr(B, ib);
  __shared__ T sBt[16];   // index: bd0 | bd1 << 1 | k << 2 | n << 3
  if (threadIdx.x < 16) {
    const int i = threadIdx.x, b0 = i & 1, b1 = (i >> 1) & 1, k = (i >> 2) & 1, n = (i >> 3) & 1;
    T v = T(0);
    if (p.hasB && k < KS && n < NS && (b0 == 0 || g.nbd > 0) && (b1 == 0 || g.nbd > 1))
      v = B[p.kB[k] + p.nB[n] + b0 * g.sb[0] + b1 * g.sb[1]];
    sBt[i] = v;
  }
  __syncthreads();
  const int pb0 = g.nbd > 0 ? g.pb[0] : 62, pb1 = g.nbd > 1 ? g.pb[1] : 62;
  const int pk = g.pk;
  const int64_t nq = p.outer >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t0 < nq; t0 += 2 * stride) {
    T a[2][KS][4];
    bool live[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t t = t0 + u * stride;
      live[u] = t < nq;
      const int64_t j0 = (live[u] ? t : 0) << 2;
      if (KS == 1) {
        const V v = *reinterpret_cast<const V *>(A + j0);
        a[u][0][0] = v.x; a[u][0][1] = v.y; a[u][0][2] = v.z; a[u][0][3] = v.w;
      } else if (pk >= 2) {
        const int64_t lo = j0 & ((int64_t(1) << pk) - 1);
        const int64_t base = ((j0 >> pk) << (pk + 1)) | lo;
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          const V v = *reinterpret_cast<const V *>(A + base + ((int64_t)k << pk));
          a[u][k][0] = v.x; a[u][k][1] = v.y; a[u][k][2] = v.z; a[u][k][3] = v.w;
        }
      } else {
        // the contracted leg is one of the two lowest bits: 8 contiguous values
        const V v0 = *reinterpret_cast<const V *>(A + 2 * j0);
        const V v1 = *reinterpret_cast<const V *>(A + 2 * j0 + 4);
        const T blk[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4)
#pragma unroll
          for (int k = 0; k < KS; ++k)
            a[u][k][q4] = pk == 0 ? blk[2 * q4 + k] : blk[((q4 >> 1) << 2) | (k << 1) | (q4 & 1)];
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!live[u]) continue;
      const int64_t j0 = (t0 + u * stride) << 2;
      T out[4 * NS];
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const int64_t j = j0 + q4;
        const int bd = (int)((j >> pb0) & 1) | ((int)((j >> pb1) & 1) << 1);
#pragma unroll
        for (int n = 0; n < NS; ++n) {
          T best = a[u][0][q4] + sBt[bd | (n << 3)];
#pragma unroll
          for (int k = 1; k < KS; ++k) best = max(best, a[u][k][q4] + sBt[bd | (k << 2) | (n << 3)]);
          out[NS * q4 + n] = best;
        }
      }
#pragma unroll
      for (int h = 0; h < NS; ++h) {
        V v;
        v.x = out[4 * h + 0]; v.y = out[4 * h + 1]; v.z = out[4 * h + 2]; v.w = out[4 * h + 3];
        *reinterpret_cast<V *>(C + NS * j0 + 4 * h) = v;
      }
    }
  }
}

// Whether a (values) gate has the streaming q = 2 form; fills g.
static bool gate2_form(const GateParams &p, const void *A, const void *B, const void *C,
                       int64_t ib, size_t elem, Gate2 *g) {
  if (p.P > 0 || p.outer < 4 || (p.outer & 3)) return false;
  if (!((p.Ks == 1 || p.Ks == 2) && (p.Ns == 1 || p.Ns == 2))) return false;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(C)) % 16 ||
      ib % 16)
    return false;
  (void)elem;
  (void)B;
  *g = Gate2{};
  g->pk = 0;
  if (p.Ks == 2) {
    if (p.kA[0] != 0 || p.kA[1] <= 0 || (p.kA[1] & (p.kA[1] - 1))) return false;
    while ((int64_t(1) << g->pk) < p.kA[1]) g->pk++;
  }
  if (p.Ns == 2 && (p.nC[0] != 0 || p.nC[1] != 1)) return false;
  // segments slowest first: dense in C (times Ns), A = C's layout with pk inserted
  int64_t js = 1;
  for (int s = p.nseg - 1; s >= 0; --s) {
    if (p.seg_sh[s] < 0) return false;
    if (p.seg_sC[s] != js * p.Ns) return false;
    const int64_t a = (p.Ks == 2 && js >= (int64_t(1) << g->pk)) ? 2 * js : js;
    if (p.Ks == 2 && js < (int64_t(1) << g->pk) && js * p.seg_size[s] > (int64_t(1) << g->pk))
      return false;
    if (p.seg_sA[s] != a) return false;
    if (p.seg_sB[s] != 0) {
      if (!p.hasB || p.seg_size[s] != 2 || g->nbd >= 2) return false;
      int b = 0;
      while ((int64_t(1) << b) < js) ++b;
      g->pb[g->nbd] = b;
      g->sb[g->nbd] = p.seg_sB[s];
      g->nbd++;
    }
    js *= p.seg_size[s];
  }
  return js == p.outer;
}

// Counting form of k_gate2: the same index map, with the P residue planes of
// every element moved alongside its value (two 16-byte accesses per plane for
// four outer indices).  Per output the terms are taken in k order: the first
// term and every larger one replace (value, counts), an equal one adds its
// counts mod p -- the rule of k_gate, so the results are identical.
// four consecutive residues (16-byte aligned): two 16-byte accesses for 8-byte
// residues, one for 4-byte ones
__device__ __forceinline__ void ld4(const uint64_t *p, uint64_t *o) {
  const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(p);
  const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(p + 2);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4(const uint32_t *p, uint32_t *o) {
  const uint4 a = *reinterpret_cast<const uint4 *>(p);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void st4(uint64_t *p, const uint64_t *v) {
  *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(v[0], v[1]);
  *reinterpret_cast<ulonglong2 *>(p + 2) = make_ulonglong2(v[2], v[3]);
}
__device__ __forceinline__ void st4(uint32_t *p, const uint32_t *v) {
  *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1], v[2], v[3]);
}

template <typename T, int KS, int NS, int P, typename R = uint64_t>
__global__ void __launch_bounds__(256) k_gate2c(const GateParams p, const Gate2 g,
                                                const T *__restrict__ A, const T *__restrict__ B,
                                                T *__restrict__ C,
                                                const R *__restrict__ nA,
                                                const R *__restrict__ nB,
                                                R *__restrict__ nC, const PrimeSet ps,
                                                int64_t ib) {
  typedef typename Vec4<T>::t V;
  A = inst_ptr(A, ib);
  C = inst_ptr(C, ib);
  nA = inst_ptr(nA, ib);
  nC = inst_ptr(nC, ib);
  if (p.hasB) {
    B = inst_ptr(B, ib);
    nB = inst_ptr(nB, ib);
  }
  __shared__ T sBt[16];            // index: bd0 | bd1 << 1 | k << 2 | n << 3
  __shared__ R sBn[P][16];
  const bool mulB = p.hasB && !p.unitB;
  if (threadIdx.x < 16) {
    const int i = threadIdx.x, b0 = i & 1, b1 = (i >> 1) & 1, k = (i >> 2) & 1, n = (i >> 3) & 1;
    const bool ok = p.hasB && k < KS && n < NS && (b0 == 0 || g.nbd > 0) && (b1 == 0 || g.nbd > 1);
    const int64_t off = ok ? p.kB[k] + p.nB[n] + b0 * g.sb[0] + b1 * g.sb[1] : 0;
    sBt[i] = ok ? B[off] : T(0);
#pragma unroll
    for (int r = 0; r < P; ++r) sBn[r][i] = (ok && mulB) ? nB[r * p.planeB + off] : R(1);
  }
  __syncthreads();
  const int pb0 = g.nbd > 0 ? g.pb[0] : 62, pb1 = g.nbd > 1 ? g.pb[1] : 62;
  const int pk = g.pk;
  const int64_t nq = p.outer >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nq; t += stride) {
    const int64_t j0 = t << 2;
    T a[KS][4];
    R na[P][KS][4];
    if (KS == 1 || pk >= 2) {
      int64_t base = j0;
      if (KS == 2) {
        const int64_t lo = j0 & ((int64_t(1) << pk) - 1);
        base = ((j0 >> pk) << (pk + 1)) | lo;
      }
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int64_t e = base + ((int64_t)k << pk);
        const V v = *reinterpret_cast<const V *>(A + e);
        a[k][0] = v.x; a[k][1] = v.y; a[k][2] = v.z; a[k][3] = v.w;
#pragma unroll
        for (int r = 0; r < P; ++r) ld4(nA + r * p.planeA + e, na[r][k]);
      }
    } else {
      // the contracted leg is one of the two lowest bits: 8 contiguous elements
      const V v0 = *reinterpret_cast<const V *>(A + 2 * j0);
      const V v1 = *reinterpret_cast<const V *>(A + 2 * j0 + 4);
      const T blk[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4)
#pragma unroll
        for (int k = 0; k < KS; ++k)
          a[k][q4] = pk == 0 ? blk[2 * q4 + k] : blk[((q4 >> 1) << 2) | (k << 1) | (q4 & 1)];
#pragma unroll
      for (int r = 0; r < P; ++r) {
        R cb[8];
        ld4(nA + r * p.planeA + 2 * j0, cb);
        ld4(nA + r * p.planeA + 2 * j0 + 4, cb + 4);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4)
#pragma unroll
          for (int k = 0; k < KS; ++k)
            na[r][k][q4] = pk == 0 ? cb[2 * q4 + k] : cb[((q4 >> 1) << 2) | (k << 1) | (q4 & 1)];
      }
    }
    T out[NS][4];
    R cout[P][NS][4];
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      const int64_t j = j0 + q4;
      const int bd = (int)((j >> pb0) & 1) | ((int)((j >> pb1) & 1) << 1);
#pragma unroll
      for (int n = 0; n < NS; ++n) {
        T best = a[0][q4] + sBt[bd | (n << 3)];
        R cnt[P];
#pragma unroll
        for (int r = 0; r < P; ++r)
          cnt[r] = mulB ? mulmodR(na[r][0][q4], sBn[r][bd | (n << 3)], ps.c[r]) : na[r][0][q4];
#pragma unroll
        for (int k = 1; k < KS; ++k) {
          const int bi = bd | (k << 2) | (n << 3);
          const T v = a[k][q4] + sBt[bi];
          if (v >= best) {
            const bool gt = v > best;
#pragma unroll
            for (int r = 0; r < P; ++r) {
              const R tr = mulB ? mulmodR(na[r][k][q4], sBn[r][bi], ps.c[r]) : na[r][k][q4];
              cnt[r] = gt ? tr : addmodR(cnt[r], tr, ps.c[r]);
            }
            best = gt ? v : best;
          }
        }
        out[n][q4] = best;
#pragma unroll
        for (int r = 0; r < P; ++r) cout[r][n][q4] = cnt[r];
      }
    }
    // C and its planes: new leg innermost, so the 4 * NS outputs are contiguous
#pragma unroll
    for (int h = 0; h < NS; ++h) {
      const int q0 = 4 * h;   // flat output index f = NS * q4 + n covers [q0, q0 + 4)
      T o4[4];
      R c4[P][4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int f = q0 + e, q4 = f / NS, n = f % NS;
        o4[e] = out[n][q4];
#pragma unroll
        for (int r = 0; r < P; ++r) c4[r][e] = cout[r][n][q4];
      }
      V v;
      v.x = o4[0]; v.y = o4[1]; v.z = o4[2]; v.w = o4[3];
      *reinterpret_cast<V *>(C + NS * j0 + q0) = v;
#pragma unroll
      for (int r = 0; r < P; ++r) st4(nC + r * p.planeC + NS * j0 + q0, c4[r]);
    }
  }
}

template <typename T>
static bool launch_gate2c(const GateParams &p, const T *A, const T *B, T *C, const uint64_t *nA,
                          const uint64_t *nB, uint64_t *nC, const PrimeSet &ps, const Batch &bt,
                          cudaStream_t st) {
  // 4 planes of 8-byte residues or 7 of 4-byte ones
  if (!((p.P == 4 && !ps.r32) || (p.P == 7 && ps.r32)) || std::getenv("TN_NO_GATE2")) return false;
  GateParams q = p;
  q.P = 0;   // gate2_form checks the value layout; the planes share it
  Gate2 g;
  if (!gate2_form(q, A, B, C, bt.ib, sizeof(T), &g)) return false;
  const int rb = ps.r32 ? 4 : 8;
  if ((reinterpret_cast<uintptr_t>(nA) | reinterpret_cast<uintptr_t>(nC)) % 16 ||
      (p.planeA * rb) % 16 || (p.planeC * rb) % 16)
    return false;
  const int64_t nq = p.outer >> 2;
  const int64_t need = (nq + 255) / 256;
#define TN_G2C(KS_, NS_, P_, R_)                                                                 \
  if (p.Ks == KS_ && p.Ns == NS_) {                                                            \
    const int64_t blocks =                                                                     \
        wave_blocks(need, bt.B, resident_slots(k_gate2c<T, KS_, NS_, P_, R_>, 256, 0));        \
    k_gate2c<T, KS_, NS_, P_, R_><<<dim3((unsigned)blocks, bt.B), 256, 0, st>>>(               \
        p, g, A, B, C, reinterpret_cast<const R_ *>(nA), reinterpret_cast<const R_ *>(nB),     \
        reinterpret_cast<R_ *>(nC), ps, bt.ib);                                                \
    return true;                                                                               \
  }
  if (ps.r32) {
    TN_G2C(1, 1, 7, uint32_t)
    TN_G2C(1, 2, 7, uint32_t)
    TN_G2C(2, 1, 7, uint32_t)
    TN_G2C(2, 2, 7, uint32_t)
  } else {
    TN_G2C(1, 1, 4, uint64_t)
    TN_G2C(1, 2, 4, uint64_t)
    TN_G2C(2, 1, 4, uint64_t)
    TN_G2C(2, 2, 4, uint64_t)
  }
#undef TN_G2C
  return false;
}

template <typename T>
static bool launch_gate2(const GateParams &p, const T *A, const T *B, T *C, const Batch &bt,
                         cudaStream_t st) {
  Gate2 g;
  if (std::getenv("TN_NO_GATE2") || !gate2_form(p, A, B, C, bt.ib, sizeof(T), &g)) return false;
  const int64_t nq = p.outer >> 2;
  const int64_t need = (nq + 511) / 512;
#define TN_G2(KS_, NS_)                                                                        \
  if (p.Ks == KS_ && p.Ns == NS_) {                                                            \
    const int64_t blocks = wave_blocks(need, bt.B, resident_slots(k_gate2<T, KS_, NS_>, 256, 0)); \
    k_gate2<T, KS_, NS_><<<dim3((unsigned)blocks, bt.B), 256, 0, st>>>(p, g, A, B, C, bt.ib);  \
    return true;                                                                               \
  }
  TN_G2(1, 1)
  TN_G2(1, 2)
  TN_G2(2, 1)
  TN_G2(2, 2)
#undef TN_G2
  return false;
}

cudaError_t launch_gate(Dtype dt, const GateParams &p, const void *xA, const void *xB, void *xC,
                        const uint64_t *nA, const uint64_t *nB, uint64_t *nC, const PrimeSet &ps,
                        const Batch &bt, cudaStream_t st) {
  if (p.outer == 0) return cudaSuccess;
  int threads = 256;
  dim3 blocks(grid_for(p.outer, threads), bt.B);
  bool cnt = p.P > 0;
  if (!cnt) {
    const bool streamed = dt == DT_F32
                              ? launch_gate2<float>(p, (const float *)xA, (const float *)xB,
                                                    (float *)xC, bt, st)
                              : launch_gate2<int32_t>(p, (const int32_t *)xA, (const int32_t *)xB,
                                                      (int32_t *)xC, bt, st);
    if (streamed) return cudaGetLastError();
    dim3 b2(grid_for((p.outer + 1) / 2, threads), bt.B);
    const bool done = dt == DT_F32
                          ? launch_gate_t<float>(p, (const float *)xA, (const float *)xB,
                                                 (float *)xC, b2, threads, bt.ib, st)
                          : launch_gate_t<int32_t>(p, (const int32_t *)xA, (const int32_t *)xB,
                                                   (int32_t *)xC, b2, threads, bt.ib, st);
    if (done) return cudaGetLastError();
  } else {
    const bool streamed =
        dt == DT_F32 ? launch_gate2c<float>(p, (const float *)xA, (const float *)xB, (float *)xC,
                                            nA, nB, nC, ps, bt, st)
                     : launch_gate2c<int32_t>(p, (const int32_t *)xA, (const int32_t *)xB,
                                              (int32_t *)xC, nA, nB, nC, ps, bt, st);
    if (streamed) return cudaGetLastError();
    if (ps.r32 && !std::getenv("TN_NO_GATE_TC")) {
      const uint32_t *a = (const uint32_t *)nA, *b = (const uint32_t *)nB;
      uint32_t *c = (uint32_t *)nC;
      if (dt == DT_F32 ? launch_gate_tc_f32(p, xA, xB, xC, a, b, c, ps, bt, st)
                       : launch_gate_tc_i32(p, xA, xB, xC, a, b, c, ps, bt, st))
        return cudaGetLastError();
    }
  }
  if (cnt && ps.r32) {
    const uint32_t *a = (const uint32_t *)nA, *b = (const uint32_t *)nB;
    uint32_t *c = (uint32_t *)nC;
    if (dt == DT_F32)
      k_gate<float, true, uint32_t><<<blocks, threads, 0, st>>>(
          p, (const float *)xA, (const float *)xB, (float *)xC, a, b, c, ps, bt.ib);
    else
      k_gate<int32_t, true, uint32_t><<<blocks, threads, 0, st>>>(
          p, (const int32_t *)xA, (const int32_t *)xB, (int32_t *)xC, a, b, c, ps, bt.ib);
    return cudaGetLastError();
  }
  if (dt == DT_F32) {
    if (cnt)
      k_gate<float, true><<<blocks, threads, 0, st>>>(p, (const float *)xA, (const float *)xB,
                                                      (float *)xC, nA, nB, nC, ps, bt.ib);
    else
      k_gate<float, false><<<blocks, threads, 0, st>>>(p, (const float *)xA, (const float *)xB,
                                                       (float *)xC, nA, nB, nC, ps, bt.ib);
  } else {
    if (cnt)
      k_gate<int32_t, true><<<blocks, threads, 0, st>>>(p, (const int32_t *)xA, (const int32_t *)xB,
                                                        (int32_t *)xC, nA, nB, nC, ps, bt.ib);
    else
      k_gate<int32_t, false><<<blocks, threads, 0, st>>>(p, (const int32_t *)xA,
                                                         (const int32_t *)xB, (int32_t *)xC, nA, nB,
                                                         nC, ps, bt.ib);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- register-tiled max-plus GEMM
//
// 128 x 128 output tile per block of 256 threads, 8 x 8 outputs per thread,
// k slabs of 16 staged in shared memory by cp.async (two stages).  The
// tropical multiply-add of two consecutive k is done with two adds and one
// three-input max (FP32), the fastest form measured on GB300; INT32 uses the
// fused add-max (DPX) instruction.  Out-of-range operands read the tropical zero.

__device__ __forceinline__ float tmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ int32_t tmax3(int32_t a, int32_t b, int32_t c) {
  return max(max(a, b), c);
}
// acc (+)= a0 (.) b0 (+) a1 (.) b1: FP32 two adds and a three-input max; INT32
// two fused add-max instructions (DPX: max(a + b, c)), same integer result
__device__ __forceinline__ float tmac2(float acc, float a0, float b0, float a1, float b1) {
  return tmax3(acc, a0 + b0, a1 + b1);
}
__device__ __forceinline__ int32_t tmac2(int32_t acc, int32_t a0, int32_t b0, int32_t a1,
                                         int32_t b1) {
  return __viaddmax_s32(a1, b1, __viaddmax_s32(a0, b0, acc));
}

constexpr int GBM = 128, GBN = 128, GBK = 16, GPAD = 4;

template <typename T>
__device__ __forceinline__ void gemm_load_tile(const GemmParams &p, const T *Ab, const T *Bb,
                                               int64_t m0, int64_t n0, int64_t k0, T *As, T *Bs) {
  const int tid = threadIdx.x;
  const T *a0 = Ab + m0 * p.sAm + k0 * p.sAk;
  const T *b0 = Bb + k0 * p.sBk + n0 * p.sBn;
  const int64_t mr = p.M - m0, kr = p.K - k0, nr = p.N - n0;
  // A: GBM x GBK elements into As[k][m]
#pragma unroll 2
  for (int r = 0; r < (GBM * GBK) / 256; ++r) {
    const int idx = tid + r * 256;
    int m, k;
    if (p.sAk == 1) { m = idx / GBK; k = idx % GBK; } else { k = idx / GBM; m = idx % GBM; }
    T *dst = As + k * (GBM + GPAD) + m;
    if (m < mr && k < kr) cp_async4(dst, a0 + m * p.sAm + k * p.sAk);
    else *dst = Lim<T>::neg();
  }
  // B: GBK x GBN elements into Bs[k][n]
#pragma unroll 2
  for (int r = 0; r < (GBN * GBK) / 256; ++r) {
    const int idx = tid + r * 256;
    int n, k;
    if (p.sBn == 1) { k = idx / GBN; n = idx % GBN; } else { n = idx / GBK; k = idx % GBK; }
    T *dst = Bs + k * (GBN + GPAD) + n;
    if (n < nr && k < kr) cp_async4(dst, b0 + k * p.sBk + n * p.sBn);
    else *dst = Lim<T>::neg();
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_mpgemm(const GemmParams p, const T *__restrict__ A,
                                                   const T *__restrict__ B, T *__restrict__ C,
                                                   int64_t ib) {
  A = inst_ptr(A, ib);
  B = inst_ptr(B, ib);
  C = inst_ptr(C, ib);
  __shared__ __align__(16) T As[2][GBK][GBM + GPAD];
  __shared__ __align__(16) T Bs[2][GBK][GBN + GPAD];
  const int64_t mt = (p.M + GBM - 1) / GBM, nt = (p.N + GBN - 1) / GBN;
  const int64_t tiles = p.batch * mt * nt;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t ksteps = (p.K + GBK - 1) / GBK;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t b = t / (mt * nt);
    const int64_t rem = t % (mt * nt);
    const int64_t m0 = (rem / nt) * GBM, n0 = (rem % nt) * GBN;
    const T *Ab = A + b * p.sAb;
    const T *Bb = B + b * p.sBb;
    T acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = Lim<T>::neg();
    __syncthreads();
    gemm_load_tile<T>(p, Ab, Bb, m0, n0, 0, &As[0][0][0], &Bs[0][0][0]);
    cp_async_commit();
    for (int64_t ks = 0; ks < ksteps; ++ks) {
      const int cur = ks & 1;
      if (ks + 1 < ksteps)
        gemm_load_tile<T>(p, Ab, Bb, m0, n0, (ks + 1) * GBK, &As[cur ^ 1][0][0], &Bs[cur ^ 1][0][0]);
      cp_async_commit();
      cp_async_wait_prev();
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GBK; kk += 2) {
        T a0[8], a1[8], b0[8], b1[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          a0[i] = As[cur][kk][ty * 4 + i];
          a0[4 + i] = As[cur][kk][64 + ty * 4 + i];
          a1[i] = As[cur][kk + 1][ty * 4 + i];
          a1[4 + i] = As[cur][kk + 1][64 + ty * 4 + i];
          b0[i] = Bs[cur][kk][tx * 4 + i];
          b0[4 + i] = Bs[cur][kk][64 + tx * 4 + i];
          b1[i] = Bs[cur][kk + 1][tx * 4 + i];
          b1[4 + i] = Bs[cur][kk + 1][64 + tx * 4 + i];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = tmac2(acc[i][j], a0[i], b0[j], a1[i], b1[j]);
      }
      __syncthreads();
    }
    T *Cb = C + b * p.sCb;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
      if (gm >= p.M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
        if (gn < p.N) Cb[gm * p.sCm + gn * p.sCn] = acc[i][j];
      }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Fast path for A = [batch][M][K] and B = [batch][K][N] (both row-major, K and N
// multiples of 4, whole 128 x 128 x 16 tiles): each k slab moves as 16-byte
// cp.async chunks (cp_async16), A staged k-contiguous (As[m][k]) and read as
// 4-k vectors.

constexpr int GAK = GBK + 4;   // padded row of As[m][k]

template <typename T>
__global__ void __launch_bounds__(256, 2) k_mpgemm16(const GemmParams p, const T *__restrict__ A,
                                                     const T *__restrict__ B, T *__restrict__ C,
                                                     int64_t ib) {
  A = inst_ptr(A, ib);
  B = inst_ptr(B, ib);
  C = inst_ptr(C, ib);
  __shared__ __align__(16) T As[2][GBM][GAK];
  __shared__ __align__(16) T Bs[2][GBK][GBN + GPAD];
  const int64_t mt = p.M / GBM, nt = p.N / GBN;
  const int64_t tiles = p.batch * mt * nt;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t ksteps = p.K / GBK;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t b = t / (mt * nt);
    const int64_t rem = t % (mt * nt);
    const int64_t m0 = (rem / nt) * GBM, n0 = (rem % nt) * GBN;
    const T *Ab = A + b * p.sAb + m0 * p.sAm;
    const T *Bb = B + b * p.sBb + n0;
    auto load = [&](int64_t ks, int buf) {
      // A: 128 rows x 16 k = 512 chunks of 4; B: 16 rows x 128 n = 512 chunks of 4
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int c = tid + r * 256;
        const int am = c / 4, ak = (c % 4) * 4;
        cp_async16(&As[buf][am][ak], Ab + am * p.sAm + ks * GBK + ak);
        const int bk = c / 32, bn = (c % 32) * 4;
        cp_async16(&Bs[buf][bk][bn], Bb + (ks * GBK + bk) * p.sBk + bn);
      }
      cp_async_commit();
    };
    T acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = Lim<T>::neg();
    __syncthreads();
    load(0, 0);
    for (int64_t ks = 0; ks < ksteps; ++ks) {
      const int cur = ks & 1;
      if (ks + 1 < ksteps) load(ks + 1, cur ^ 1);
      else cp_async_commit();
      cp_async_wait_prev();
      __syncthreads();
#pragma unroll
      for (int kq = 0; kq < GBK; kq += 2) {
        // rows ty*4+i and 64+ty*4+i at k = kq, kq+1 (one 8-byte load per row)
        T a0[8], a1[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int m = i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4);
          const typename Vec2<T>::t v = *reinterpret_cast<const typename Vec2<T>::t *>(&As[cur][m][kq]);
          a0[i] = v.x;
          a1[i] = v.y;
        }
        T b0[8], b1[8];
        {
          typedef typename Vec4<T>::t V4;
          const V4 u0 = *reinterpret_cast<const V4 *>(&Bs[cur][kq][tx * 4]);
          const V4 u1 = *reinterpret_cast<const V4 *>(&Bs[cur][kq][64 + tx * 4]);
          const V4 w0 = *reinterpret_cast<const V4 *>(&Bs[cur][kq + 1][tx * 4]);
          const V4 w1 = *reinterpret_cast<const V4 *>(&Bs[cur][kq + 1][64 + tx * 4]);
          b0[0] = u0.x; b0[1] = u0.y; b0[2] = u0.z; b0[3] = u0.w;
          b0[4] = u1.x; b0[5] = u1.y; b0[6] = u1.z; b0[7] = u1.w;
          b1[0] = w0.x; b1[1] = w0.y; b1[2] = w0.z; b1[3] = w0.w;
          b1[4] = w1.x; b1[5] = w1.y; b1[6] = w1.z; b1[7] = w1.w;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = tmac2(acc[i][j], a0[i], b0[j], a1[i], b1[j]);
      }
      __syncthreads();
    }
    T *Cb = C + b * p.sCb;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
        Cb[gm * p.sCm + gn * p.sCn] = acc[i][j];
      }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

static bool mpgemm16_ok(const GemmParams &p, const void *A, const void *B) {
  return p.sAk == 1 && p.sBn == 1 && p.M % GBM == 0 && p.N % GBN == 0 && p.K % GBK == 0 &&
         p.sAm % 4 == 0 && p.sBk % 4 == 0 && p.sAb % 4 == 0 && p.sBb % 4 == 0 &&
         (reinterpret_cast<uintptr_t>(A) % 16) == 0 && (reinterpret_cast<uintptr_t>(B) % 16) == 0;
}

// ---- tile autotuner.  Candidates: staging (0: 16-byte cp.async, 1: 4-byte)
// x resident blocks per SM (2 or 8).  Every candidate computes each output as
// the max of the same single-rounding sums, so results are bit-identical and
// only time decides.  A shape class is timed once, on its first launch
// outside stream capture (its last candidate run leaves the result in C);
// choices can persist in the file named by TN_AUTOTUNE_CACHE.
struct GemmTile {
  int variant, per_sm;
};

static std::mutex g_tune_mu;
static std::map<std::string, GemmTile> g_tune;
static bool g_tune_loaded = false;
static thread_local bool g_tune_off = false;   // set by callers that must not wait

bool set_gemm_autotune(bool on) {
  const bool was = !g_tune_off;
  g_tune_off = !on;
  return was;
}

static std::string gemm_key(Dtype dt, const GemmParams &p, const Batch &bt, bool v16) {
  char k[192];
  std::snprintf(k, sizeof(k), "dt%d b%lld m%lld n%lld k%lld B%d ak%d bn%d v%d", (int)dt,
                (long long)p.batch, (long long)p.M, (long long)p.N, (long long)p.K, bt.B,
                (int)(p.sAk == 1), (int)(p.sBn == 1), (int)v16);
  return k;
}

static void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = std::getenv("TN_AUTOTUNE_CACHE");
  if (!path) return;
  FILE *f = std::fopen(path, "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof(line), f)) {
    char *bar = std::strchr(line, '|');
    if (!bar) continue;
    *bar = 0;
    GemmTile t{};
    if (std::sscanf(bar + 1, "%d %d", &t.variant, &t.per_sm) == 2) g_tune[line] = t;
  }
  std::fclose(f);
}

static void tune_store(const std::string &key, GemmTile t) {
  const char *path = std::getenv("TN_AUTOTUNE_CACHE");
  if (!path) return;
  if (FILE *f = std::fopen(path, "a")) {
    std::fprintf(f, "%s|%d %d\n", key.c_str(), t.variant, t.per_sm);
    std::fclose(f);
  }
}

static cudaError_t run_mpgemm(Dtype dt, const GemmParams &p, const void *A, const void *B, void *C,
                              const Batch &bt, cudaStream_t st, GemmTile t) {
  const int64_t tiles = p.batch * ((p.M + GBM - 1) / GBM) * ((p.N + GBN - 1) / GBN);
  const int64_t cap = std::max<int64_t>(1, num_sms() * t.per_sm / bt.B);
  dim3 blocks((unsigned)(tiles < cap ? tiles : cap), bt.B);
  if (t.variant == 0) {
    if (dt == DT_F32)
      k_mpgemm16<float><<<blocks, 256, 0, st>>>(p, (const float *)A, (const float *)B, (float *)C,
                                                bt.ib);
    else
      k_mpgemm16<int32_t><<<blocks, 256, 0, st>>>(p, (const int32_t *)A, (const int32_t *)B,
                                                  (int32_t *)C, bt.ib);
  } else {
    if (dt == DT_F32)
      k_mpgemm<float><<<blocks, 256, 0, st>>>(p, (const float *)A, (const float *)B, (float *)C,
                                              bt.ib);
    else
      k_mpgemm<int32_t><<<blocks, 256, 0, st>>>(p, (const int32_t *)A, (const int32_t *)B,
                                                (int32_t *)C, bt.ib);
  }
  return cudaGetLastError();
}

// ---- split-K form for steps with a handful of outputs and a long K (the
// contraction of two big tensors into the scalar root, or a few states):
// blocks take K ranges, reduce their maxima in shared memory and combine
// them with atomicMax on an order-preserving unsigned key written over C,
// decoded in place afterwards (max is exact, so the result equals the tiled
// kernel's).  Counting planes combine per-block sums mod p with a
// compare-and-swap add.
constexpr int kSplitOut = 16;          // largest batch * M * N of the split-K form
constexpr int64_t kSplitMinK = 1 << 14;

static bool splitk_ok(const GemmParams &p) {
  return p.batch * p.M * p.N <= kSplitOut && p.K >= kSplitMinK;
}

__device__ __forceinline__ uint32_t order_key(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ uint32_t order_key(int32_t x) { return (uint32_t)x ^ 0x80000000u; }
__device__ __forceinline__ void from_key(uint32_t k, float *x) {
  *x = __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ void from_key(uint32_t k, int32_t *x) { *x = (int32_t)(k ^ 0x80000000u); }

__device__ __forceinline__ void splitk_out(const GemmParams &p, int o, int64_t *oa, int64_t *ob,
                                           int64_t *oc) {
  const int64_t n = o % p.N, m = (o / p.N) % p.M, b = o / (p.N * p.M);
  *oa = b * p.sAb + m * p.sAm;
  *ob = b * p.sBb + n * p.sBn;
  *oc = b * p.sCb + m * p.sCm + n * p.sCn;
}

// phase 0: keys of the tropical zero; 2: decode keys into values
template <typename T>
__global__ void k_splitk_keys(const GemmParams p, T *C, int phase, int64_t ib) {
  C = inst_ptr(C, ib);
  const int o = threadIdx.x;
  if (o >= p.batch * p.M * p.N) return;
  int64_t oa, ob, oc;
  splitk_out(p, o, &oa, &ob, &oc);
  uint32_t *kc = reinterpret_cast<uint32_t *>(C + oc);
  if (phase == 0) *kc = 0u;
  else from_key(*kc, C + oc);
}

template <typename T>
__global__ void __launch_bounds__(256) k_mpgemm_splitk(const GemmParams p, const T *__restrict__ A,
                                                       const T *__restrict__ B, T *C, int64_t ib) {
  A = inst_ptr(A, ib);
  B = inst_ptr(B, ib);
  C = inst_ptr(C, ib);
  const int nout = (int)(p.batch * p.M * p.N);
  __shared__ uint32_t red[kSplitOut][8];
  for (int o = 0; o < nout; ++o) {
    int64_t oa, ob, oc;
    splitk_out(p, o, &oa, &ob, &oc);
    uint32_t best = 0u;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < p.K;
         k += (int64_t)gridDim.x * blockDim.x) {
      const T v = A[oa + k * p.sAk] + B[ob + k * p.sBk];
      best = max(best, order_key(v));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, d));
    if ((threadIdx.x & 31) == 0) red[o][threadIdx.x >> 5] = best;
  }
  __syncthreads();
  if (threadIdx.x < nout) {
    uint32_t best = 0u;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) best = max(best, red[threadIdx.x][w]);
    int64_t oa, ob, oc;
    splitk_out(p, threadIdx.x, &oa, &ob, &oc);
    atomicMax(reinterpret_cast<uint32_t *>(C + oc), best);
  }
}

// counting planes: n_i[o] = sum over k with A + B == C of nA_i nB_i (mod p_i)
// *dst = *dst + v (mod p) by compare-and-swap
__device__ __forceinline__ void cas_addmod(uint64_t *dst, uint64_t v, uint64_t c) {
  unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
  unsigned long long old = *d, assumed;
  do {
    assumed = old;
    old = atomicCAS(d, assumed, (unsigned long long)addmod61(assumed, v, c));
  } while (old != assumed);
}
__device__ __forceinline__ void cas_addmod(uint32_t *dst, uint32_t v, uint64_t c) {
  unsigned int *d = reinterpret_cast<unsigned int *>(dst);
  unsigned int old = *d, assumed;
  do {
    assumed = old;
    old = atomicCAS(d, assumed, addmod31(assumed, v, c));
  } while (old != assumed);
}

template <typename R>
__global__ void k_splitk_count_zero(const GemmParams p, R *nC, int64_t ib) {
  nC = inst_ptr(nC, ib);
  const int o = threadIdx.x;
  if (o >= p.batch * p.M * p.N) return;
  int64_t oa, ob, oc;
  splitk_out(p, o, &oa, &ob, &oc);
  for (int i = 0; i < p.P; ++i) nC[i * p.planeC + oc] = R(0);
}

template <typename T, typename R>
__global__ void __launch_bounds__(256) k_gemm_count_splitk(
    const GemmParams p, const T *__restrict__ A, const T *__restrict__ B, const T *__restrict__ C,
    const R *__restrict__ nA, const R *__restrict__ nB, R *nC,
    const PrimeSet ps, int64_t ib) {
  A = inst_ptr(A, ib);
  B = inst_ptr(B, ib);
  C = inst_ptr(C, ib);
  nA = inst_ptr(nA, ib);
  nB = inst_ptr(nB, ib);
  nC = inst_ptr(nC, ib);
  const int nout = (int)(p.batch * p.M * p.N);
  __shared__ R red[TN_MAX_PRIMES][8];
  for (int o = 0; o < nout; ++o) {
    int64_t oa, ob, oc;
    splitk_out(p, o, &oa, &ob, &oc);
    const T x = C[oc];
    R cnt[TN_MAX_PRIMES];
#pragma unroll
    for (int i = 0; i < TN_MAX_PRIMES; ++i) cnt[i] = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < p.K;
         k += (int64_t)gridDim.x * blockDim.x) {
      if (A[oa + k * p.sAk] + B[ob + k * p.sBk] == x) {
#pragma unroll
        for (int i = 0; i < TN_MAX_PRIMES; ++i)
          if (i < p.P)
            cnt[i] = addmodR(cnt[i], mulmodR(nA[i * p.planeA + oa + k * p.sAk],
                                             nB[i * p.planeB + ob + k * p.sBk], ps.c[i]),
                             ps.c[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < TN_MAX_PRIMES; ++i) {
      if (i >= p.P) break;
      R v = cnt[i];
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) v = addmodR(v, (R)__shfl_xor_sync(0xffffffffu, v, d), ps.c[i]);
      if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < p.P) {
      const int i = threadIdx.x;
      R v = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = addmodR(v, red[i][w], ps.c[i]);
      if (v) cas_addmod(nC + i * p.planeC + oc, v, ps.c[i]);
    }
    __syncthreads();
  }
}

static unsigned splitk_blocks(const GemmParams &p, const Batch &bt) {
  const int64_t want = (p.K + 256 * 16 - 1) / (256 * 16);   // about 16 k per thread
  const int64_t cap = std::max<int64_t>(1, (int64_t)num_sms() * 8 / bt.B);
  return (unsigned)std::max<int64_t>(1, std::min(want, cap));
}

template <typename T>
static cudaError_t launch_splitk(const GemmParams &p, const T *A, const T *B, T *C,
                                 const Batch &bt, cudaStream_t st) {
  k_splitk_keys<T><<<dim3(1, bt.B), 32, 0, st>>>(p, C, 0, bt.ib);
  k_mpgemm_splitk<T><<<dim3(splitk_blocks(p, bt), bt.B), 256, 0, st>>>(p, A, B, C, bt.ib);
  k_splitk_keys<T><<<dim3(1, bt.B), 32, 0, st>>>(p, C, 2, bt.ib);
  return cudaGetLastError();
}

template <typename T, typename R>
static cudaError_t launch_count_splitk(const GemmParams &p, const T *A, const T *B, const T *C,
                                       const R *nA, const R *nB, R *nC, const PrimeSet &ps,
                                       const Batch &bt, cudaStream_t st) {
  k_splitk_count_zero<R><<<dim3(1, bt.B), 32, 0, st>>>(p, nC, bt.ib);
  k_gemm_count_splitk<T, R><<<dim3(splitk_blocks(p, bt), bt.B), 256, 0, st>>>(
      p, A, B, C, nA, nB, nC, ps, bt.ib);
  return cudaGetLastError();
}

cudaError_t launch_mpgemm(Dtype dt, const GemmParams &p, const void *A, const void *B, void *C,
                          const Batch &bt, cudaStream_t st) {
  const int64_t tiles = p.batch * ((p.M + GBM - 1) / GBM) * ((p.N + GBN - 1) / GBN);
  if (tiles == 0) return cudaSuccess;
  if (splitk_ok(p)) {
    if (dt == DT_F32)
      return launch_splitk(p, (const float *)A, (const float *)B, (float *)C, bt, st);
    return launch_splitk(p, (const int32_t *)A, (const int32_t *)B, (int32_t *)C, bt, st);
  }
  const bool v16 = mpgemm16_ok(p, A, B) && bt.ib % 16 == 0 && std::getenv("TN_GEMM_SCALAR") == nullptr;
  // a forced candidate ("variant per_sm"), e.g. for tests
  if (const char *f = std::getenv("TN_GEMM_TILE")) {
    GemmTile t{1, 8};
    if (std::sscanf(f, "%d %d", &t.variant, &t.per_sm) == 2 && (t.variant == 1 || v16) &&
        t.per_sm > 0)
      return run_mpgemm(dt, p, A, B, C, bt, st, t);
  }
  const GemmTile fallback{v16 ? 0 : 1, 8};
  const std::string key = gemm_key(dt, p, bt, v16);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return run_mpgemm(dt, p, A, B, C, bt, st, it->second);
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (g_tune_off || std::getenv("TN_NO_AUTOTUNE") || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone)
    return run_mpgemm(dt, p, A, B, C, bt, st, fallback);
  std::vector<GemmTile> cand;
  for (int v = v16 ? 0 : 1; v <= 1; ++v)
    for (int per_sm : {2, 8}) cand.push_back({v, per_sm});
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  GemmTile best = fallback;
  float best_ms = 1e30f;
  for (const GemmTile &t : cand) {
    cudaError_t e = run_mpgemm(dt, p, A, B, C, bt, st, t);   // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = run_mpgemm(dt, p, A, B, C, bt, st, t);
    cudaEventRecord(e1, st);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return e != cudaSuccess ? e : cudaGetLastError();
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune.emplace(key, best).second) tune_store(key, best);
  }
  return run_mpgemm(dt, p, A, B, C, bt, st, best);
}

// Counting planes of a GEMM step: n_i[b,m,n] = sum over the k with
// A.x + B.x == C.x of A.n_i B.n_i (mod p_i).  One output per thread.
template <typename T, typename R>
__global__ void k_gemm_count(const GemmParams p, const T *__restrict__ A, const T *__restrict__ B,
                             const T *__restrict__ C, const R *__restrict__ nA,
                             const R *__restrict__ nB, R *__restrict__ nC,
                             const PrimeSet ps, int64_t ib) {
  A = inst_ptr(A, ib);
  B = inst_ptr(B, ib);
  C = inst_ptr(C, ib);
  nA = inst_ptr(nA, ib);
  nB = inst_ptr(nB, ib);
  nC = inst_ptr(nC, ib);
  const int64_t total = p.batch * p.M * p.N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t % p.N, m = (t / p.N) % p.M, b = t / (p.N * p.M);
    const int64_t oa = b * p.sAb + m * p.sAm, ob = b * p.sBb + n * p.sBn;
    const int64_t oc = b * p.sCb + m * p.sCm + n * p.sCn;
    const T x = C[oc];
    R cnt[TN_MAX_PRIMES];
#pragma unroll
    for (int i = 0; i < TN_MAX_PRIMES; ++i) cnt[i] = 0;
    for (int64_t k = 0; k < p.K; ++k) {
      if (A[oa + k * p.sAk] + B[ob + k * p.sBk] == x) {
#pragma unroll
        for (int i = 0; i < TN_MAX_PRIMES; ++i)
          if (i < p.P)
            cnt[i] = addmodR(cnt[i],
                             mulmodR(nA[i * p.planeA + oa + k * p.sAk],
                                     nB[i * p.planeB + ob + k * p.sBk], ps.c[i]),
                             ps.c[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < TN_MAX_PRIMES; ++i)
      if (i < p.P) nC[i * p.planeC + oc] = cnt[i];
  }
}

// Counting planes of a GEMM step, tiled: a block owns 32 x 32 outputs (lanes
// along n, each warp four rows), k slabs of 16 with the values and residues
// of A and B staged in shared memory, and C's values read once.  Each output
// sums the products of the counts over the k that reach its value.
constexpr int GCT = 32, GCK = 16;

template <typename T, typename R, int P>
__global__ void __launch_bounds__(256) k_gemm_count_t(const GemmParams p, const T *__restrict__ A,
                                                      const T *__restrict__ B,
                                                      const T *__restrict__ C,
                                                      const R *__restrict__ nA,
                                                      const R *__restrict__ nB,
                                                      R *__restrict__ nC, const PrimeSet ps,
                                                      int64_t ib) {
  A = inst_ptr(A, ib);
  B = inst_ptr(B, ib);
  C = inst_ptr(C, ib);
  nA = inst_ptr(nA, ib);
  nB = inst_ptr(nB, ib);
  nC = inst_ptr(nC, ib);
  __shared__ T sA[GCT][GCK + 1], sB[GCK][GCT];
  __shared__ R sAn[P][GCT][GCK + 1], sBn[P][GCK][GCT];
  __shared__ unsigned char okA[GCT][GCK + 1], okB[GCK][GCT];
  const int64_t tm = (p.M + GCT - 1) / GCT, tn = (p.N + GCT - 1) / GCT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t tile = blockIdx.x; tile < p.batch * tm * tn; tile += gridDim.x) {
    const int64_t b = tile / (tm * tn), m0 = (tile / tn) % tm * GCT, n0 = tile % tn * GCT;
    const int64_t n = n0 + tx;
    T x[4];
    R acc[4][P];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t m = m0 + ty * 4 + r;
      x[r] = (m < p.M && n < p.N) ? C[b * p.sCb + m * p.sCm + n * p.sCn] : T(0);
#pragma unroll
      for (int i = 0; i < P; ++i) acc[r][i] = 0;
    }
    for (int64_t k0 = 0; k0 < p.K; k0 += GCK) {
      __syncthreads();
      for (int e = threadIdx.x; e < GCT * GCK; e += 256) {
        // A tile [m][k] (k fastest), B tile [k][n] (n fastest)
        const int am = e / GCK, ak = e % GCK;
        const int64_t gm = m0 + am, gk = k0 + ak;
        const bool va = gm < p.M && gk < p.K;
        const int64_t oa = b * p.sAb + gm * p.sAm + gk * p.sAk;
        sA[am][ak] = va ? A[oa] : T(0);
        okA[am][ak] = va;
#pragma unroll
        for (int i = 0; i < P; ++i) sAn[i][am][ak] = va ? nA[i * p.planeA + oa] : R(0);
        const int bk = e / GCT, bn = e % GCT;
        const int64_t hk = k0 + bk, hn = n0 + bn;
        const bool vb = hk < p.K && hn < p.N;
        const int64_t ob = b * p.sBb + hk * p.sBk + hn * p.sBn;
        sB[bk][bn] = vb ? B[ob] : T(0);
        okB[bk][bn] = vb;
#pragma unroll
        for (int i = 0; i < P; ++i) sBn[i][bk][bn] = vb ? nB[i * p.planeB + ob] : R(0);
      }
      __syncthreads();
      const int kn = (int)((p.K - k0) < GCK ? (p.K - k0) : GCK);
      for (int k = 0; k < kn; ++k) {
        const T bv = sB[k][tx];
        const bool bok = okB[k][tx];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int am = ty * 4 + r;
          if (bok && okA[am][k] && sA[am][k] + bv == x[r]) {
#pragma unroll
            for (int i = 0; i < P; ++i)
              acc[r][i] = addmodR(acc[r][i], mulmodR(sAn[i][am][k], sBn[i][k][tx], ps.c[i]), ps.c[i]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t m = m0 + ty * 4 + r;
      if (m >= p.M || n >= p.N) continue;
      const int64_t oc = b * p.sCb + m * p.sCm + n * p.sCn;
#pragma unroll
      for (int i = 0; i < P; ++i) nC[i * p.planeC + oc] = acc[r][i];
    }
  }
}

template <typename T, typename R, int P>
static void launch_gemm_count_t(const GemmParams &p, const void *A, const void *B, const void *C,
                                const void *nA, const void *nB, void *nC, const PrimeSet &ps,
                                const Batch &bt, cudaStream_t st) {
  const int64_t tiles = p.batch * ((p.M + GCT - 1) / GCT) * ((p.N + GCT - 1) / GCT);
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * 8));
  k_gemm_count_t<T, R, P><<<dim3((unsigned)blocks, bt.B), 256, 0, st>>>(
      p, (const T *)A, (const T *)B, (const T *)C, (const R *)nA, (const R *)nB, (R *)nC, ps,
      bt.ib);
}

cudaError_t launch_gemm_count(Dtype dt, const GemmParams &p, const void *xA, const void *xB,
                              const void *xC, const uint64_t *nA, const uint64_t *nB, uint64_t *nC,
                              const PrimeSet &ps, const Batch &bt, cudaStream_t st) {
  int64_t total = p.batch * p.M * p.N;
  if (total == 0) return cudaSuccess;
  const uint32_t *a4 = (const uint32_t *)nA, *b4 = (const uint32_t *)nB;
  uint32_t *c4 = (uint32_t *)nC;
  if (splitk_ok(p)) {
    if (dt == DT_F32)
      return ps.r32 ? launch_count_splitk(p, (const float *)xA, (const float *)xB,
                                          (const float *)xC, a4, b4, c4, ps, bt, st)
                    : launch_count_splitk(p, (const float *)xA, (const float *)xB,
                                          (const float *)xC, nA, nB, nC, ps, bt, st);
    return ps.r32 ? launch_count_splitk(p, (const int32_t *)xA, (const int32_t *)xB,
                                        (const int32_t *)xC, a4, b4, c4, ps, bt, st)
                  : launch_count_splitk(p, (const int32_t *)xA, (const int32_t *)xB,
                                        (const int32_t *)xC, nA, nB, nC, ps, bt, st);
  }
  if (!std::getenv("TN_GEMM_COUNT_FLAT")) {
    // tiled forms for the residue layouts in use
    const bool f = dt == DT_F32;
    if (ps.r32 && p.P == 7) {
      if (f) launch_gemm_count_t<float, uint32_t, 7>(p, xA, xB, xC, nA, nB, nC, ps, bt, st);
      else launch_gemm_count_t<int32_t, uint32_t, 7>(p, xA, xB, xC, nA, nB, nC, ps, bt, st);
      return cudaGetLastError();
    }
    if (ps.r32 && p.P == 1) {
      if (f) launch_gemm_count_t<float, uint32_t, 1>(p, xA, xB, xC, nA, nB, nC, ps, bt, st);
      else launch_gemm_count_t<int32_t, uint32_t, 1>(p, xA, xB, xC, nA, nB, nC, ps, bt, st);
      return cudaGetLastError();
    }
    if (!ps.r32 && p.P == 4) {
      if (f) launch_gemm_count_t<float, uint64_t, 4>(p, xA, xB, xC, nA, nB, nC, ps, bt, st);
      else launch_gemm_count_t<int32_t, uint64_t, 4>(p, xA, xB, xC, nA, nB, nC, ps, bt, st);
      return cudaGetLastError();
    }
  }
  dim3 blocks(grid_for(total, 256), bt.B);
  if (dt == DT_F32) {
    if (ps.r32)
      k_gemm_count<float, uint32_t><<<blocks, 256, 0, st>>>(
          p, (const float *)xA, (const float *)xB, (const float *)xC, a4, b4, c4, ps, bt.ib);
    else
      k_gemm_count<float, uint64_t><<<blocks, 256, 0, st>>>(
          p, (const float *)xA, (const float *)xB, (const float *)xC, nA, nB, nC, ps, bt.ib);
  } else {
    if (ps.r32)
      k_gemm_count<int32_t, uint32_t><<<blocks, 256, 0, st>>>(
          p, (const int32_t *)xA, (const int32_t *)xB, (const int32_t *)xC, a4, b4, c4, ps, bt.ib);
    else
      k_gemm_count<int32_t, uint64_t><<<blocks, 256, 0, st>>>(
          p, (const int32_t *)xA, (const int32_t *)xB, (const int32_t *)xC, nA, nB, nC, ps, bt.ib);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- permutation

template <typename E>
__global__ void k_permute(const PermParams p, const E *__restrict__ in, E *__restrict__ out,
                          int64_t planeIn, int64_t planeOut, int64_t ib) {
  // blockIdx.y: residue plane, blockIdx.z: instance
  const E *src = reinterpret_cast<const E *>(reinterpret_cast<const char *>(in) + blockIdx.z * ib) +
                 blockIdx.y * planeIn;
  E *dst = reinterpret_cast<E *>(reinterpret_cast<char *>(out) + blockIdx.z * ib) +
           blockIdx.y * planeOut;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < p.total;
       o += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = o, off = 0;
    for (int j = p.r - 1; j >= 0; --j) {
      int64_t d = p.dims[j];
      off += (r % d) * p.sin[j];
      r /= d;
    }
    dst[o] = src[off];
  }
}

// ---- q = 2: tiled bit-permutation transpose (PermBits, perm_bits.h).

__device__ __forceinline__ int perm_swz(const PermBits &pb, int L) {
#pragma unroll
  for (int i = 0; i < 5; ++i)
    if (i < pb.nsw) L ^= ((L >> (5 + pb.sw_row[i])) & 1) << pb.sw_bank[i];
  return L;
}

template <typename E>
__global__ void __launch_bounds__(256) k_permute2(const PermBits pb, const E *__restrict__ in,
                                                  E *__restrict__ out, int64_t planeIn,
                                                  int64_t planeOut, int64_t ib) {
  // blockIdx.y: residue plane, blockIdx.z: instance
  const E *src = reinterpret_cast<const E *>(reinterpret_cast<const char *>(in) + blockIdx.z * ib) +
                 blockIdx.y * planeIn;
  E *dst = reinterpret_cast<E *>(reinterpret_cast<char *>(out) + blockIdx.z * ib) +
           blockIdx.y * planeOut;
  __shared__ E tile[1024];
  const int n = 1 << pb.nT;
  // this thread's elements of every tile: local index j = tid + 256 i
  int rl[4], wl[4];
  int64_t ro[4], wo[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = threadIdx.x + 256 * i;
    int L = 0;
    int64_t oi = 0, oo = 0;
    for (int t = 0; t < pb.nT; ++t)
      if ((j >> t) & 1) {
        L |= 1 << pb.rd_local[t];
        oi += int64_t(1) << pb.rd_in[t];
        oo += int64_t(1) << pb.wr_out[t];
      }
    rl[i] = perm_swz(pb, L);
    ro[i] = oi;
    wl[i] = perm_swz(pb, j);
    wo[i] = oo;
  }
  for (int64_t tau = blockIdx.x; tau < pb.tiles; tau += gridDim.x) {
    int64_t bin = 0, bout = 0;
    for (int g = 0; g < pb.nseg; ++g) {
      const int64_t v = (tau >> pb.seg_t[g]) & ((int64_t(1) << pb.seg_len[g]) - 1);
      bin += v << pb.seg_in[g];
      bout += v << pb.seg_out[g];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (threadIdx.x + 256 * i < n) tile[rl[i]] = src[bin + ro[i]];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (threadIdx.x + 256 * i < n) dst[bout + wo[i]] = tile[wl[i]];
    __syncthreads();
  }
}

cudaError_t launch_permute(const PermParams &p, const void *xin, void *xout, const uint64_t *nin,
                           uint64_t *nout, const Batch &bt, cudaStream_t st) {
  if (p.total == 0) return cudaSuccess;
  PermBits pb;
  if (perm_bits(p, &pb)) {
    // a few tiles per block; instances and residue planes on the other grid axes
    const int64_t per_inst = std::max<int64_t>(1, (int64_t)num_sms() * 8 / bt.B);
    const unsigned gx = (unsigned)std::min<int64_t>(pb.tiles, per_inst);
    k_permute2<uint32_t><<<dim3(gx, 1, bt.B), 256, 0, st>>>(pb, (const uint32_t *)xin,
                                                             (uint32_t *)xout, 0, 0, bt.ib);
    if (p.P > 0 && p.rbytes == 4)
      k_permute2<uint32_t><<<dim3(gx, p.P, bt.B), 256, 0, st>>>(
          pb, (const uint32_t *)nin, (uint32_t *)nout, p.planeIn, p.planeOut, bt.ib);
    else if (p.P > 0)
      k_permute2<uint64_t><<<dim3(gx, p.P, bt.B), 256, 0, st>>>(pb, nin, nout, p.planeIn,
                                                                p.planeOut, bt.ib);
    return cudaGetLastError();
  }
  int blocks = grid_for(p.total, 256);
  k_permute<uint32_t><<<dim3(blocks, 1, bt.B), 256, 0, st>>>(p, (const uint32_t *)xin,
                                                             (uint32_t *)xout, 0, 0, bt.ib);
  if (p.P > 0 && p.rbytes == 4)
    k_permute<uint32_t><<<dim3(blocks, p.P, bt.B), 256, 0, st>>>(
        p, (const uint32_t *)nin, (uint32_t *)nout, p.planeIn, p.planeOut, bt.ib);
  else if (p.P > 0)
    k_permute<uint64_t><<<dim3(blocks, p.P, bt.B), 256, 0, st>>>(p, nin, nout, p.planeIn,
                                                                 p.planeOut, bt.ib);
  return cudaGetLastError();
}


// ---------------------------------------------------------------- fused gate chains

template <int Q> __device__ __forceinline__ int div_p(int x, int d, int sh) {
  return Q == 2 ? (x >> sh) : x / d;
}
template <int Q> __device__ __forceinline__ int mod_q(int x) { return Q == 2 ? (x & 1) : x % Q; }

// B offset (within B) of the batch digits of local index x.
template <int Q>
__device__ __forceinline__ int gate_boff(const ChainGate &g, int x) {
  int o = 0;
  if (g.nb > 0) o += mod_q<Q>(div_p<Q>(x, g.lsb[0], g.lsbh[0])) * (int)g.sBb[0];
  if (g.nb > 1) o += mod_q<Q>(div_p<Q>(x, g.lsb[1], g.lsbh[1])) * (int)g.sBb[1];
  return o;
}


// q = 2 replace gate whose B is a plain 2x2 matrix (no tile legs): the
// matrix sits in registers and pairs are moved as 2-vectors.
template <typename T>
__device__ __forceinline__ void replace2(const ChainGate &g, const T *src, T *dst, const T *sB,
                                         int tile) {
  typedef typename Vec2<T>::t V;
  const T m00 = sB[0], m01 = sB[g.sBn], m10 = sB[g.sBk], m11 = sB[g.sBk + g.sBn];
  if (g.ls == 1) {
    const V *vs = reinterpret_cast<const V *>(src);
    V *vd = reinterpret_cast<V *>(dst);
    for (int j = threadIdx.x; j < tile / 2; j += blockDim.x) {
      V v = vs[j], o;
      o.x = max(v.x + m00, v.y + m10);
      o.y = max(v.x + m01, v.y + m11);
      vd[j] = o;
    }
    return;
  }
  for (int jj = threadIdx.x; jj < tile / 4; jj += blockDim.x) {
    const int j = 2 * jj;
    const int x = ((j >> g.lsh) << (g.lsh + 1)) | (j & (g.ls - 1));
    const V a = *reinterpret_cast<const V *>(src + x);
    const V b = *reinterpret_cast<const V *>(src + x + g.ls);
    V o0, o1;
    o0.x = max(a.x + m00, b.x + m10);
    o0.y = max(a.y + m00, b.y + m10);
    o1.x = max(a.x + m01, b.x + m11);
    o1.y = max(a.y + m01, b.y + m11);
    *reinterpret_cast<V *>(dst + x) = o0;
    *reinterpret_cast<V *>(dst + x + g.ls) = o1;
  }
}

// q = 2 diagonal gate on one or two tile legs: 2 or 4 values in registers.
template <typename T>
__device__ __forceinline__ void diag2(const ChainGate &g, const T *src, T *dst, const T *sB,
                                      int tile) {
  if (g.nb == 2) {
    const T b00 = sB[0], b01 = sB[g.sBb[1]], b10 = sB[g.sBb[0]], b11 = sB[g.sBb[0] + g.sBb[1]];
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
      const int d0 = (i >> g.lsbh[0]) & 1, d1 = (i >> g.lsbh[1]) & 1;
      const T add = d0 ? (d1 ? b11 : b10) : (d1 ? b01 : b00);
      dst[i] = src[i] + add;
    }
  } else {
    const T b0 = sB[0], b1 = sB[g.sBb[0]];
    for (int i = threadIdx.x; i < tile; i += blockDim.x)
      dst[i] = src[i] + (((i >> g.lsbh[0]) & 1) ? b1 : b0);
  }
}

// Apply one gate to a tile in shared memory (src may equal dst): a replace
// gate maps each q-tuple along the replaced leg, a diagonal gate adds B.
template <typename T, int Q>
__device__ __forceinline__ void apply_gate(const ChainGate &g, const T *src, T *dst,
                                           const T *sB, int tile) {
  if (Q == 2 && g.kind == 0 && g.nb == 0) {
    replace2<T>(g, src, dst, sB, tile);
    return;
  }
  if (Q == 2 && g.kind == 1 && g.nb >= 1) {
    diag2<T>(g, src, dst, sB, tile);
    return;
  }
  if (g.kind == 0) {
    const int n = tile / Q;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int hi = div_p<Q>(j, g.ls, g.lsh);
      const int x = hi * g.ls * Q + (j - hi * g.ls);
      const int bo = gate_boff<Q>(g, x);
      T in[Q];
#pragma unroll
      for (int u = 0; u < Q; ++u) in[u] = src[x + u * g.ls];
#pragma unroll
      for (int v = 0; v < Q; ++v) {
        T best = in[0] + sB[bo + v * (int)g.sBn];
#pragma unroll
        for (int u = 1; u < Q; ++u) best = max(best, in[u] + sB[bo + u * (int)g.sBk + v * (int)g.sBn]);
        dst[x + v * g.ls] = best;
      }
    }
  } else {
    for (int i = threadIdx.x; i < tile; i += blockDim.x) dst[i] = src[i] + sB[gate_boff<Q>(g, i)];
  }
}

// Counting version: values and P residue planes (plane stride `tile`).
template <typename T, int Q, typename R>
__device__ __forceinline__ void apply_gate_count(const ChainGate &g, T *s, R *sn,
                                                 const T *sB, const R *sBn, int nBel,
                                                 int tile, int P, const PrimeSet &ps) {
  if (g.kind == 0) {
    const int n = tile / Q;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int hi = div_p<Q>(j, g.ls, g.lsh);
      const int x = hi * g.ls * Q + (j - hi * g.ls);
      const int64_t bo = gate_boff<Q>(g, x);
      T in[Q], out[Q];
#pragma unroll
      for (int u = 0; u < Q; ++u) in[u] = s[x + u * g.ls];
#pragma unroll
      for (int v = 0; v < Q; ++v) {
        T best = in[0] + sB[bo + v * g.sBn];
#pragma unroll
        for (int u = 1; u < Q; ++u) best = max(best, in[u] + sB[bo + u * g.sBk + v * g.sBn]);
        out[v] = best;
      }
      for (int pl = 0; pl < P; ++pl) {
        R *np = sn + (int64_t)pl * tile;
        const R *bp = sBn + (int64_t)pl * nBel;
        R nin[Q], nout[Q];
#pragma unroll
        for (int u = 0; u < Q; ++u) nin[u] = np[x + u * g.ls];
#pragma unroll
        for (int v = 0; v < Q; ++v) {
          R c = 0;
#pragma unroll
          for (int u = 0; u < Q; ++u) {
            const int64_t bi = bo + u * g.sBk + v * g.sBn;
            if (in[u] + sB[bi] == out[v]) c = addmodR(c, mulmodR(nin[u], bp[bi], ps.c[pl]), ps.c[pl]);
          }
          nout[v] = c;
        }
#pragma unroll
        for (int v = 0; v < Q; ++v) np[x + v * g.ls] = nout[v];
      }
#pragma unroll
      for (int v = 0; v < Q; ++v) s[x + v * g.ls] = out[v];
    }
  } else {
    for (int i = threadIdx.x; i < tile; i += blockDim.x) {
      const int64_t bo = gate_boff<Q>(g, i);
      s[i] = s[i] + sB[bo];
      for (int pl = 0; pl < P; ++pl)
        sn[(int64_t)pl * tile + i] = mulmodR(sn[(int64_t)pl * tile + i], sBn[(int64_t)pl * nBel + bo],
                                             ps.c[pl]);
    }
  }
}

// Copy every gate's B (values, and planes when P > 0) into shared memory.
template <typename T, typename R>
__device__ __forceinline__ void load_gate_operands(const ChainParams &p, const T *X,
                                                   const R *Xn, T *sB, R *sBn,
                                                   int stride_el) {
  for (int gi = 0; gi < p.ngates; ++gi) {
    const ChainGate &g = p.g[gi];
    for (int e = threadIdx.x; e < g.nBel; e += blockDim.x) {
      sB[gi * stride_el + e] = X[g.offB + e];
      for (int pl = 0; pl < p.P; ++pl)
        sBn[((int64_t)gi * p.P + pl) * stride_el + e] = Xn[g.offBn + pl * g.planeB + e];
    }
  }
}

template <int Q>
__device__ __forceinline__ int64_t tile_elem_off(const ChainParams &p, int i) {
  const int h = Q == 2 ? (i >> p.loh) : i / p.lo;
  return p.hi_off[h] + (i - h * p.lo);
}

constexpr int kGateBMax = 27;  // q^3 elements of one gate operand

template <typename T, int Q, bool COUNT, typename R = uint64_t>
__global__ void __launch_bounds__(256) k_chain(const ChainParams p, const T *__restrict__ X,
                                               const R *__restrict__ Xn,
                                               const T *__restrict__ Ax,
                                               const R *__restrict__ An,
                                               T *__restrict__ Cx, R *__restrict__ Cn,
                                               const PrimeSet ps, int64_t ib) {
  X = inst_ptr(X, ib);
  Ax = inst_ptr(Ax, ib);
  Cx = inst_ptr(Cx, ib);
  if (COUNT) {
    Xn = inst_ptr(Xn, ib);
    An = inst_ptr(An, ib);
    Cn = inst_ptr(Cn, ib);
  }
  extern __shared__ __align__(16) char smem[];
  T *s = reinterpret_cast<T *>(smem);
  T *sB = s + p.tile;
  R *sn = reinterpret_cast<R *>(
      smem + ((sizeof(T) * (p.tile + TN_CHAIN_MAX_G * kGateBMax) + 15) / 16) * 16);
  R *sBn = sn + (int64_t)p.P * p.tile;
  load_gate_operands<T, R>(p, X, Xn, sB, sBn, kGateBMax);
  for (int64_t o = blockIdx.x; o < p.outer; o += gridDim.x) {
    int64_t r = o, base = 0;
    for (int sg = p.nseg - 1; sg >= 0; --sg) {
      if (Q == 2) {
        base += (r & (p.seg_size[sg] - 1)) * p.seg_s[sg];
        r >>= p.seg_sh[sg];
      } else {
        const int64_t sz = p.seg_size[sg];
        base += (r % sz) * p.seg_s[sg];
        r /= sz;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p.tile; i += blockDim.x) {
      const int64_t off = base + tile_elem_off<Q>(p, i);
      s[i] = Ax[off];
      if (COUNT)
        for (int pl = 0; pl < p.P; ++pl) sn[(int64_t)pl * p.tile + i] = An[pl * p.planeA + off];
    }
    __syncthreads();
    for (int gi = 0; gi < p.ngates; ++gi) {
      if (COUNT)
        apply_gate_count<T, Q, R>(p.g[gi], s, sn, sB + gi * kGateBMax,
                               sBn + (int64_t)gi * p.P * kGateBMax, kGateBMax, p.tile, p.P, ps);
      else
        apply_gate<T, Q>(p.g[gi], s, s, sB + gi * kGateBMax, p.tile);
      __syncthreads();
    }
    for (int i = threadIdx.x; i < p.tile; i += blockDim.x) {
      const int64_t off = base + tile_elem_off<Q>(p, i);
      Cx[off] = s[i];
      if (COUNT)
        for (int pl = 0; pl < p.P; ++pl) Cn[pl * p.planeC + off] = sn[(int64_t)pl * p.tile + i];
    }
  }
}

size_t chain_smem_bytes(const ChainParams &p, size_t elem) {
  size_t a = ((elem * (p.tile + TN_CHAIN_MAX_G * kGateBMax) + 15) / 16) * 16;
  return a + (size_t)p.P * 8 * (p.tile + (size_t)TN_CHAIN_MAX_G * kGateBMax);
}

template <typename T, int Q, bool COUNT, typename R = uint64_t>
static cudaError_t launch_chain_t(const ChainParams &p, const char *arena, const void *Ax,
                                  const uint64_t *An, void *Cx, uint64_t *Cn, const PrimeSet &ps,
                                  const Batch &bt, cudaStream_t st) {
  size_t sm = chain_smem_bytes(p, sizeof(T));
  static size_t configured = 0;
  if (sm > 48 * 1024 && sm > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_chain<T, Q, COUNT, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    configured = sm;
  }
  const int64_t gmax = num_sms() * 8;
  int64_t blocks = p.outer < gmax ? p.outer : gmax;
  k_chain<T, Q, COUNT, R><<<dim3((unsigned)blocks, bt.B), 256, sm, st>>>(
      p, reinterpret_cast<const T *>(arena), reinterpret_cast<const R *>(arena),
      static_cast<const T *>(Ax), reinterpret_cast<const R *>(An), static_cast<T *>(Cx),
      reinterpret_cast<R *>(Cn), ps, bt.ib);
  return cudaGetLastError();
}

cudaError_t launch_rchain(Dtype dt, const ChainParams &p, const char *arena, const void *Ax,
                          void *Cx, const Batch &bt, cudaStream_t st);
cudaError_t launch_rchain_count(Dtype dt, const ChainParams &p, const char *arena,
                                const void *Ax, const uint64_t *An, void *Cx, uint64_t *Cn,
                                const PrimeSet &ps, const Batch &bt, cudaStream_t st);

cudaError_t launch_chain(Dtype dt, const ChainParams &p, const char *arena, const void *Ax,
                         const uint64_t *An, void *Cx, uint64_t *Cn, const PrimeSet &ps,
                         const Batch &bt, cudaStream_t st) {
  if (p.outer == 0) return cudaSuccess;
  if (p.mode == 1 && p.P > 0) return launch_rchain_count(dt, p, arena, Ax, An, Cx, Cn, ps, bt, st);
  if (p.mode == 1) return launch_rchain(dt, p, arena, Ax, Cx, bt, st);
  const bool c = p.P > 0;
  if (c && ps.r32) {
    if (dt == DT_F32)
      return p.q == 2 ? launch_chain_t<float, 2, true, uint32_t>(p, arena, Ax, An, Cx, Cn, ps, bt, st)
                      : launch_chain_t<float, 3, true, uint32_t>(p, arena, Ax, An, Cx, Cn, ps, bt, st);
    return p.q == 2 ? launch_chain_t<int32_t, 2, true, uint32_t>(p, arena, Ax, An, Cx, Cn, ps, bt, st)
                    : launch_chain_t<int32_t, 3, true, uint32_t>(p, arena, Ax, An, Cx, Cn, ps, bt, st);
  }
  if (dt == DT_F32) {
    if (p.q == 2) return c ? launch_chain_t<float, 2, true>(p, arena, Ax, An, Cx, Cn, ps, bt, st)
                           : launch_chain_t<float, 2, false>(p, arena, Ax, An, Cx, Cn, ps, bt, st);
    return c ? launch_chain_t<float, 3, true>(p, arena, Ax, An, Cx, Cn, ps, bt, st)
             : launch_chain_t<float, 3, false>(p, arena, Ax, An, Cx, Cn, ps, bt, st);
  }
  if (p.q == 2) return c ? launch_chain_t<int32_t, 2, true>(p, arena, Ax, An, Cx, Cn, ps, bt, st)
                         : launch_chain_t<int32_t, 2, false>(p, arena, Ax, An, Cx, Cn, ps, bt, st);
  return c ? launch_chain_t<int32_t, 3, true>(p, arena, Ax, An, Cx, Cn, ps, bt, st)
           : launch_chain_t<int32_t, 3, false>(p, arena, Ax, An, Cx, Cn, ps, bt, st);
}

// Traceback of one chain record by the whole block: reload the input tile,
// replay the gates keeping every intermediate tile, then walk back.
template <typename T, int Q>
__device__ void trace_chain(const ChainTrace &ct, const T *X, int8_t *state, int *err, char *smem,
                            int64_t *sbase) {
  const ChainParams &p = ct.p;
  T *buf = reinterpret_cast<T *>(smem);                 // (ngates + 1) tiles
  T *sB = buf + (int64_t)(p.ngates + 1) * p.tile;       // gate operands
  if (threadIdx.x == 0) {
    int64_t b = ct.offIn;
    for (int i = 0; i < ct.nout; ++i) {
      int d = state[ct.out_spin[i]];
      if (d < 0 || d >= Q) { *err = 1; d = 0; }
      b += (int64_t)d * ct.out_stride[i];
    }
    *sbase = b;
  }
  load_gate_operands<T, uint64_t>(p, X, nullptr, sB, nullptr, kGateBMax);
  __syncthreads();
  const int64_t base = *sbase;
  for (int i = threadIdx.x; i < p.tile; i += blockDim.x) buf[i] = X[base + tile_elem_off<Q>(p, i)];
  __syncthreads();
  for (int gi = 0; gi < p.ngates; ++gi) {
    apply_gate<T, Q>(p.g[gi], buf + (int64_t)gi * p.tile, buf + (int64_t)(gi + 1) * p.tile,
                     sB + gi * kGateBMax, p.tile);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int x = 0;
    for (int j = 0; j < p.t; ++j) {
      int d = state[ct.local_spin[j]];
      if (d < 0 || d >= Q) { *err = 1; d = 0; }
      x = x * Q + d;
    }
    for (int gi = p.ngates - 1; gi >= 0; --gi) {
      const ChainGate &g = p.g[gi];
      if (g.kind != 0) continue;
      const T *src = buf + (int64_t)gi * p.tile;
      const T *gB = sB + gi * kGateBMax;
      const int v = mod_q<Q>(div_p<Q>(x, g.ls, g.lsh));
      const int x0 = x - v * g.ls;
      const int64_t bo = gate_boff<Q>(g, x0);
      int bu = 0;
      T best = src[x0] + gB[bo + v * g.sBn];
      for (int u = 1; u < Q; ++u) {
        T val = src[x0 + u * g.ls] + gB[bo + u * g.sBk + v * g.sBn];
        if (val > best) { best = val; bu = u; }
      }
      state[g.kspin] = (int8_t)bu;
      x = x0 + bu * g.ls;
    }
  }
  __syncthreads();
}


// ---------------------------------------------------------------- register chains (q = 2)
//
// Gate kinds in a register chain: 0 replace on register bit J = ls, whose B
// may depend on one more leg (nb = 1); 1 a diagonal gate on one or two legs.
// A leg is a register bit (lsb >= 0) or fixed per thread (digit =
// (base >> lsbh) & 1).


// mask / fixed-digit form of leg k: digit(e) = ((e & mask) != 0) | fixed
__device__ __forceinline__ void leg_sel(const ChainGate &g, int k, int64_t base, int *mask,
                                        int *fixed) {
  if (g.lsb[k] >= 0) {
    *mask = 1 << g.lsb[k];
    *fixed = 0;
  } else {
    *mask = 0;
    *fixed = (int)((base >> g.lsbh[k]) & 1);
  }
}

template <int RB, int J, typename T>
__device__ __forceinline__ void rc_replace(T (&v)[1 << RB], const ChainGate &g, const T *sB,
                                           int64_t base) {
  // B of the replace gate for each digit w of its optional extra leg
  const int wl = g.nb > 0 ? (int)g.sBb[0] : 0;
  int wm = 0, wf = 0;
  if (g.nb > 0) leg_sel(g, 0, base, &wm, &wf);
  const T a00 = sB[0], a01 = sB[g.sBn], a10 = sB[g.sBk], a11 = sB[g.sBk + g.sBn];
  if (g.nb == 0) {
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) {
      if (e & (1 << J)) continue;
      const T a = v[e], b = v[e | (1 << J)];
      v[e] = max(a + a00, b + a10);
      v[e | (1 << J)] = max(a + a01, b + a11);
    }
    return;
  }
  const T b00 = sB[wl], b01 = sB[wl + g.sBn], b10 = sB[wl + g.sBk], b11 = sB[wl + g.sBk + g.sBn];
#pragma unroll
  for (int e = 0; e < (1 << RB); ++e) {
    if (e & (1 << J)) continue;
    const int w = ((e & wm) != 0) | wf;
    const T m00 = w ? b00 : a00, m01 = w ? b01 : a01, m10 = w ? b10 : a10, m11 = w ? b11 : a11;
    const T a = v[e], b = v[e | (1 << J)];
    v[e] = max(a + m00, b + m10);
    v[e | (1 << J)] = max(a + m01, b + m11);
  }
}

// Diagonal gate with its register legs known at compile time (K < 0: no
// register leg in that slot): every element gets one add, the value picked
// by compile-time digits.
template <int RB, int K0, int K1, typename T>
__device__ __forceinline__ void rc_diag_t(T (&v)[1 << RB], T c00, T c01, T c10, T c11) {
#pragma unroll
  for (int e = 0; e < (1 << RB); ++e) {
    const int x0 = K0 >= 0 ? (e >> (K0 < 0 ? 0 : K0)) & 1 : 0;
    const int x1 = K1 >= 0 ? (e >> (K1 < 0 ? 0 : K1)) & 1 : 0;
    v[e] = v[e] + (x0 ? (x1 ? c11 : c10) : (x1 ? c01 : c00));
  }
}

template <int RB, typename T>
__device__ __forceinline__ void rc_diag(T (&v)[1 << RB], const ChainGate &g, const T *sB,
                                        int64_t base) {
  // table over (leg0, leg1); fixed legs are collapsed per thread first
  const int s0 = (int)g.sBb[0], s1 = g.nb > 1 ? (int)g.sBb[1] : 0;
  T c00 = sB[0], c01 = sB[s1], c10 = sB[s0], c11 = sB[s0 + s1];
  int k0 = g.lsb[0], k1 = g.nb > 1 ? g.lsb[1] : -1;
  if (k0 < 0) {
    const int f = (int)((base >> g.lsbh[0]) & 1);
    c00 = f ? c10 : c00;
    c01 = f ? c11 : c01;
  }
  if (g.nb > 1 && k1 < 0) {
    const int f = (int)((base >> g.lsbh[1]) & 1);
    c00 = f ? c01 : c00;
    c10 = f ? c11 : c10;
  }
  if (g.nb < 2) k1 = -1;
  // after collapsing, a missing leg reads digit 0 (c00 / c10 for leg 1)
#define RC_D(A, B) rc_diag_t<RB, A, B>(v, c00, c01, c10, c11)
  switch ((k0 + 1) * 6 + (k1 + 1)) {
    case 0: RC_D(-1, -1); break;
    case 1: RC_D(-1, 0); break;
    case 2: RC_D(-1, 1); break;
    case 3: RC_D(-1, 2); break;
    case 4: RC_D(-1, 3); break;
    case 5: RC_D(-1, 4); break;
    case 6: RC_D(0, -1); break;
    case 8: RC_D(0, 1); break;
    case 9: RC_D(0, 2); break;
    case 10: RC_D(0, 3); break;
    case 11: RC_D(0, 4); break;
    case 12: RC_D(1, -1); break;
    case 13: RC_D(1, 0); break;
    case 15: RC_D(1, 2); break;
    case 16: RC_D(1, 3); break;
    case 17: RC_D(1, 4); break;
    case 18: RC_D(2, -1); break;
    case 19: RC_D(2, 0); break;
    case 20: RC_D(2, 1); break;
    case 22: RC_D(2, 3); break;
    case 23: RC_D(2, 4); break;
    case 24: RC_D(3, -1); break;
    case 25: RC_D(3, 0); break;
    case 26: RC_D(3, 1); break;
    case 27: RC_D(3, 2); break;
    case 29: RC_D(3, 4); break;
    case 30: RC_D(4, -1); break;
    case 31: RC_D(4, 0); break;
    case 32: RC_D(4, 1); break;
    case 33: RC_D(4, 2); break;
    case 34: RC_D(4, 3); break;
    default: break;
  }
#undef RC_D
}


// Offset of the tensor element of outer index tau (legs other than the
// register legs); every size and stride is a power of two.
template <typename I>
__device__ __forceinline__ I rc_base(const ChainParams &p, int64_t tau) {
  I base = 0;
  I t = (I)tau;
  for (int sg = p.nseg - 1; sg >= 0; --sg) {
    base += (t & (I)(p.seg_size[sg] - 1)) << p.seg_ssh[sg];
    t >>= p.seg_sh[sg];
  }
  return base;
}

// Every thread walks its outer indices with a two-stage pipeline: the 2^RB
// elements of the next index are copied global -> shared memory with
// cp.async (into the thread's own column of a [2^RB][threads] stage, so no
// block barrier is needed) while the current ones are transformed in
// registers and stored.  Element offsets of the register legs are built
// incrementally from the RB leg strides; I is the index type (32-bit when
// the tensor has fewer than 2^31 elements).
template <typename T, int RB, typename I, int STAGES, int MINB>
__global__ void __launch_bounds__(256, MINB) k_rchain(const ChainParams p,
                                                                  const T *__restrict__ X,
                                                                  const T *__restrict__ A,
                                                                  T *__restrict__ C, int64_t ib) {
  X = inst_ptr(X, ib);
  A = inst_ptr(A, ib);
  C = inst_ptr(C, ib);
  __shared__ T sB[TN_CHAIN_MAX_G * kGateBMax];
  extern __shared__ __align__(16) char rstage[];
  T *stage = reinterpret_cast<T *>(rstage);
  load_gate_operands<T, uint64_t>(p, X, nullptr, sB, nullptr, kGateBMax);
  __syncthreads();
  I sS[RB];
#pragma unroll
  for (int j = 0; j < RB; ++j) sS[j] = (I)p.hi_off[1 << j];
  const int nt = blockDim.x, tid = threadIdx.x;
  const int64_t step = (int64_t)gridDim.x * nt;
  int64_t tau = blockIdx.x * (int64_t)nt + tid;
  auto issue = [&](int64_t t, T *dst) {
    if (t < p.outer) {
      const T *src = A + rc_base<I>(p, t);
      I o[1 << RB];
      o[0] = 0;
#pragma unroll
      for (int e = 1; e < (1 << RB); ++e) {
        const int hb = 31 - __clz(e);
        o[e] = o[e ^ (1 << hb)] + sS[hb];
      }
#pragma unroll
      for (int e = 0; e < (1 << RB); ++e) cp_async4(dst + e * nt + tid, src + o[e]);
    }
    cp_async_commit();
  };
  auto slot = [&](int it) { return stage + (it % STAGES) * (1 << RB) * nt; };
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) issue(tau + s * step, slot(s));
  for (int it = 0; tau < p.outer; tau += step, ++it) {
    T *cur = slot(it);
    issue(tau + (STAGES - 1) * step, slot(it + STAGES - 1));
    // all but the STAGES - 1 most recent groups are complete: the current slot is ready
    if (STAGES == 3)
      asm volatile("cp.async.wait_group 2;\n" ::: "memory");
    else
      cp_async_wait_prev();
    const I bi = rc_base<I>(p, tau);
    const int64_t base = bi;
    T v[1 << RB];
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) v[e] = cur[e * nt + tid];
    for (int gi = 0; gi < p.ngates; ++gi) {
      const ChainGate &g = p.g[gi];
      const T *gB = sB + gi * kGateBMax;
      if (g.kind != 0) {
        rc_diag<RB>(v, g, gB, base);
        continue;
      }
      switch (g.ls) {
        case 0: rc_replace<RB, 0>(v, g, gB, base); break;
        case 1: rc_replace<RB, 1>(v, g, gB, base); break;
        case 2: rc_replace<RB, 2>(v, g, gB, base); break;
        case 3: rc_replace<RB, 3>(v, g, gB, base); break;
        default: rc_replace<RB, RB - 1>(v, g, gB, base); break;
      }
    }
    T *dst = C + bi;
    I o[1 << RB];
    o[0] = 0;
#pragma unroll
    for (int e = 1; e < (1 << RB); ++e) {
      const int hb = 31 - __clz(e);
      o[e] = o[e ^ (1 << hb)] + sS[hb];
    }
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) dst[o[e]] = v[e];
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---- folded register chains (q = 2, values): table gates.
//
// Tables are built once per block: value i of table gate t is the sum of its
// components, component c reading original gate cg[c]'s operand at the offset
// given by the index bits of its legs.  Components are summed in order, so
// the traceback rebuilds bit-identical tables.

// replace on register bit J with an optional extra register leg K: the
// table slice for the thread's fixed digits is lo (K digit 0) / hi (1), each
// (x=0,x'=0), (1,0), (0,1), (1,1).
template <int RB, int J, int K, typename T, typename V>
__device__ __forceinline__ void tc_rep(T (&v)[1 << RB], const V &lo, const V &hi) {
  if constexpr (J < RB && K < RB) {
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) {
      if (e & (1 << J)) continue;
      const int e1 = e | (1 << J);
      const bool k = K >= 0 ? ((e >> (K < 0 ? 0 : K)) & 1) != 0 : false;
      const T t0 = k ? hi.x : lo.x, t1 = k ? hi.y : lo.y, t2 = k ? hi.z : lo.z,
              t3 = k ? hi.w : lo.w;
      const T a = v[e], b = v[e1];
      v[e] = max(a + t0, b + t1);
      v[e1] = max(a + t2, b + t3);
    }
  }
}

// diagonal table gate on register legs J (index bit 0) and K (bit 1), -1 for
// none; rare after folding, so one body with the legs read at run time
template <int RB, typename T, typename V>
__device__ __forceinline__ void tc_diag(T (&v)[1 << RB], int code, const V &lo) {
  const int J = (code - 42) / 7 - 1, K = (code - 42) % 7 - 1;
  const int mj = J >= 0 ? 1 << J : 0, mk = K >= 0 ? 1 << K : 0;
#pragma unroll
  for (int e = 0; e < (1 << RB); ++e) {
    const bool x0 = (e & mj) != 0, x1 = (e & mk) != 0;
    v[e] = v[e] + (x1 ? (x0 ? lo.w : lo.z) : (x0 ? lo.y : lo.x));
  }
}

// dispatch: replace on J with extra leg K is code J * 7 + K + 1; diagonal
// gates are 42 + (J + 1) * 7 + K + 1
template <int RB, typename T, typename V>
__device__ __forceinline__ void tc_apply(int code, T (&v)[1 << RB], const V &lo, const V &hi) {
#define TC_R(J, K) case (J) * 7 + (K) + 1: tc_rep<RB, J, K>(v, lo, hi); break;
  switch (code) {
    TC_R(0, -1) TC_R(0, 1) TC_R(0, 2) TC_R(0, 3) TC_R(0, 4) TC_R(0, 5)
    TC_R(1, -1) TC_R(1, 0) TC_R(1, 2) TC_R(1, 3) TC_R(1, 4) TC_R(1, 5)
    TC_R(2, -1) TC_R(2, 0) TC_R(2, 1) TC_R(2, 3) TC_R(2, 4) TC_R(2, 5)
    TC_R(3, -1) TC_R(3, 0) TC_R(3, 1) TC_R(3, 2) TC_R(3, 4) TC_R(3, 5)
    TC_R(4, -1) TC_R(4, 0) TC_R(4, 1) TC_R(4, 2) TC_R(4, 3) TC_R(4, 5)
    TC_R(5, -1) TC_R(5, 0) TC_R(5, 1) TC_R(5, 2) TC_R(5, 3) TC_R(5, 4)
    default:
      if (code >= 42) tc_diag<RB>(v, code, lo);
      break;
  }
#undef TC_R
}

// final contraction on register bit J (extra leg K): state e with bit J clear
// keeps max over the bit of value + table (lo / hi by K digit: .x for digit 0,
// .y for digit 1)
template <int RB, int J, int K, typename T, typename V>
__device__ __forceinline__ void tc_con(T (&v)[1 << RB], const V &lo, const V &hi) {
  if constexpr (J < RB && K < RB) {
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) {
      if (e & (1 << J)) continue;
      const bool k = K >= 0 ? ((e >> (K < 0 ? 0 : K)) & 1) != 0 : false;
      const T t0 = k ? hi.x : lo.x, t1 = k ? hi.y : lo.y;
      v[e] = max(v[e] + t0, v[e | (1 << J)] + t1);
    }
  }
}

template <int RB, typename T, typename V>
__device__ __forceinline__ void tc_contract(int code, T (&v)[1 << RB], const V &lo, const V &hi) {
#define TC_C(J, K) case 100 + (J) * 7 + (K) + 1: tc_con<RB, J, K>(v, lo, hi); break;
  switch (code) {
    TC_C(0, -1) TC_C(0, 1) TC_C(0, 2) TC_C(0, 3) TC_C(0, 4) TC_C(0, 5)
    TC_C(1, -1) TC_C(1, 0) TC_C(1, 2) TC_C(1, 3) TC_C(1, 4) TC_C(1, 5)
    TC_C(2, -1) TC_C(2, 0) TC_C(2, 1) TC_C(2, 3) TC_C(2, 4) TC_C(2, 5)
    TC_C(3, -1) TC_C(3, 0) TC_C(3, 1) TC_C(3, 2) TC_C(3, 4) TC_C(3, 5)
    TC_C(4, -1) TC_C(4, 0) TC_C(4, 1) TC_C(4, 2) TC_C(4, 3) TC_C(4, 5)
    TC_C(5, -1) TC_C(5, 0) TC_C(5, 1) TC_C(5, 2) TC_C(5, 3) TC_C(5, 4)
    default: break;
  }
#undef TC_C
}

// digits of the fixed legs (bits of the outer index tau) -> table slice offset
// (8 values per slice)
__device__ __forceinline__ int tc_slice(const int4 &d, int64_t tau) {
  const int s0 = d.z & 0xff, s1 = (d.z >> 8) & 0xff, s2 = (d.z >> 16) & 0xff;
  const int f = (int)((tau >> s0) & 1) | ((int)((tau >> s1) & 1) << 1) |
                ((int)((tau >> s2) & 1) << 2);
  return d.y + f * 8;
}

// element offset of outer index tau in a layout whose segment shifts are ssh
template <typename I>
__device__ __forceinline__ I rc_base_l(const ChainParams &p, int64_t tau, const int32_t *ssh) {
  I base = 0;
  I t = (I)tau;
  for (int sg = p.nseg - 1; sg >= 0; --sg) {
    base += (t & (I)(p.seg_size[sg] - 1)) << ssh[sg];
    t >>= p.seg_sh[sg];
  }
  return base;
}

// The register-chain pipeline of k_rchain with table gates: the descriptor of
// gate gi+2 and the table slice of gate gi+1 are loaded while gate gi runs.
template <typename T, int RB, typename I, int STAGES, int MINB, int NT = 256>
__global__ void __launch_bounds__(NT, MINB) k_tchain(const ChainParams p,
                                                      const T *__restrict__ X,
                                                      const T *__restrict__ A,
                                                      T *__restrict__ C, int64_t ib) {
  typedef typename Vec4<T>::t V;
  X = inst_ptr(X, ib);
  A = inst_ptr(A, ib);
  C = inst_ptr(C, ib);
  __shared__ __align__(16) T sT[TN_CHAIN_MAX_G * TN_TG_TABLE];
  __shared__ int4 sD[TN_CHAIN_MAX_G + 3];
  extern __shared__ __align__(16) char rstage[];
  T *stage = reinterpret_cast<T *>(rstage);
  I sS[RB], sO[RB];   // register-leg strides in the input and in the output
#pragma unroll
  for (int j = 0; j < RB; ++j) {
    sS[j] = (I)p.hi_in[1 << j];
    sO[j] = (I)p.hi_out[1 << j];
  }
  const int nt = blockDim.x, tid = threadIdx.x;
  const int64_t step = (int64_t)gridDim.x * nt;
  int64_t tau = blockIdx.x * (int64_t)nt + tid;
  auto issue = [&](int64_t t, T *dst) {
    if (t < p.outer) {
      const T *src = A + rc_base_l<I>(p, t, p.ssh_in);
      I o[1 << RB];
      o[0] = 0;
#pragma unroll
      for (int e = 1; e < (1 << RB); ++e) {
        const int hb = 31 - __clz(e);
        o[e] = o[e ^ (1 << hb)] + sS[hb];
      }
#pragma unroll
      for (int e = 0; e < (1 << RB); ++e) cp_async4(dst + e * nt + tid, src + o[e]);
    }
    cp_async_commit();
  };
  auto slot = [&](int it) { return stage + (it % STAGES) * (1 << RB) * nt; };
  // the first inputs are in flight while the tables are built
#pragma unroll
  for (int s2 = 0; s2 < STAGES - 1; ++s2) issue(tau + s2 * step, slot(s2));
  build_tables<T>(p, X, sT);
  if (threadIdx.x < TN_CHAIN_MAX_G + 3) {
    const int k = threadIdx.x;
    int4 d = make_int4(-1, 0, 0, 0);
    if (k < p.ntg) {
      const TGate &t = p.tg[k];
      int sh[TN_TG_MAXF];
      for (int i = 0; i < TN_TG_MAXF; ++i) sh[i] = i < t.nf ? t.fsh[i] : 62;   // 0 bit
      d = make_int4(t.code, t.toff, sh[0] | (sh[1] << 8) | (sh[2] << 16), 0);
    }
    sD[k] = d;
  }
  __syncthreads();
  // a final contraction runs after the loop and halves the stored states
  const bool con = p.ntg > 0 && p.tg[p.ntg - 1].kind == 2;
  const int ntg = con ? p.ntg - 1 : p.ntg;
  const int cmask = con ? 1 << p.tg[p.ntg - 1].J : 0;
  for (int it = 0; tau < p.outer; tau += step, ++it) {
    T *cur = slot(it);
    issue(tau + (STAGES - 1) * step, slot(it + STAGES - 1));
    if (STAGES == 3)
      asm volatile("cp.async.wait_group 2;\n" ::: "memory");
    else
      cp_async_wait_prev();
    const I bi = rc_base_l<I>(p, tau, p.ssh_out);
    T v[1 << RB];
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) v[e] = cur[e * nt + tid];
    // two gates per trip: gate gi runs on (loA, hiA) while gate gi+1's slice
    // loads into (loB, hiB), and the other way round
    int4 dA = sD[0], dB = sD[1];
    int a = tc_slice(dA, tau);
    V loA = *reinterpret_cast<const V *>(sT + a), hiA = *reinterpret_cast<const V *>(sT + a + 4);
    for (int gi = 0; gi < ntg; gi += 2) {
      a = tc_slice(dB, tau);
      const V loB = *reinterpret_cast<const V *>(sT + a);
      const V hiB = *reinterpret_cast<const V *>(sT + a + 4);
      const int4 dA2 = sD[gi + 2];
      tc_apply<RB>(dA.x, v, loA, hiA);
      if (gi + 1 >= ntg) break;
      a = tc_slice(dA2, tau);
      loA = *reinterpret_cast<const V *>(sT + a);
      hiA = *reinterpret_cast<const V *>(sT + a + 4);
      const int4 dB2 = sD[gi + 3];
      tc_apply<RB>(dB.x, v, loB, hiB);
      dA = dA2;
      dB = dB2;
    }
    if (con) {
      const int4 dc = sD[ntg];
      const int ac = tc_slice(dc, tau);
      tc_contract<RB>(dc.x, v, *reinterpret_cast<const V *>(sT + ac),
                      *reinterpret_cast<const V *>(sT + ac + 4));
    }
    T *dst = C + bi;
    I o[1 << RB];
    o[0] = 0;
#pragma unroll
    for (int e = 1; e < (1 << RB); ++e) {
      const int hb = 31 - __clz(e);
      o[e] = o[e ^ (1 << hb)] + sO[hb];
    }
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e)
      if (!(e & cmask)) dst[o[e]] = v[e];
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---- counting register chains (q = 2; 4 residue planes of 61-bit primes or 7
// of 31-bit primes): every thread keeps the 2^RB values and their residues in
// registers.  A tie adds the
// counts of the tied states; the gate's own counts multiply in unless it is a
// leaf (all counts 1).

// 2^LW consecutive 4-byte words (8- or 16-byte aligned) to and from registers
template <int LW, typename W>
__device__ __forceinline__ void rcc_vload(const W *src, W *dst) {
  static_assert(sizeof(W) == 4, "vector accesses of 4-byte words");
  if constexpr (LW == 1) {
    const uint2 x = *reinterpret_cast<const uint2 *>(src);
    dst[0] = __builtin_bit_cast(W, x.x);
    dst[1] = __builtin_bit_cast(W, x.y);
  } else {
    const uint4 x = *reinterpret_cast<const uint4 *>(src);
    dst[0] = __builtin_bit_cast(W, x.x);
    dst[1] = __builtin_bit_cast(W, x.y);
    dst[2] = __builtin_bit_cast(W, x.z);
    dst[3] = __builtin_bit_cast(W, x.w);
  }
}
template <int LW, typename W>
__device__ __forceinline__ void rcc_vstore(W *dst, const W *src) {
  static_assert(sizeof(W) == 4, "vector accesses of 4-byte words");
  if constexpr (LW == 1) {
    *reinterpret_cast<uint2 *>(dst) =
        make_uint2(__builtin_bit_cast(uint32_t, src[0]), __builtin_bit_cast(uint32_t, src[1]));
  } else {
    *reinterpret_cast<uint4 *>(dst) =
        make_uint4(__builtin_bit_cast(uint32_t, src[0]), __builtin_bit_cast(uint32_t, src[1]),
                   __builtin_bit_cast(uint32_t, src[2]), __builtin_bit_cast(uint32_t, src[3]));
  }
}

template <int RB, int NP, bool UNIT, typename T, typename R>
__device__ __forceinline__ void rcc_replace(int J, T (&v)[1 << RB], R (&n)[NP][1 << RB],
                                            const ChainGate &g, const T *sB, const R *sBn,
                                            int64_t base, const PrimeSet &ps) {
  int wm = 0, wf = 0;
  if (g.nb > 0) leg_sel(g, 0, base, &wm, &wf);
  const int wl = g.nb > 0 ? (int)g.sBb[0] : 0;
#pragma unroll
  for (int e = 0; e < (1 << RB); ++e) {
    if (e & (1 << J)) continue;
    const int e1 = e | (1 << J);
    const int bo = ((((e & wm) != 0) | wf) ? wl : 0);
    const int i00 = bo, i01 = bo + (int)g.sBn, i10 = bo + (int)g.sBk, i11 = bo + (int)(g.sBk + g.sBn);
    const T a = v[e], b = v[e1];
    const T s00 = a + sB[i00], s10 = b + sB[i10], s01 = a + sB[i01], s11 = b + sB[i11];
    const T o0 = max(s00, s10), o1 = max(s01, s11);
    const bool t00 = s00 == o0, t10 = s10 == o0, t01 = s01 == o1, t11 = s11 == o1;
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) {
      const uint64_t c = ps.c[pl];
      const R na = n[pl][e], nb = n[pl][e1];
      if (UNIT) {
        // leaf operand: counts of the tied states add (at least one is tied)
        const R both = addmodR(na, nb, c);
        n[pl][e] = t00 ? (t10 ? both : na) : nb;
        n[pl][e1] = t01 ? (t11 ? both : na) : nb;
      } else {
        const R *bn = sBn + pl * kGateBMax;
        const R a0 = mulmodR(na, bn[i00], c), b0 = mulmodR(nb, bn[i10], c);
        const R a1 = mulmodR(na, bn[i01], c), b1 = mulmodR(nb, bn[i11], c);
        n[pl][e] = t00 ? (t10 ? addmodR(a0, b0, c) : a0) : b0;
        n[pl][e1] = t01 ? (t11 ? addmodR(a1, b1, c) : a1) : b1;
      }
    }
    v[e] = o0;
    v[e1] = o1;
  }
}

template <int RB, int NP, typename T, typename R>
__device__ __forceinline__ void rcc_diag(T (&v)[1 << RB], R (&n)[NP][1 << RB],
                                         const ChainGate &g, const T *sB, const R *sBn,
                                         int64_t base, const PrimeSet &ps) {
  int m0 = 0, f0 = 0, m1 = 0, f1 = 0;
  leg_sel(g, 0, base, &m0, &f0);
  if (g.nb > 1) leg_sel(g, 1, base, &m1, &f1);
  const int s0 = (int)g.sBb[0], s1 = g.nb > 1 ? (int)g.sBb[1] : 0;
#pragma unroll
  for (int e = 0; e < (1 << RB); ++e) {
    const int x0 = ((e & m0) != 0) | f0, x1 = ((e & m1) != 0) | f1;
    const int bo = x0 * s0 + x1 * s1;
    v[e] = v[e] + sB[bo];
  }
  if (g.unitB) return;
#pragma unroll
  for (int e = 0; e < (1 << RB); ++e) {
    const int x0 = ((e & m0) != 0) | f0, x1 = ((e & m1) != 0) | f1;
    const int bo = x0 * s0 + x1 * s1;
#pragma unroll
    for (int pl = 0; pl < NP; ++pl)
      n[pl][e] = mulmodR(n[pl][e], sBn[pl * kGateBMax + bo], ps.c[pl]);
  }
}

// LW > 0 (4-byte residues only): register legs 0..LW-1 sit at memory positions
// 0..LW-1 (low_legs_first), so the 2^LW states that differ in them are
// consecutive words and each array moves with one 8- or 16-byte access.
template <typename T, int RB, int NP, typename R = uint64_t, int LW = 0>
__global__ void __launch_bounds__(256, 2) k_rchain_count(const ChainParams p,
                                                         const T *__restrict__ X,
                                                         const R *__restrict__ Xn,
                                                         const T *__restrict__ A,
                                                         const R *__restrict__ An,
                                                         T *__restrict__ C,
                                                         R *__restrict__ Cn,
                                                         const PrimeSet ps, int64_t ib) {
  X = inst_ptr(X, ib);
  Xn = inst_ptr(Xn, ib);
  A = inst_ptr(A, ib);
  An = inst_ptr(An, ib);
  C = inst_ptr(C, ib);
  Cn = inst_ptr(Cn, ib);
  __shared__ T sB[TN_CHAIN_MAX_G * kGateBMax];
  __shared__ R sBn[TN_CHAIN_MAX_G * NP * kGateBMax];
  __shared__ int64_t soff[1 << RB];
  load_gate_operands<T, R>(p, X, Xn, sB, sBn, kGateBMax);
  for (int e = threadIdx.x; e < (1 << RB); e += blockDim.x) soff[e] = p.hi_off[e];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t tau = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tau < p.outer; tau += stride) {
    int64_t r = tau, base = 0;
    for (int sg = p.nseg - 1; sg >= 0; --sg) {
      base += (r & (p.seg_size[sg] - 1)) * p.seg_s[sg];
      r >>= p.seg_sh[sg];
    }
    T v[1 << RB];
    R n[NP][1 << RB];
    if constexpr (LW == 0) {
#pragma unroll
      for (int e = 0; e < (1 << RB); ++e) {
        const int64_t off = base + soff[e];
        v[e] = A[off];
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) n[pl][e] = An[pl * p.planeA + off];
      }
    } else {
#pragma unroll
      for (int e = 0; e < (1 << RB); e += 1 << LW) {
        const int64_t off = base + soff[e];
        rcc_vload<LW>(A + off, &v[e]);
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) rcc_vload<LW>(An + pl * p.planeA + off, &n[pl][e]);
      }
    }
    for (int gi = 0; gi < p.ngates; ++gi) {
      const ChainGate &g = p.g[gi];
      const T *gB = sB + gi * kGateBMax;
      const R *gBn = sBn + (int64_t)gi * NP * kGateBMax;
      if (g.kind != 0) {
        rcc_diag<RB, NP>(v, n, g, gB, gBn, base, ps);
        continue;
      }
      if (g.unitB) {
        switch (g.ls) {
          case 0: rcc_replace<RB, NP, true>(0, v, n, g, gB, gBn, base, ps); break;
          case 1: rcc_replace<RB, NP, true>(1, v, n, g, gB, gBn, base, ps); break;
          default: rcc_replace<RB, NP, true>(2, v, n, g, gB, gBn, base, ps); break;
        }
      } else {
        switch (g.ls) {
          case 0: rcc_replace<RB, NP, false>(0, v, n, g, gB, gBn, base, ps); break;
          case 1: rcc_replace<RB, NP, false>(1, v, n, g, gB, gBn, base, ps); break;
          default: rcc_replace<RB, NP, false>(2, v, n, g, gB, gBn, base, ps); break;
        }
      }
    }
    if constexpr (LW == 0) {
#pragma unroll
      for (int e = 0; e < (1 << RB); ++e) {
        const int64_t off = base + soff[e];
        C[off] = v[e];
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) Cn[pl * p.planeC + off] = n[pl][e];
      }
    } else {
#pragma unroll
      for (int e = 0; e < (1 << RB); e += 1 << LW) {
        const int64_t off = base + soff[e];
        rcc_vstore<LW>(C + off, &v[e]);
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) rcc_vstore<LW>(Cn + pl * p.planeC + off, &n[pl][e]);
      }
    }
  }
}

// Register legs of a counting chain renumbered so that the legs at memory
// positions 0 and 1 (element strides 1 and 2), where there are such, become
// legs 0 and 1 (state bits 0 and 1); returns how many lead (0..2).  The chain
// computes the same values: every gate names its legs through the new numbers.
static int low_legs_first(const ChainParams &p, ChainParams *q) {
  const int RB = p.t;
  int l0 = -1, l1 = -1;
  for (int b = 0; b < RB; ++b) {
    if (p.hi_off[1 << b] == 1) l0 = b;
    if (p.hi_off[1 << b] == 2) l1 = b;
  }
  const int lw = l0 < 0 ? 0 : l1 < 0 ? 1 : 2;
  *q = p;
  if (lw == 0) return 0;
  int perm[TN_CHAIN_MAX_T];   // old leg -> new leg
  int next = lw;
  for (int b = 0; b < RB; ++b) perm[b] = b == l0 ? 0 : (lw == 2 && b == l1) ? 1 : next++;
  for (int e = 0; e < (1 << RB); ++e) {
    int f = 0;
    for (int b = 0; b < RB; ++b)
      if ((e >> b) & 1) f |= 1 << perm[b];
    q->hi_off[f] = p.hi_off[e];
    q->hi_in[f] = p.hi_in[e];
    q->hi_out[f] = p.hi_out[e];
  }
  for (int i = 0; i < p.ngates; ++i) {
    ChainGate &g = q->g[i];
    if (g.kind == 0 || g.kind == 2) g.ls = perm[p.g[i].ls];
    for (int k = 0; k < 2 && k < g.nb; ++k)
      if (p.g[i].lsb[k] >= 0) g.lsb[k] = perm[p.g[i].lsb[k]];
  }
  return lw;
}

cudaError_t launch_rchain_count(Dtype dt, const ChainParams &p, const char *arena,
                                const void *Ax, const uint64_t *An, void *Cx, uint64_t *Cn,
                                const PrimeSet &ps, const Batch &bt, cudaStream_t st) {
  if (p.t != 3 || !((p.P == 4 && !ps.r32) || (p.P == 7 && ps.r32))) return cudaErrorInvalidValue;
  const int64_t need = (p.outer + 255) / 256;
  // vector accesses (4-byte residues): the low legs lead, and every array
  // start, plane distance and instance stride is a multiple of the vector
  ChainParams q;
  int lw = ps.r32 && !std::getenv("TN_RCC_NO_VEC") ? low_legs_first(p, &q) : 0;
  if (lw > 0) {
    const uint64_t vb = 4u << lw;
    const bool aligned = (reinterpret_cast<uintptr_t>(Ax) | reinterpret_cast<uintptr_t>(Cx) |
                          reinterpret_cast<uintptr_t>(An) | reinterpret_cast<uintptr_t>(Cn)) %
                                 vb == 0 &&
                         (uint64_t)bt.ib % vb == 0 && p.planeA % (1 << lw) == 0 &&
                         p.planeC % (1 << lw) == 0;
    if (!aligned) lw = 0;
  }
  const ChainParams &pp = lw > 0 ? q : p;
#define TN_RCC(T_, NP_, R_, LW_)                                                                 \
  do {                                                                                           \
    const int64_t blocks =                                                                       \
        wave_blocks(need, bt.B, resident_slots(k_rchain_count<T_, 3, NP_, R_, LW_>, 256, 0));    \
    k_rchain_count<T_, 3, NP_, R_, LW_><<<dim3((unsigned)blocks, bt.B), 256, 0, st>>>(           \
        pp, reinterpret_cast<const T_ *>(arena), reinterpret_cast<const R_ *>(arena),            \
        static_cast<const T_ *>(Ax), reinterpret_cast<const R_ *>(An), static_cast<T_ *>(Cx),    \
        reinterpret_cast<R_ *>(Cn), ps, bt.ib);                                                  \
  } while (0)
  if (dt == DT_F32) {
    if (!ps.r32) TN_RCC(float, 4, uint64_t, 0);
    else if (lw == 2) TN_RCC(float, 7, uint32_t, 2);
    else if (lw == 1) TN_RCC(float, 7, uint32_t, 1);
    else TN_RCC(float, 7, uint32_t, 0);
  } else {
    if (!ps.r32) TN_RCC(int32_t, 4, uint64_t, 0);
    else if (lw == 2) TN_RCC(int32_t, 7, uint32_t, 2);
    else if (lw == 1) TN_RCC(int32_t, 7, uint32_t, 1);
    else TN_RCC(int32_t, 7, uint32_t, 0);
  }
#undef TN_RCC
  return cudaGetLastError();
}

// Traceback of a register chain by one warp: lane e holds element e of the
// 2^t elements of the fixed outer index; the gates are replayed (every
// intermediate kept in shared memory) with the forward's operation order,
// then lane 0 undoes each replace gate with the first-index argmax.
// Traceback of a folded register chain: the 32 elements selected by the
// outer spins are recomputed through the table gates in a warp (the same
// sums as the forward kernel), then walked backwards through the replace
// gates; ties keep the contracted digit 0.
template <typename T>
__device__ void trace_tchain(const ChainTrace &ct, const T *X, int8_t *state, int *err, T *buf,
                             T *sT) {
  const ChainParams &p = ct.p;
  const int E = p.tile;
  build_tables<T>(p, X, sT);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    int64_t part = 0, tpart = 0;   // input offset and outer index tau of the outer spins
    for (int i = lane; i < ct.nout; i += 32) {
      int d = state[ct.out_spin[i]];
      if (d < 0 || d > 1) { *err = 1; d = 0; }
      part += (int64_t)d * ct.out_stride[i];
      tpart += (int64_t)d << ct.out_rank[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
      part += __shfl_xor_sync(0xffffffffu, part, o);
      tpart += __shfl_xor_sync(0xffffffffu, tpart, o);
    }
    const int64_t base = part, tau = tpart;
    auto slice = [&](const TGate &t) {
      int f = 0;
      for (int i = 0; i < t.nf; ++i) f |= (int)((tau >> t.fsh[i]) & 1) << i;
      return sT + t.toff + f * 8;
    };
    for (int e = lane; e < E; e += 32) buf[e] = X[ct.offIn + base + p.hi_in[e]];
    __syncwarp();
    for (int gi = 0; gi < p.ntg; ++gi) {
      const TGate &t = p.tg[gi];
      const T *src = buf + (int64_t)gi * E;
      T *dst = buf + (int64_t)(gi + 1) * E;
      const T *tab = slice(t);
      for (int e = lane; e < E; e += 32) {
        if (t.kind == 2) {   // final contraction: states with bit J clear
          if (!(e & (1 << t.J))) {
            const int k = t.K >= 0 ? (e >> t.K) & 1 : 0;
            dst[e] = max(src[e] + tab[k * 4], src[e | (1 << t.J)] + tab[k * 4 + 1]);
          }
        } else if (t.kind != 0) {
          const int x0 = t.J >= 0 ? (e >> t.J) & 1 : 0, x1 = t.K >= 0 ? (e >> t.K) & 1 : 0;
          dst[e] = src[e] + tab[x0 | (x1 << 1)];
        } else if (!(e & (1 << t.J))) {
          const int e1 = e | (1 << t.J);
          const int k = t.K >= 0 ? (e >> t.K) & 1 : 0;
          const T a = src[e], b = src[e1];
          dst[e] = max(a + tab[k * 4 + 0], b + tab[k * 4 + 1]);
          dst[e1] = max(a + tab[k * 4 + 2], b + tab[k * 4 + 3]);
        }
      }
      __syncwarp();
    }
    if (lane == 0) {
      // a final contraction's leg is not fixed yet: its digit is chosen first
      const int cj = p.ntg > 0 && p.tg[p.ntg - 1].kind == 2 ? p.tg[p.ntg - 1].J : -1;
      int x = 0;
      for (int j = 0; j < p.t; ++j) {
        if (j == cj) continue;
        int d = state[ct.local_spin[j]];
        if (d < 0 || d > 1) { *err = 1; d = 0; }
        x |= d << j;
      }
      for (int gi = p.ntg - 1; gi >= 0; --gi) {
        const TGate &t = p.tg[gi];
        if (t.kind == 2) {
          const T *src = buf + (int64_t)gi * E;
          const T *tab = slice(t);
          const int k = t.K >= 0 ? (x >> t.K) & 1 : 0;
          const T c0 = src[x] + tab[k * 4], c1 = src[x | (1 << t.J)] + tab[k * 4 + 1];
          const int u = c1 > c0 ? 1 : 0;
          state[t.kspin] = (int8_t)u;
          x |= u << t.J;
          continue;
        }
        if (t.kind != 0) continue;
        const T *src = buf + (int64_t)gi * E;
        const T *tab = slice(t);
        const int v = (x >> t.J) & 1;
        const int x0 = x & ~(1 << t.J);
        const int k = t.K >= 0 ? (x0 >> t.K) & 1 : 0;
        const T c0 = src[x0] + tab[k * 4 + v * 2 + 0];
        const T c1 = src[x0 | (1 << t.J)] + tab[k * 4 + v * 2 + 1];
        const int u = c1 > c0 ? 1 : 0;
        state[t.kspin] = (int8_t)u;
        x = x0 | (u << t.J);
      }
    }
  }
  __syncthreads();
}

template <typename T>
__device__ void trace_rchain(const ChainTrace &ct, const T *X, int8_t *state, int *err,
                             char *smem, int64_t *sbase) {
  const ChainParams &p = ct.p;
  const int E = p.tile;   // 32
  T *buf = reinterpret_cast<T *>(smem);
  T *sBg = buf + (int64_t)(p.ngates + 1) * E;   // staged gate operands
  if (p.ntg > 0) {
    trace_tchain<T>(ct, X, state, err, buf, sBg);
    return;
  }
  load_gate_operands<T, uint64_t>(p, X, nullptr, sBg, nullptr, kGateBMax);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    int64_t part = 0;
    for (int i = lane; i < ct.nout; i += 32) {
      int d = state[ct.out_spin[i]];
      if (d < 0 || d > 1) { *err = 1; d = 0; }
      part += (int64_t)d * ct.out_stride[i];
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const int64_t base = part;
    auto digit = [&](const ChainGate &g, int k, int e) {
      return g.lsb[k] >= 0 ? ((e >> g.lsb[k]) & 1) : (int)((base >> g.lsbh[k]) & 1);
    };
    for (int e = lane; e < E; e += 32) buf[e] = X[ct.offIn + base + p.hi_off[e]];
    __syncwarp();
    for (int gi = 0; gi < p.ngates; ++gi) {
      const ChainGate &g = p.g[gi];
      const T *src = buf + (int64_t)gi * E;
      T *dst = buf + (int64_t)(gi + 1) * E;
      const T *gB = sBg + gi * kGateBMax;
      if (g.kind != 0) {
        for (int e = lane; e < E; e += 32) {
          const int x0 = digit(g, 0, e), x1 = g.nb > 1 ? digit(g, 1, e) : 0;
          dst[e] = src[e] + gB[x0 * (int)g.sBb[0] + (g.nb > 1 ? x1 * (int)g.sBb[1] : 0)];
        }
      } else {
        for (int e = lane; e < E; e += 32) {
          if (e & (1 << g.ls)) continue;
          const int e1 = e | (1 << g.ls);
          const int w = g.nb > 0 ? digit(g, 0, e) : 0;
          const int bo = w * (g.nb > 0 ? (int)g.sBb[0] : 0);
          const T a = src[e], b = src[e1];
          dst[e] = max(a + gB[bo], b + gB[bo + g.sBk]);
          dst[e1] = max(a + gB[bo + g.sBn], b + gB[bo + g.sBk + g.sBn]);
        }
      }
      __syncwarp();
    }
    if (lane == 0) {
      int x = 0;
      for (int j = 0; j < p.t; ++j) {
        int d = state[ct.local_spin[j]];
        if (d < 0 || d > 1) { *err = 1; d = 0; }
        x |= d << j;
      }
      for (int gi = p.ngates - 1; gi >= 0; --gi) {
        const ChainGate &g = p.g[gi];
        if (g.kind != 0) continue;
        const T *src = buf + (int64_t)gi * E;
        const T *gB = sBg + gi * kGateBMax;
        const int v = (x >> g.ls) & 1;
        const int x0 = x & ~(1 << g.ls);
        const int w = g.nb > 0 ? digit(g, 0, x0) : 0;
        const int bo = w * (g.nb > 0 ? (int)g.sBb[0] : 0);
        const T c0 = src[x0] + gB[bo + v * g.sBn];
        const T c1 = src[x0 | (1 << g.ls)] + gB[bo + g.sBk + v * g.sBn];
        const int u = c1 > c0 ? 1 : 0;
        state[g.kspin] = (int8_t)u;
        x = x0 | (u << g.ls);
      }
    }
  }
  __syncthreads();
  (void)sbase;
}

template <typename T, int RB, typename I, int STAGES, int MINB>
static cudaError_t launch_rchain_s(const ChainParams &p, const char *arena, const void *Ax,
                                   void *Cx, int blocks, const Batch &bt, cudaStream_t st) {
  const size_t smem = (size_t)STAGES * (1 << RB) * 256 * sizeof(T);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_rchain<T, RB, I, STAGES, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (RB == 5 && p.ntg > 0) {
    static bool tconfigured = false;
    if (!tconfigured) {
      cudaError_t e = cudaFuncSetAttribute(k_tchain<T, RB, I, STAGES, MINB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      tconfigured = true;
    }
    k_tchain<T, RB, I, STAGES, MINB><<<dim3(blocks, bt.B), 256, smem, st>>>(
        p, reinterpret_cast<const T *>(arena), static_cast<const T *>(Ax), static_cast<T *>(Cx),
        bt.ib);
    return cudaGetLastError();
  }
  k_rchain<T, RB, I, STAGES, MINB><<<dim3(blocks, bt.B), 256, smem, st>>>(
      p, reinterpret_cast<const T *>(arena), static_cast<const T *>(Ax), static_cast<T *>(Cx),
      bt.ib);
  return cudaGetLastError();
}

template <typename T, int RB, typename I>
static cudaError_t launch_rchain_i(const ChainParams &p, const char *arena, const void *Ax,
                                   void *Cx, int blocks, size_t smem, const Batch &bt,
                                   cudaStream_t st) {
  (void)smem;
  static const int minb = std::getenv("TN_RCHAIN_MINB") ? std::atoi(std::getenv("TN_RCHAIN_MINB"))
                                                        : 2;
  if (RB >= 5 && minb == 3) return launch_rchain_s<T, RB, I, 2, 3>(p, arena, Ax, Cx, blocks, bt, st);
  return launch_rchain_s<T, RB, I, 2, RB >= 5 ? 2 : 4>(p, arena, Ax, Cx, blocks, bt, st);
}

template <typename T, int RB>
static cudaError_t launch_rchain_t(const ChainParams &p, const char *arena, const void *Ax,
                                   void *Cx, int blocks, size_t smem, const Batch &bt,
                                   cudaStream_t st) {
  // tensor size = outer * 2^RB elements
  if (p.outer * (int64_t(1) << RB) < (int64_t(1) << 31))
    return launch_rchain_i<T, RB, int32_t>(p, arena, Ax, Cx, blocks, smem, bt, st);
  return launch_rchain_i<T, RB, int64_t>(p, arena, Ax, Cx, blocks, smem, bt, st);
}

// six register legs (64 states per thread): blocks of 128 threads, three per SM
template <typename T, typename I>
static cudaError_t launch_tchain6(const ChainParams &p, const char *arena, const void *Ax, void *Cx,
                                  const Batch &bt, cudaStream_t st) {
  constexpr int NT = 128;
  const size_t smem = (size_t)2 * 64 * NT * sizeof(T);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_tchain<T, 6, I, 2, 3, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int64_t blocks = (p.outer + NT - 1) / NT;
  const int64_t cap = std::max<int64_t>(1, num_sms() * 3 / bt.B);
  if (blocks > cap) blocks = cap;
  k_tchain<T, 6, I, 2, 3, NT><<<dim3((unsigned)blocks, bt.B), NT, smem, st>>>(
      p, reinterpret_cast<const T *>(arena), static_cast<const T *>(Ax), static_cast<T *>(Cx),
      bt.ib);
  return cudaGetLastError();
}

cudaError_t launch_rchain(Dtype dt, const ChainParams &p, const char *arena, const void *Ax,
                          void *Cx, const Batch &bt, cudaStream_t st) {
  if (p.outer == 0) return cudaSuccess;
  if (p.t == 6) {
    if (p.ntg == 0) return cudaErrorInvalidValue;   // six legs need the folded tables
    const bool i32 = p.outer * 64 < (int64_t(1) << 31);
    if (dt == DT_F32)
      return i32 ? launch_tchain6<float, int32_t>(p, arena, Ax, Cx, bt, st)
                 : launch_tchain6<float, int64_t>(p, arena, Ax, Cx, bt, st);
    return i32 ? launch_tchain6<int32_t, int32_t>(p, arena, Ax, Cx, bt, st)
               : launch_tchain6<int32_t, int64_t>(p, arena, Ax, Cx, bt, st);
  }
  if (p.t != 4 && p.t != 5) return cudaErrorInvalidValue;
  // resident blocks only (2 or 4 per SM); each thread then pipelines several indices
  static const int minb = std::getenv("TN_RCHAIN_MINB") ? std::atoi(std::getenv("TN_RCHAIN_MINB"))
                                                        : 2;
  const int per_sm = p.t == 5 ? (minb == 3 ? 3 : 2) : 4;
  int64_t blocks = (p.outer + 255) / 256;
  const int64_t cap = std::max<int64_t>(1, num_sms() * per_sm / bt.B);
  if (blocks > cap) blocks = cap;
  const size_t smem = (size_t)2 * (1 << p.t) * 256 * 4;
  if (dt == DT_F32) {
    if (p.t == 5) return launch_rchain_t<float, 5>(p, arena, Ax, Cx, (int)blocks, smem, bt, st);
    return launch_rchain_t<float, 4>(p, arena, Ax, Cx, (int)blocks, smem, bt, st);
  }
  if (p.t == 5) return launch_rchain_t<int32_t, 5>(p, arena, Ax, Cx, (int)blocks, smem, bt, st);
  return launch_rchain_t<int32_t, 4>(p, arena, Ax, Cx, (int)blocks, smem, bt, st);
}

// ---------------------------------------------------------------- traceback

// Steps are processed in order (the host lists them top-down).  For each, the
// fixed legs select the slice of A and B, the block finds the first k that
// maximises A + B, and the contracted spins take the digits of k.
constexpr int kTraceThreads = 128;  // all threads copy records and build tables; warp 0 walks

// (value, k) pair reduction keeping the larger value, the smaller k on ties.
template <typename T>
__device__ __forceinline__ void argmax_merge(T &v, int &k, T v2, int k2) {
  if (k2 != 0x7fffffff && (k == 0x7fffffff || v2 > v || (v2 == v && k2 < k))) {
    v = v2;
    k = k2;
  }
}

// One block walks the records in order (the host lists them top-down).  The
// spin state lives in shared memory (`sst`) for the whole walk.  Plain
// records: the fixed legs select a slice of A and B, the block finds the first
// k maximising A + B and assigns the contracted spins.  Chain records:
// trace_chain above.
template <typename T, int Q>
__global__ void __launch_bounds__(kTraceThreads) k_trace(const TraceStep *__restrict__ steps,
                                                         int nsteps,
                                                         const ChainTrace *__restrict__ chains,
                                                         const char *__restrict__ arena,
                                                         int8_t *state, int nspins, int *err,
                                                         int64_t ib) {
  // one block per instance: its arena slice and its spin state
  arena += blockIdx.x * ib;
  state += (int64_t)blockIdx.x * nspins;
  extern __shared__ __align__(16) char tsmem[];
  int8_t *sst = reinterpret_cast<int8_t *>(tsmem);
  char *work = tsmem + ((nspins + 15) / 16) * 16;
  const T *X = reinterpret_cast<const T *>(arena);
  __shared__ int64_t sbase[2];
  __shared__ int serr;
  if (threadIdx.x == 0) serr = 0;
  for (int i = threadIdx.x; i < nspins; i += blockDim.x) sst[i] = state[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // records are copied into shared memory by all threads; the copy of record
  // s + 1 is in flight (registers) while record s is walked
  constexpr int kWords = (int)((sizeof(ChainTrace) + 7) / 8);
  constexpr int kPer = (kWords + kTraceThreads - 1) / kTraceThreads;
  __shared__ __align__(16) unsigned long long srec2[2][kWords];
  unsigned long long tmp[kPer];
  auto fetch = [&](int s2) {
    const int ch = steps[s2].chain;
    const unsigned long long *src = ch >= 0
        ? reinterpret_cast<const unsigned long long *>(&chains[ch])
        : reinterpret_cast<const unsigned long long *>(&steps[s2]);
    const int words = (int)((ch >= 0 ? sizeof(ChainTrace) : sizeof(TraceStep)) / 8);
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int w = threadIdx.x + i * kTraceThreads;
      tmp[i] = w < words ? src[w] : 0ull;
    }
  };
  auto put = [&](unsigned long long *dst) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int w = threadIdx.x + i * kTraceThreads;
      if (w < kWords) dst[w] = tmp[i];
    }
  };
  if (nsteps > 0) {
    fetch(0);
    put(srec2[0]);
  }
  __syncthreads();
  for (int s = 0; s < nsteps; ++s) {
    const int chain = steps[s].chain;
    unsigned long long *srec = srec2[s & 1];
    if (s + 1 < nsteps) fetch(s + 1);
    if (chain >= 0) {
      const ChainTrace &ct = *reinterpret_cast<const ChainTrace *>(srec);
      if (ct.p.mode == 1)
        trace_rchain<T>(ct, X, sst, &serr, work, &sbase[0]);
      else
        trace_chain<T, Q>(ct, X, sst, &serr, work, &sbase[0]);
      if (s + 1 < nsteps) put(srec2[(s + 1) & 1]);
      __syncthreads();
      continue;
    }
    const TraceStep &st = *reinterpret_cast<const TraceStep *>(srec);
    if (threadIdx.x < 32) {   // warp 0 alone walks plain records
      // one warp: fixed legs select the slices of A and B
      int64_t pa = 0, pb = 0;
      for (int i = lane; i < st.nfa; i += 32) {
        int d = sst[st.fa_spin[i]];
        if (d < 0 || d >= Q) { serr = 1; d = 0; }
        pa += (int64_t)d * st.fa_stride[i];
      }
      if (st.offB >= 0)
        for (int i = lane; i < st.nfb; i += 32) {
          int d = sst[st.fb_spin[i]];
          if (d < 0 || d >= Q) { serr = 1; d = 0; }
          pb += (int64_t)d * st.fb_stride[i];
        }
      for (int o = 16; o > 0; o >>= 1) {
        pa += __shfl_xor_sync(0xffffffffu, pa, o);
        pb += __shfl_xor_sync(0xffffffffu, pb, o);
      }
      const int64_t ba = st.offA + pa, bb = st.offB + pb;
      T best = Lim<T>::neg();
      int bk = 0x7fffffff;
      for (int k = lane; k < st.Ks; k += 32) {
        int64_t oa = ba, ob = bb;
        int r = k;
        for (int j = st.nk - 1; j >= 0; --j) {
          const int d = r % Q;
          r /= Q;
          oa += d * st.k_sA[j];
          ob += d * st.k_sB[j];
        }
        T v = X[oa];
        if (st.offB >= 0) v = v + X[ob];
        argmax_merge(best, bk, v, k);
      }
      for (int o = 16; o > 0; o >>= 1) {
        T v2 = __shfl_xor_sync(0xffffffffu, best, o);
        int k2 = __shfl_xor_sync(0xffffffffu, bk, o);
        argmax_merge(best, bk, v2, k2);
      }
      if (lane == 0) {
        int r = bk;
        for (int j = st.nk - 1; j >= 0; --j) {
          sst[st.k_spin[j]] = (int8_t)(r % Q);
          r /= Q;
        }
      }
    }
    if (s + 1 < nsteps) put(srec2[(s + 1) & 1]);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nspins; i += blockDim.x) state[i] = sst[i];
  if (threadIdx.x == 0 && serr) *err = 1;
}

size_t trace_smem_bytes(const ChainParams &p, size_t elem) {
  if (p.mode == 1)
    return elem * ((size_t)(p.ngates + 1) * p.tile + (size_t)TN_CHAIN_MAX_G * TN_TG_TABLE);
  return elem * ((size_t)(p.ngates + 1) * p.tile + (size_t)TN_CHAIN_MAX_G * kGateBMax);
}

size_t trace_state_bytes(int nspins) { return ((size_t)(nspins + 15) / 16) * 16; }

template <typename T, int Q>
static cudaError_t launch_trace_t(const TraceStep *d_steps, int nsteps, const ChainTrace *chains,
                                  size_t smem, const char *arena, int8_t *state, int nspins,
                                  int *err, const Batch &bt, cudaStream_t st) {
  smem += trace_state_bytes(nspins);
  static size_t configured = 0;
  // static shared memory (two record buffers) comes on top: raise the dynamic
  // limit whenever a larger request arrives, not only past 48 KB
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_trace<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  k_trace<T, Q><<<bt.B, kTraceThreads, smem, st>>>(d_steps, nsteps, chains, arena, state, nspins,
                                                   err, bt.ib);
  return cudaGetLastError();
}

cudaError_t launch_trace(Dtype dt, int q, const TraceStep *d_steps, int nsteps,
                         const ChainTrace *d_chains, size_t smem, const char *arena, int8_t *state,
                         int nspins, int *err, const Batch &bt, cudaStream_t st) {
  if (nsteps == 0) return cudaSuccess;
  if (dt == DT_F32)
    return q == 2 ? launch_trace_t<float, 2>(d_steps, nsteps, d_chains, smem, arena, state, nspins,
                                             err, bt, st)
                  : launch_trace_t<float, 3>(d_steps, nsteps, d_chains, smem, arena, state, nspins,
                                             err, bt, st);
  return q == 2 ? launch_trace_t<int32_t, 2>(d_steps, nsteps, d_chains, smem, arena, state, nspins,
                                             err, bt, st)
                : launch_trace_t<int32_t, 3>(d_steps, nsteps, d_chains, smem, arena, state, nspins,
                                             err, bt, st);
}

// ---------------------------------------------------------------- gradient / output

__global__ void k_grad(int q, int n, int m, const int32_t *eu, const int32_t *ev,
                       const int8_t *state, float *dJ, float *dh) {
  state += (int64_t)blockIdx.y * n;
  if (dJ) dJ += (int64_t)blockIdx.y * m;
  if (dh) dh += (int64_t)blockIdx.y * n;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m && dJ) {
    int a = state[eu[t]], b = state[ev[t]];
    float g;
    if (q == 2) g = -(float)((1 - 2 * a) * (1 - 2 * b));
    else g = (a == b) ? -1.f : 0.f;
    dJ[t] = g;
  }
  if (t < n && dh) dh[t] = (q == 2) ? -(float)(1 - 2 * state[t]) : 0.f;
}

cudaError_t launch_grad(int q, int n, int m, const int32_t *eu, const int32_t *ev,
                        const int8_t *state, float *dJ, float *dh, int B, cudaStream_t st) {
  int64_t tot = n > m ? n : m;
  if (tot == 0) return cudaSuccess;
  k_grad<<<dim3((unsigned)((tot + 255) / 256), B), 256, 0, st>>>(q, n, m, eu, ev, state, dJ, dh);
  return cudaGetLastError();
}

__global__ void k_state_out(int q, int n, const int8_t *state, int8_t *out) {
  state += (int64_t)blockIdx.y * n;
  out += (int64_t)blockIdx.y * n;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (q == 2) ? (int8_t)(1 - 2 * state[t]) : state[t];
}

cudaError_t launch_state_out(int q, int n, const int8_t *state, int8_t *out, int B,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_state_out<<<dim3((n + 255) / 256, B), 256, 0, st>>>(q, n, state, out);
  return cudaGetLastError();
}

}  // namespace tn
