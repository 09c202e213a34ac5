// kernels.cu -- CUDA kernels of the tropical contraction (sm_103a).
//
// Element algebra (Eq. 2): (+) = max, (.) = +.  Counting tuples (Sec. II):
// (x1, n1) (.) (x2, n2) = (x1 + x2, n1 n2); (+) keeps the larger x and adds
// the counts on a tie.  Counts are residues modulo 61-bit primes 2^61 - c.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kernels.h"

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

static constexpr uint64_t M61 = (1ull << 61) - 1;

// a * b mod p for p = 2^61 - c, a, b < p, c < 2^10.  The 122-bit product is
// folded twice with 2^61 = c (mod p) (pseudo-Mersenne reduction, Crandall 1992).
__device__ __forceinline__ uint64_t mulmod61(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t lo = a * b;
  uint64_t hi = __umul64hi(a, b);
  uint64_t x1 = (hi << 3) | (lo >> 61);   // product >> 61, < 2^61
  uint64_t x0 = lo & M61;
  uint64_t t_lo = x1 * c;
  uint64_t t_hi = __umul64hi(x1, c);
  uint64_t y_lo = t_lo + x0;
  uint64_t y_hi = t_hi + (y_lo < t_lo ? 1ull : 0ull);
  uint64_t y1 = (y_hi << 3) | (y_lo >> 61);  // < 2^11
  uint64_t z = y1 * c + (y_lo & M61);        // < 2^61 + 2^21 < 2p
  uint64_t p = M61 + 1 - c;
  return z >= p ? z - p : z;
}

__device__ __forceinline__ uint64_t addmod61(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t p = M61 + 1 - c;
  uint64_t s = a + b;
  return s >= p ? s - p : s;
}

static inline int grid_for(int64_t n, int threads, int max_blocks = 152 * 32) {
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
template <typename T>
__global__ void k_leaves(const LeafDesc *__restrict__ d, int nleaves, int q,
                         const float *__restrict__ J, const float *__restrict__ h, char *arena,
                         int P) {
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
    uint64_t *n = reinterpret_cast<uint64_t *>(arena + L.off_n);
    for (int i = 0; i < P; ++i) n[i * L.plane + idx] = 1ull;
  }
}

cudaError_t launch_leaves(Dtype dt, int q, const LeafDesc *d_leaves, int nleaves, const float *J,
                          const float *h, char *arena, int P, cudaStream_t st) {
  if (nleaves == 0) return cudaSuccess;
  int64_t total = (int64_t)nleaves * q * q;
  int threads = 256;
  int blocks = (int)((total + threads - 1) / threads);
  if (dt == DT_F32)
    k_leaves<float><<<blocks, threads, 0, st>>>(d_leaves, nleaves, q, J, h, arena, P);
  else
    k_leaves<int32_t><<<blocks, threads, 0, st>>>(d_leaves, nleaves, q, J, h, arena, P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- gate contraction

// C[o, n] = max_k A[o, k] + B[o, k, n], one outer index per thread.
template <typename T, bool COUNT>
__global__ void __launch_bounds__(256) k_gate(const GateParams p, const T *__restrict__ A,
                                              const T *__restrict__ B, T *__restrict__ C,
                                              const uint64_t *__restrict__ nA,
                                              const uint64_t *__restrict__ nB,
                                              uint64_t *__restrict__ nC, const PrimeSet ps) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < p.outer; o += stride) {
    int64_t r = o, oa = 0, ob = 0, oc = 0;
    for (int s = p.nseg - 1; s >= 0; --s) {
      int64_t sz = p.seg_size[s];
      int64_t i = r % sz;
      r /= sz;
      oa += i * p.seg_sA[s];
      ob += i * p.seg_sB[s];
      oc += i * p.seg_sC[s];
    }
    for (int n = 0; n < p.Ns; ++n) {
      T best = Lim<T>::neg();
      uint64_t cnt[TN_MAX_PRIMES];
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
                uint64_t na = nA[i * p.planeA + oa + p.kA[k]];
                uint64_t t = p.hasB ? mulmod61(na, nB[i * p.planeB + ob + p.kB[k] + p.nB[n]], ps.c[i])
                                    : na;
                cnt[i] = gt ? t : addmod61(cnt[i], t, ps.c[i]);
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

cudaError_t launch_gate(Dtype dt, const GateParams &p, const void *xA, const void *xB, void *xC,
                        const uint64_t *nA, const uint64_t *nB, uint64_t *nC, const PrimeSet &ps,
                        cudaStream_t st) {
  if (p.outer == 0) return cudaSuccess;
  int threads = 256;
  int blocks = grid_for(p.outer, threads);
  bool cnt = p.P > 0;
  if (dt == DT_F32) {
    if (cnt)
      k_gate<float, true><<<blocks, threads, 0, st>>>(p, (const float *)xA, (const float *)xB,
                                                      (float *)xC, nA, nB, nC, ps);
    else
      k_gate<float, false><<<blocks, threads, 0, st>>>(p, (const float *)xA, (const float *)xB,
                                                       (float *)xC, nA, nB, nC, ps);
  } else {
    if (cnt)
      k_gate<int32_t, true><<<blocks, threads, 0, st>>>(p, (const int32_t *)xA, (const int32_t *)xB,
                                                        (int32_t *)xC, nA, nB, nC, ps);
    else
      k_gate<int32_t, false><<<blocks, threads, 0, st>>>(p, (const int32_t *)xA,
                                                         (const int32_t *)xB, (int32_t *)xC, nA, nB,
                                                         nC, ps);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- tiled max-plus GEMM

// 64 x 64 output tile per block of 256 threads, 4 x 4 per thread, k slabs of
// 16 staged in shared memory.  Out-of-range operands read the tropical zero.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm(const GemmParams p, const T *__restrict__ A,
                                              const T *__restrict__ B, T *__restrict__ C) {
  constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int64_t mt = (p.M + BM - 1) / BM, nt = (p.N + BN - 1) / BN;
  const int64_t tiles = p.batch * mt * nt;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t b = t / (mt * nt);
    const int64_t rem = t % (mt * nt);
    const int64_t m0 = (rem / nt) * BM, n0 = (rem % nt) * BN;
    const T *Ab = A + b * p.sAb;
    const T *Bb = B + b * p.sBb;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = Lim<T>::neg();
    for (int64_t k0 = 0; k0 < p.K; k0 += BK) {
      for (int idx = tid; idx < BM * BK; idx += 256) {
        int m, k;
        if (p.sAm == 1) { m = idx % BM; k = idx / BM; } else { k = idx % BK; m = idx / BK; }
        int64_t gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < p.M && gk < p.K) ? Ab[gm * p.sAm + gk * p.sAk] : Lim<T>::neg();
      }
      for (int idx = tid; idx < BN * BK; idx += 256) {
        int n, k;
        if (p.sBn == 1) { n = idx % BN; k = idx / BN; } else { k = idx % BK; n = idx / BK; }
        int64_t gn = n0 + n, gk = k0 + k;
        Bs[k][n] = (gn < p.N && gk < p.K) ? Bb[gk * p.sBk + gn * p.sBn] : Lim<T>::neg();
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = max(acc[i][j], a[i] + bv[j]);
      }
      __syncthreads();
    }
    T *Cb = C + b * p.sCb;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int64_t gm = m0 + ty * TM + i, gn = n0 + tx * TN + j;
        if (gm < p.M && gn < p.N) Cb[gm * p.sCm + gn * p.sCn] = acc[i][j];
      }
  }
}

cudaError_t launch_gemm(Dtype dt, const GemmParams &p, const void *A, const void *B, void *C,
                        cudaStream_t st) {
  int64_t tiles = p.batch * ((p.M + 63) / 64) * ((p.N + 63) / 64);
  if (tiles == 0) return cudaSuccess;
  int blocks = (int)(tiles < 152 * 16 ? tiles : 152 * 16);
  if (dt == DT_F32)
    k_gemm<float><<<blocks, 256, 0, st>>>(p, (const float *)A, (const float *)B, (float *)C);
  else
    k_gemm<int32_t><<<blocks, 256, 0, st>>>(p, (const int32_t *)A, (const int32_t *)B,
                                            (int32_t *)C);
  return cudaGetLastError();
}

// Counting planes of a GEMM step: n_i[b,m,n] = sum over the k with
// A.x + B.x == C.x of A.n_i B.n_i (mod p_i).  One output per thread.
template <typename T>
__global__ void k_gemm_count(const GemmParams p, const T *__restrict__ A, const T *__restrict__ B,
                             const T *__restrict__ C, const uint64_t *__restrict__ nA,
                             const uint64_t *__restrict__ nB, uint64_t *__restrict__ nC,
                             const PrimeSet ps) {
  const int64_t total = p.batch * p.M * p.N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t % p.N, m = (t / p.N) % p.M, b = t / (p.N * p.M);
    const int64_t oa = b * p.sAb + m * p.sAm, ob = b * p.sBb + n * p.sBn;
    const int64_t oc = b * p.sCb + m * p.sCm + n * p.sCn;
    const T x = C[oc];
    uint64_t cnt[TN_MAX_PRIMES];
#pragma unroll
    for (int i = 0; i < TN_MAX_PRIMES; ++i) cnt[i] = 0;
    for (int64_t k = 0; k < p.K; ++k) {
      if (A[oa + k * p.sAk] + B[ob + k * p.sBk] == x) {
#pragma unroll
        for (int i = 0; i < TN_MAX_PRIMES; ++i)
          if (i < p.P)
            cnt[i] = addmod61(cnt[i],
                              mulmod61(nA[i * p.planeA + oa + k * p.sAk],
                                       nB[i * p.planeB + ob + k * p.sBk], ps.c[i]),
                              ps.c[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < TN_MAX_PRIMES; ++i)
      if (i < p.P) nC[i * p.planeC + oc] = cnt[i];
  }
}

cudaError_t launch_gemm_count(Dtype dt, const GemmParams &p, const void *xA, const void *xB,
                              const void *xC, const uint64_t *nA, const uint64_t *nB, uint64_t *nC,
                              const PrimeSet &ps, cudaStream_t st) {
  int64_t total = p.batch * p.M * p.N;
  if (total == 0) return cudaSuccess;
  int blocks = grid_for(total, 256);
  if (dt == DT_F32)
    k_gemm_count<float><<<blocks, 256, 0, st>>>(p, (const float *)xA, (const float *)xB,
                                                (const float *)xC, nA, nB, nC, ps);
  else
    k_gemm_count<int32_t><<<blocks, 256, 0, st>>>(p, (const int32_t *)xA, (const int32_t *)xB,
                                                  (const int32_t *)xC, nA, nB, nC, ps);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- permutation

template <typename E>
__global__ void k_permute(const PermParams p, const E *__restrict__ in, E *__restrict__ out,
                          int64_t planeIn, int64_t planeOut) {
  const E *src = in + blockIdx.y * planeIn;
  E *dst = out + blockIdx.y * planeOut;
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

cudaError_t launch_permute(const PermParams &p, const void *xin, void *xout, const uint64_t *nin,
                           uint64_t *nout, cudaStream_t st) {
  if (p.total == 0) return cudaSuccess;
  int blocks = grid_for(p.total, 256);
  k_permute<uint32_t><<<dim3(blocks, 1), 256, 0, st>>>(p, (const uint32_t *)xin, (uint32_t *)xout,
                                                       0, 0);
  if (p.P > 0)
    k_permute<uint64_t><<<dim3(blocks, p.P), 256, 0, st>>>(p, nin, nout, p.planeIn, p.planeOut);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- traceback

// Steps are processed in order (the host lists them top-down).  For each, the
// fixed legs select the slice of A and B, the block finds the first k that
// maximises A + B, and the contracted spins take the digits of k.
template <typename T>
__global__ void __launch_bounds__(256) k_trace(const TraceStep *__restrict__ steps, int nsteps,
                                               const char *__restrict__ arena, int8_t *state, int q,
                                               int *err) {
  const T *X = reinterpret_cast<const T *>(arena);
  __shared__ int64_t sbase[2];
  __shared__ T sv[256];
  __shared__ int32_t sk[256];
  for (int s = 0; s < nsteps; ++s) {
    const TraceStep &st = steps[s];
    if (threadIdx.x == 0) {
      // every fixed leg was assigned by an ancestor step; an unassigned or
      // out-of-range digit is a planning error: flag it and read index 0
      int64_t a = st.offA, b = st.offB;
      for (int i = 0; i < st.nfa; ++i) {
        int d = state[st.fa_spin[i]];
        if (d < 0 || d >= q) { *err = 1; d = 0; }
        a += (int64_t)d * st.fa_stride[i];
      }
      if (st.offB >= 0)
        for (int i = 0; i < st.nfb; ++i) {
          int d = state[st.fb_spin[i]];
          if (d < 0 || d >= q) { *err = 1; d = 0; }
          b += (int64_t)d * st.fb_stride[i];
        }
      sbase[0] = a;
      sbase[1] = b;
    }
    __syncthreads();
    const int64_t ba = sbase[0], bb = sbase[1];
    T best = Lim<T>::neg();
    int32_t bk = 0x7fffffff;
    for (int k = threadIdx.x; k < st.Ks; k += blockDim.x) {
      int64_t oa = ba, ob = bb;
      int r = k;
      for (int j = st.nk - 1; j >= 0; --j) {
        int d = r % q;
        r /= q;
        oa += d * st.k_sA[j];
        ob += d * st.k_sB[j];
      }
      T v = X[oa];
      if (st.offB >= 0) v = v + X[ob];
      if (bk == 0x7fffffff || v > best) { best = v; bk = k; }
    }
    sv[threadIdx.x] = best;
    sk[threadIdx.x] = bk;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        T v2 = sv[threadIdx.x + w];
        int32_t k2 = sk[threadIdx.x + w];
        if (k2 != 0x7fffffff &&
            (sk[threadIdx.x] == 0x7fffffff || v2 > sv[threadIdx.x] ||
             (v2 == sv[threadIdx.x] && k2 < sk[threadIdx.x]))) {
          sv[threadIdx.x] = v2;
          sk[threadIdx.x] = k2;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      int r = sk[0];
      for (int j = st.nk - 1; j >= 0; --j) {
        state[st.k_spin[j]] = (int8_t)(r % q);
        r /= q;
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_trace(Dtype dt, int q, const TraceStep *d_steps, int nsteps,
                           const char *arena, int8_t *state, int *err, cudaStream_t st) {
  if (nsteps == 0) return cudaSuccess;
  if (dt == DT_F32)
    k_trace<float><<<1, 256, 0, st>>>(d_steps, nsteps, arena, state, q, err);
  else
    k_trace<int32_t><<<1, 256, 0, st>>>(d_steps, nsteps, arena, state, q, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- gradient / output

__global__ void k_grad(int q, int n, int m, const int32_t *eu, const int32_t *ev,
                       const int8_t *state, float *dJ, float *dh) {
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
                        const int8_t *state, float *dJ, float *dh, cudaStream_t st) {
  int64_t tot = n > m ? n : m;
  if (tot == 0) return cudaSuccess;
  k_grad<<<(int)((tot + 255) / 256), 256, 0, st>>>(q, n, m, eu, ev, state, dJ, dh);
  return cudaGetLastError();
}

__global__ void k_state_out(int q, int n, const int8_t *state, int8_t *out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (q == 2) ? (int8_t)(1 - 2 * state[t]) : state[t];
}

cudaError_t launch_state_out(int q, int n, const int8_t *state, int8_t *out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_state_out<<<(n + 255) / 256, 256, 0, st>>>(q, n, state, out);
  return cudaGetLastError();
}

}  // namespace tn
