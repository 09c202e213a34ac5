// gate_count.cuh -- counting gate contractions with compile-time shapes.  The
// kernel template is instantiated in gate_count_i32.cu and gate_count_f32.cu
// (translation units of their own, compiled in parallel with kernels.cu); the
// forms cover the steps of the counting plans with 4-byte residue planes (7
// planes, or 1 in the per-pass counts).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "chain_dev.cuh"
#include "modarith.cuh"

namespace tn {

// Counting gate contraction with compile-time K, N and plane count: two outer
// indices per thread; every value and residue of A (and of B, unless its counts
// are all 1) is loaded before any is compared, then the counts of the maximal
// k add up (ties) with predicated modular products.
template <typename T, int KS, int NS, int P, typename R>
__global__ void __launch_bounds__(256) k_gate_tc(const GateParams p, const T *__restrict__ A,
                                                 const T *__restrict__ B, T *__restrict__ C,
                                                 const R *__restrict__ nA,
                                                 const R *__restrict__ nB, R *__restrict__ nC,
                                                 const PrimeSet ps, int64_t ib) {
  A = inst_ptr(A, ib);
  C = inst_ptr(C, ib);
  nA = inst_ptr(nA, ib);
  nC = inst_ptr(nC, ib);
  if (p.hasB) {
    B = inst_ptr(B, ib);
    nB = inst_ptr(nB, ib);
  }
  const bool mulB = p.hasB && !p.unitB;
  int64_t kA[KS], kB[KS];
#pragma unroll
  for (int k = 0; k < KS; ++k) { kA[k] = p.kA[k]; kB[k] = p.kB[k]; }
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
    R na[2][P][KS];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        const int64_t e = live[u] ? oa[u] + kA[k] : 0;
        a[u][k] = A[e];
#pragma unroll
        for (int i = 0; i < P; ++i) na[u][i][k] = nA[i * p.planeA + e];
      }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!live[u]) continue;
#pragma unroll
      for (int n = 0; n < NS; ++n) {
        const int64_t nb = p.nB[n];
        T v[KS];
        R bn[P][KS];
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          const int64_t e = ob[u] + kB[k] + nb;
          v[k] = a[u][k] + (p.hasB ? B[e] : T(0));
#pragma unroll
          for (int i = 0; i < P; ++i) bn[i][k] = mulB ? nB[i * p.planeB + e] : R(1);
        }
        T best = v[0];
#pragma unroll
        for (int k = 1; k < KS; ++k) best = max(best, v[k]);
        const int64_t c = oc[u] + p.nC[n];
        C[c] = best;
#pragma unroll
        for (int i = 0; i < P; ++i) {
          R cnt = 0;
#pragma unroll
          for (int k = 0; k < KS; ++k) {
            if (v[k] == best) {
              const R t = mulB ? mulmodR(na[u][i][k], bn[i][k], ps.c[i]) : na[u][i][k];
              cnt = addmodR(cnt, t, ps.c[i]);
            }
          }
          nC[i * p.planeC + c] = cnt;
        }
      }
    }
  }
}

template <typename T, typename R>
bool launch_gate_tc_r(const GateParams &p, const T *A, const T *B, T *C, const R *nA,
                             const R *nB, R *nC, const PrimeSet &ps, dim3 blocks, int64_t ib,
                             cudaStream_t st) {
#define TN_GTC(KS_, NS_, P_)                                                                  \
  if (p.Ks == KS_ && p.Ns == NS_ && p.P == P_) {                                              \
    k_gate_tc<T, KS_, NS_, P_, R><<<blocks, 256, 0, st>>>(p, A, B, C, nA, nB, nC, ps, ib);   \
    return true;                                                                            \
  }
#define TN_GTC_P(P_)                                                                          \
  TN_GTC(1, 1, P_) TN_GTC(1, 2, P_) TN_GTC(2, 1, P_) TN_GTC(1, 4, P_) TN_GTC(2, 4, P_)        \
  TN_GTC(2, 16, P_)
  TN_GTC_P(1)
  TN_GTC_P(7)
#undef TN_GTC_P
#undef TN_GTC
  return false;
}

// launch the form of `p` with 4-byte planes; false when there is none
template <typename T>
bool launch_gate_tc_typed(const GateParams &p, const T *A, const T *B, T *C, const uint32_t *nA,
                          const uint32_t *nB, uint32_t *nC, const PrimeSet &ps, const Batch &bt,
                          cudaStream_t st) {
  int64_t nb = ((p.outer + 1) / 2 + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 32;
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  return launch_gate_tc_r<T, uint32_t>(p, A, B, C, nA, nB, nC, ps, dim3((unsigned)nb, bt.B), bt.ib,
                                       st);
}

}  // namespace tn
