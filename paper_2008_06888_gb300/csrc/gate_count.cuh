// gate_count.cuh -- counting gate contractions with compile-time shapes.  The
// kernel template is instantiated in gate_count_i32.cu and gate_count_f32.cu
// (translation units of their own, compiled in parallel with kernels.cu); the
// forms cover the steps of the counting plans with 4-byte residue planes (7
// planes, or 1 in the per-pass counts).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdlib>

#include "kernels.h"
#include "chain_dev.cuh"
#include "modarith.cuh"

namespace tn {

// Counting gate contraction with compile-time K, N and plane count: two outer
// indices per thread; every value and residue of A (and of B, unless its counts
// are all 1) is loaded before any is compared, then the counts of the maximal
// k add up (ties) with predicated modular products.
// Four consecutive 4-byte words (16-byte aligned) stored with one access.
template <typename W>
__device__ __forceinline__ void gtc_store4(W *dst, const W *src) {
  static_assert(sizeof(W) == 4, "4-byte words");
  *reinterpret_cast<uint4 *>(dst) =
      make_uint4(__builtin_bit_cast(uint32_t, src[0]), __builtin_bit_cast(uint32_t, src[1]),
                 __builtin_bit_cast(uint32_t, src[2]), __builtin_bit_cast(uint32_t, src[3]));
}

// VC: the NS outputs of an outer index are NS consecutive words of C (and of
// each plane), so every four of them are stored with one 16-byte access.
template <typename T, int KS, int NS, int P, typename R, bool VC = false>
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
    // output n of outer index u: the max over k and the counts of the tied k
    auto out_one = [&](int u, int n, T &best, R (&cnt)[P]) {
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
      best = v[0];
#pragma unroll
      for (int k = 1; k < KS; ++k) best = max(best, v[k]);
#pragma unroll
      for (int i = 0; i < P; ++i) {
        R c = 0;
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          if (v[k] == best) {
            const R t = mulB ? mulmodR(na[u][i][k], bn[i][k], ps.c[i]) : na[u][i][k];
            c = addmodR(c, t, ps.c[i]);
          }
        }
        cnt[i] = c;
      }
    };
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!live[u]) continue;
      if constexpr (VC) {
#pragma unroll
        for (int n0 = 0; n0 < NS; n0 += 4) {
          T best4[4];
          R cnt4[P][4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            R cnt[P];
            out_one(u, n0 + j, best4[j], cnt);
#pragma unroll
            for (int i = 0; i < P; ++i) cnt4[i][j] = cnt[i];
          }
          const int64_t c = oc[u] + n0;
          gtc_store4(C + c, best4);
#pragma unroll
          for (int i = 0; i < P; ++i) gtc_store4(nC + i * p.planeC + c, cnt4[i]);
        }
      } else {
#pragma unroll
        for (int n = 0; n < NS; ++n) {
          T best;
          R cnt[P];
          out_one(u, n, best, cnt);
          const int64_t c = oc[u] + p.nC[n];
          C[c] = best;
#pragma unroll
          for (int i = 0; i < P; ++i) nC[i * p.planeC + c] = cnt[i];
        }
      }
    }
  }
}

template <typename T, typename R>
bool launch_gate_tc_r(const GateParams &p, const T *A, const T *B, T *C, const R *nA,
                             const R *nB, R *nC, const PrimeSet &ps, dim3 blocks, int64_t ib,
                             bool vc, cudaStream_t st) {
#define TN_GTC(KS_, NS_, P_)                                                                  \
  if (p.Ks == KS_ && p.Ns == NS_ && p.P == P_) {                                              \
    k_gate_tc<T, KS_, NS_, P_, R><<<blocks, 256, 0, st>>>(p, A, B, C, nA, nB, nC, ps, ib);   \
    return true;                                                                            \
  }
#define TN_GTC_P(P_)                                                                          \
  TN_GTC(1, 1, P_) TN_GTC(1, 2, P_) TN_GTC(2, 1, P_) TN_GTC(1, 4, P_) TN_GTC(2, 4, P_)        \
  TN_GTC(2, 16, P_)
  if (vc && p.Ks == 2 && p.Ns == 16 && (p.P == 7 || p.P == 1)) {
    if (p.P == 7)
      k_gate_tc<T, 2, 16, 7, R, true><<<blocks, 256, 0, st>>>(p, A, B, C, nA, nB, nC, ps, ib);
    else
      k_gate_tc<T, 2, 16, 1, R, true><<<blocks, 256, 0, st>>>(p, A, B, C, nA, nB, nC, ps, ib);
    return true;
  }
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
  // 16-byte output stores: the outputs of an outer index are consecutive words,
  // and every output start, plane distance and instance stride is a multiple
  // of four words
  bool vc = p.Ns % 4 == 0 && !std::getenv("TN_GATE_TC_NO_VEC") &&
            (reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(nC)) % 16 == 0 &&
            (uint64_t)bt.ib % 16 == 0 && p.planeC % 4 == 0;
  for (int n = 0; vc && n < p.Ns; ++n) vc = p.nC[n] == n;
  for (int s = 0; vc && s < p.nseg; ++s) vc = p.seg_sC[s] % 4 == 0;
  return launch_gate_tc_r<T, uint32_t>(p, A, B, C, nA, nB, nC, ps, dim3((unsigned)nb, bt.B), bt.ib,
                                       vc, st);
}

}  // namespace tn
